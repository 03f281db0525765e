// api.cu -- the sensai C ABI (include/sensai.h): context, device memory,
// sequencing of the Gibbs phases, host/device pointer handling, errors.
//
// Host code here only validates arguments, allocates, copies and launches;
// every arithmetic step of the sampler runs in the kernels of sweep.cu,
// dict.cu, hyper.cu and geometry.cu.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "internal.cuh"

using namespace sensai;

namespace {

thread_local std::string g_last_error;

sensai_status fail(sensai_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

}  // namespace

namespace sensai {
void record_error(const char* msg) { g_last_error = msg; }
}  // namespace sensai

struct sensai_ctx {
    int device = 0;
    Geom g{};
    sensai_params prm{};
    double a_over_K = 0, b_scaled = 0;
    int maxobs = 0, max_slots = 0;
    long long n_observed = 0;
    SweepPlan sweep_plan{};
    float* Dsl = nullptr;       // dictionary slices (streamed code sweep only)
    int64_t t = 0;
    bool frame_set = false;
    bool ge_set = false;
    bool codes_valid = false;   // m / part_s2 describe the current codes
    bool resid_valid = false;   // R / part_r2 describe the current residual
    bool resid_fresh = false;   // R is x - D W rebuilt from the state (what a code sweep starts from)
    bool r2_valid = false;      // part_r2 holds the current residual energy (for the gamma_eps draw)
    int n_r2 = 0;               // valid entries of part_r2
    int n_s2 = 0;               // valid entries of part_s2
    bool broken = false;
    FILE* trace = nullptr;               // per-iteration metrics lines (sensai_trace)
    std::vector<float> trace_clean;      // ground truth of the trace's PSNR (empty: none)
    std::vector<float> trace_rec;        // host copy of the reconstruction
    std::chrono::steady_clock::time_point trace_last{};
    cudaStream_t last_stream = nullptr;
    long long launches = 0;     // kernels launched by this context
    bool profiling = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> timed[4];  // per phase

    uint32_t* mask_bits = nullptr;
    int* imgoff = nullptr;
    uint16_t* nobs = nullptr;
    uint16_t* obs = nullptr;
    uint32_t* Ibits = nullptr;
    uint32_t* Ipre = nullptr;
    int* Icnt = nullptr;
    int* Rbase = nullptr;
    int* Ilist = nullptr;       // per pixel: patches observing it, in slot order
    int* misc = nullptr;        // [0] max observed per patch, [1] max slots per pixel
    float* x = nullptr;
    float* D = nullptr;
    float* W = nullptr;
    uint32_t* Zb = nullptr;
    float* R = nullptr;
    float* Y = nullptr;         // per-patch reconstructions, P x N
    float* Dc = nullptr;        // dictionary operands of the tensor-core reconstruction
    float* out = nullptr;       // frame-sized staging buffer
    double* pi = nullptr;
    float* lpi = nullptr;
    int* m = nullptr;
    double* part_s2 = nullptr;
    double* part_r2 = nullptr;
    double* ge_part = nullptr;  // scratch of the initial gamma_eps
    unsigned int* chunk_counter = nullptr;
    DevScalars* sc = nullptr;
    int* pos = nullptr;         // [maxobs][N] residual position of each observed pixel, by sweep slot
    int* perm = nullptr;        // [Npad] sweep slot -> patch: decreasing |Omega_i| (obs, nobs, pos, Zb by slot)
    // dense-statistics dictionary draw (gram.cu), when it applies
    bool gram = false;
    bool xlist_valid = false;   // Xlist holds the current frame's values
    float* Xlist = nullptr;     // frame value of every (pixel, observing patch) entry of Ilist
    int4* items = nullptr;      // work items: segments of the per-pixel patch lists
    long long n_items = 0;
    int gram_grid = 0;
    float* Cpart = nullptr;     // [items][128][128]
    float* Ypart = nullptr;     // [items][2][128]
    double* C64 = nullptr;      // [P][128][128]
    double* Y64 = nullptr;      // [P][128]
    int* pitem_start = nullptr; // [P + 1]
    int* pitem_idx = nullptr;   // [items]
    double* mean_acc = nullptr; // [nframe] running sum of reconstructions (sensai_mean_*)
    long long mean_count = 0;   // reconstructions in mean_acc
    bool t_on_device = false;   // kernels read the iteration index from sc->t_iter (graph capture)
    DictSpacePlan ds{};         // space-organised dictionary sweep (cooperative launch), when it runs
    ServeEngine* serve = nullptr;   // live serving engine, when started
};

namespace {

#define SENSAI_CUDA(ctx, call)                                                                   \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return cuda_failure((ctx), e_, #call, __LINE__);                 \
    } while (0)

sensai_status cuda_failure(sensai_ctx* ctx, cudaError_t e, const char* what, int line)
{
    if (ctx) ctx->broken = true;
    const sensai_status st = (e == cudaErrorMemoryAllocation) ? SENSAI_ENOMEM : SENSAI_ECUDA;
    return fail(st, "CUDA error %d (%s) at api.cu:%d in %s", (int)e, cudaGetErrorString(e), line, what);
}

// Host-side fault injection, for tests of the clean-up paths (no GPU fault):
// with SENSAI_FAULT=alloc:N in the environment, the N-th device allocation
// (1-based) of each sensai_create reports cudaErrorMemoryAllocation without
// allocating.  Armed per call and per thread.
thread_local int g_alloc_fault = 0;   // allocations left until the injected failure (0: none)

struct FaultScope {
    FaultScope()
    {
        g_alloc_fault = 0;
        const char* f = getenv("SENSAI_FAULT");
        if (f && strncmp(f, "alloc:", 6) == 0) g_alloc_fault = atoi(f + 6);
    }
    ~FaultScope() { g_alloc_fault = 0; }
};

template <typename T>
cudaError_t dalloc(T** p, size_t count)
{
    *p = nullptr;
    if (g_alloc_fault > 0 && --g_alloc_fault == 0) return cudaErrorMemoryAllocation;
    if (count == 0) count = 1;
    return cudaMalloc((void**)p, sizeof(T) * count);
}

bool is_device_pointer(const void* p)
{
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

void free_all(sensai_ctx* c)
{
    void* ptrs[] = {c->mask_bits, c->imgoff, c->nobs, c->obs, c->Ibits, c->Ipre, c->Icnt, c->Rbase, c->Ilist,
                    c->misc, c->x, c->D, c->W, c->Zb, c->R, c->Y, c->out, c->pi, c->lpi, c->m,
                    c->part_s2, c->part_r2, c->chunk_counter, c->sc, c->pos, c->Dsl, c->ge_part, c->Dc,
                    c->perm, c->mean_acc, c->Xlist, c->items, c->Cpart, c->Ypart, c->pitem_start,
                    c->pitem_idx, c->C64, c->Y64, c->sweep_plan.counter2};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c->sweep_plan.fork) cudaEventDestroy(c->sweep_plan.fork);
    if (c->sweep_plan.join) cudaEventDestroy(c->sweep_plan.join);
    if (c->sweep_plan.side) cudaStreamDestroy(c->sweep_plan.side);
    ds_free(&c->ds);
}

enum Phase { kPhaseCodes = 0, kPhaseDict = 1, kPhaseHyper = 2, kPhaseRecon = 3 };

// Event pair around one phase on its launching stream (only while profiling).
struct PhaseTimer {
    sensai_ctx* ctx;
    int phase;
    cudaStream_t s;
    cudaEvent_t start = nullptr;
    PhaseTimer(sensai_ctx* c, int ph, cudaStream_t st) : ctx(c), phase(ph), s(st)
    {
        if (!ctx->profiling) return;
        if (cudaEventCreate(&start) != cudaSuccess || cudaEventRecord(start, s) != cudaSuccess) {
            cudaGetLastError();
            start = nullptr;
        }
    }
    void stop()
    {
        if (!start) return;
        cudaEvent_t end = nullptr;
        if (cudaEventCreate(&end) == cudaSuccess && cudaEventRecord(end, s) == cudaSuccess) {
            ctx->timed[phase].emplace_back(start, end);
        } else {
            cudaGetLastError();
            cudaEventDestroy(start);
            if (end) cudaEventDestroy(end);
        }
        start = nullptr;
    }
};

void clear_timers(sensai_ctx* ctx)
{
    for (auto& v : ctx->timed) {
        for (auto& pr : v) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
        v.clear();
    }
}

sensai_status enter(sensai_ctx* ctx)
{
    if (!ctx) return fail(SENSAI_EINVAL, "null context");
    if (ctx->broken) return fail(SENSAI_ESTATE, "context unusable after an earlier CUDA error");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_failure(ctx, e, "cudaSetDevice", __LINE__);
    return SENSAI_OK;
}

sensai_status copy_frame(sensai_ctx* ctx, const float* frame, cudaStream_t s)
{
    const size_t bytes = sizeof(float) * (size_t)ctx->g.nframe;
    const cudaMemcpyKind kind = is_device_pointer(frame) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    SENSAI_CUDA(ctx, cudaMemcpyAsync(ctx->x, frame, bytes, kind, s));
    if (kind == cudaMemcpyHostToDevice) SENSAI_CUDA(ctx, cudaStreamSynchronize(s));
    ctx->frame_set = true;
    ctx->xlist_valid = false;
    ctx->resid_valid = false;
    ctx->resid_fresh = false;
    ctx->r2_valid = false;
    return SENSAI_OK;
}

sensai_status ensure_gamma_eps(sensai_ctx* ctx, cudaStream_t s)
{
    if (ctx->ge_set) return SENSAI_OK;
    SENSAI_CUDA(ctx, launch_init_gamma_eps(ctx->g, ctx->x, ctx->mask_bits, ctx->sc, ctx->ge_part, s));
    ctx->launches += 2;
    ctx->ge_set = true;
    return SENSAI_OK;
}

// R and part_r2 <- the residual x - D W rebuilt from the state.
// With the dictionary resident in shared memory this is the sweep's own
// rebuild (rebuild_kernel); a streamed dictionary takes residual_kernel, the
// same fused multiply-adds in the same order.
SweepArgs sweep_args(const sensai_ctx* ctx);

sensai_status rebuild_residual(sensai_ctx* ctx, cudaStream_t s)
{
    const SweepPlan& plan = ctx->sweep_plan;
    if (plan.slice_atoms == 0 && plan.grid > 0) {
        SENSAI_CUDA(ctx, launch_rebuild(sweep_args(ctx), ctx->maxobs, plan.grid, s));
        ctx->n_r2 = ctx->g.NW * plan.lanes;
    } else {
        SENSAI_CUDA(ctx, launch_residual(ctx->g, ctx->x, ctx->obs, ctx->nobs, ctx->perm, ctx->imgoff, ctx->D,
                                         ctx->W, ctx->pos, ctx->R, ctx->part_r2, s));
        ctx->n_r2 = ctx->g.NW;
    }
    ctx->launches += 1;
    ctx->resid_valid = true;
    ctx->resid_fresh = true;
    ctx->r2_valid = true;
    return SENSAI_OK;
}

// part_r2 describes the current residual (as the last phase left it, or rebuilt).
sensai_status ensure_r2(sensai_ctx* ctx, cudaStream_t s)
{
    if (ctx->r2_valid) return SENSAI_OK;
    return rebuild_residual(ctx, s);
}

// The current residual in R (as the last phase left it, or rebuilt).
sensai_status ensure_residual(sensai_ctx* ctx, cudaStream_t s)
{
    if (ctx->resid_valid) return SENSAI_OK;
    return rebuild_residual(ctx, s);
}

sensai_status ensure_code_stats(sensai_ctx* ctx, cudaStream_t s)
{
    if (ctx->codes_valid) return SENSAI_OK;
    SENSAI_CUDA(ctx, launch_code_stats(ctx->g, ctx->W, ctx->Zb, ctx->perm, ctx->m, ctx->part_s2, s));
    ctx->launches += 1;
    ctx->codes_valid = true;
    ctx->n_s2 = ctx->g.NW;
    return SENSAI_OK;
}

SweepArgs sweep_args(const sensai_ctx* ctx)
{
    SweepArgs a{};
    a.g = ctx->g;
    a.x = ctx->x;
    a.obs = ctx->obs;
    a.nobs = ctx->nobs;
    a.perm = ctx->perm;
    a.imgoff = ctx->imgoff;
    a.D = ctx->D;
    a.W = ctx->W;
    a.Zb = ctx->Zb;
    a.lpi = ctx->lpi;
    a.sc = ctx->sc;
    a.pos = ctx->pos;
    a.R = ctx->R;
    a.part_s2 = ctx->part_s2;
    a.part_r2 = ctx->part_r2;
    a.chunk_counter = ctx->chunk_counter;
    a.sc_out = ctx->sc;
    a.keys = philox_round_keys(ctx->prm.seed);
    a.t = (uint32_t)ctx->t;
    a.t_dev = ctx->t_on_device;
    return a;
}

DictArgs dict_args(const sensai_ctx* ctx)
{
    DictArgs a{};
    a.g = ctx->g;
    a.D = ctx->D;
    a.W = ctx->W;
    a.Ilist = ctx->Ilist;
    a.Rbase = ctx->Rbase;
    a.R = ctx->R;
    a.sc = ctx->sc;
    a.part_r2 = ctx->part_r2;
    a.seed = ctx->prm.seed;
    a.t = (uint32_t)ctx->t;
    a.t_dev = ctx->t_on_device;
    return a;
}

HyperArgs hyper_args(const sensai_ctx* ctx)
{
    HyperArgs a{};
    a.g = ctx->g;
    a.Zb = ctx->Zb;
    a.m = ctx->m;
    a.arrive = reinterpret_cast<unsigned int*>(ctx->m + ctx->g.K);
    a.part_s2 = ctx->part_s2;
    a.n_s2 = ctx->n_s2;
    a.part_r2 = ctx->part_r2;
    a.n_r2 = ctx->n_r2;
    a.n_observed = ctx->n_observed;
    a.a_over_K = ctx->a_over_K;
    a.b_scaled = ctx->b_scaled;
    a.c = ctx->prm.c;
    a.d = ctx->prm.d;
    a.e = ctx->prm.e;
    a.f = ctx->prm.f;
    a.pi = ctx->pi;
    a.lpi = ctx->lpi;
    a.sc = ctx->sc;
    a.seed = ctx->prm.seed;
    a.t = (uint32_t)ctx->t;
    a.t_dev = ctx->t_on_device;
    a.full_s = (ctx->prm.flags & SENSAI_FLAG_GAMMA_S_FULL) != 0;
    return a;
}

sensai_status run_sweep(sensai_ctx* ctx, cudaStream_t s)
{
    if (!ctx->frame_set) return fail(SENSAI_ESTATE, "no frame: call sensai_set_frame or pass a frame");
    sensai_status st = ensure_gamma_eps(ctx, s);
    if (st != SENSAI_OK) return st;
    SweepArgs a = sweep_args(ctx);
    if (ctx->R) {
        // the sweep starts from the residual rebuilt from the state (the
        // phases before it leave R updated incrementally), so its bits depend
        // on the state alone: read from R when R holds exactly that, else
        // rebuilt inside the sweep (dictionary resident in shared memory) or
        // by residual_kernel first (streamed dictionary)
        if (ctx->resid_fresh) {
            a.R_in = ctx->R;
        } else if (ctx->sweep_plan.slice_atoms != 0) {
            if ((st = rebuild_residual(ctx, s)) != SENSAI_OK) return st;
            a.R_in = ctx->R;
        }
        if (ctx->gram) a.R = nullptr;   // no phase reads the residual the sweep ends with
    }
    const SweepPlan plan = ctx->sweep_plan;
    PhaseTimer timer(ctx, kPhaseCodes, s);
    int nl = 0;
    SENSAI_CUDA(ctx, launch_code_sweep(a, plan, ctx->maxobs, ctx->Dsl, s, &nl));
    if (ctx->prm.flags & SENSAI_FLAG_GAMMA_S_FULL) {
        SENSAI_CUDA(ctx, launch_prior_s2(ctx->g, ctx->Zb, ctx->perm, ctx->sc, a.t, a.t_dev, ctx->prm.seed,
                                         plan.lanes, ctx->part_s2, s));
        ++nl;
    }
    timer.stop();
    ctx->launches += nl;
    ctx->codes_valid = true;
    ctx->resid_valid = !ctx->gram;   // R holds the sweep's final residual (not kept by gram contexts)
    ctx->resid_fresh = false;
    ctx->r2_valid = true;
    ctx->n_s2 = ctx->g.NW * plan.lanes;   // one partial per work unit
    ctx->n_r2 = ctx->g.NW * plan.lanes;
    return SENSAI_OK;
}

sensai_status run_gram(sensai_ctx* ctx, cudaStream_t s)
{
    if (!ctx->xlist_valid) {
        SENSAI_CUDA(ctx, launch_xlist(ctx->g, ctx->Ilist, ctx->Rbase, ctx->max_slots, ctx->imgoff, ctx->x,
                                      ctx->Xlist, s));
        ctx->launches += 1;
        ctx->xlist_valid = true;
    }
    GramArgs a{};
    a.g = ctx->g;
    a.W = ctx->W;
    a.Ilist = ctx->Ilist;
    a.Xlist = ctx->Xlist;
    a.items = ctx->items;
    a.n_items = ctx->n_items;
    a.Cpart = ctx->Cpart;
    a.Ypart = ctx->Ypart;
    a.pitem_start = ctx->pitem_start;
    a.pitem_idx = ctx->pitem_idx;
    a.C64 = ctx->C64;
    a.Y64 = ctx->Y64;
    a.D = ctx->D;
    a.sc = ctx->sc;
    a.seed = ctx->prm.seed;
    a.t = (uint32_t)ctx->t;
    a.t_dev = ctx->t_on_device;
    a.tf32 = (ctx->prm.flags & SENSAI_FLAG_TF32_STATISTICS) != 0;
    a.status = &ctx->sc->status;
    {
        PhaseTimer timer(ctx, kPhaseDict, s);
        SENSAI_CUDA(ctx, launch_gram(a, ctx->gram_grid, s));
        timer.stop();
    }
    ctx->launches += 3;
    // the post-draw residual for the gamma_eps draw and the next code sweep
    return rebuild_residual(ctx, s);
}

sensai_status run_dictionary(sensai_ctx* ctx, cudaStream_t s)
{
    if (!ctx->frame_set) return fail(SENSAI_ESTATE, "no frame: call sensai_set_frame or pass a frame");
    sensai_status st = ensure_gamma_eps(ctx, s);
    if (st != SENSAI_OK) return st;
    if (ctx->gram) return run_gram(ctx, s);
    st = ensure_residual(ctx, s);
    if (st != SENSAI_OK) return st;
    if (ctx->ds.grid > 0) {
        DictSpaceArgs a{};
        a.g = ctx->g;
        a.D = ctx->D;
        a.W = ctx->W;
        a.R = ctx->R;
        a.pidx = ctx->ds.pidx;
        a.np = ctx->ds.np;
        a.base = ctx->ds.base;
        a.sc = ctx->sc;
        a.part_r2 = ctx->part_r2;
        a.part = ctx->ds.part;
        a.delta = ctx->ds.delta;
        a.bar = ctx->ds.bar;
        a.own_max = ctx->ds.own_max;
        a.seed = ctx->prm.seed;
        a.t = (uint32_t)ctx->t;
        PhaseTimer timer(ctx, kPhaseDict, s);
        SENSAI_CUDA(ctx, launch_dict_space(a, ctx->ds, s));
        timer.stop();
        ctx->launches += 1;
        ctx->n_r2 = ctx->ds.grid;
        ctx->resid_fresh = false;   // updated incrementally by the draws
        ctx->r2_valid = true;
        return SENSAI_OK;
    }
    const DictArgs a = dict_args(ctx);
    PhaseTimer timer(ctx, kPhaseDict, s);
    SENSAI_CUDA(ctx, launch_dict(a, ctx->max_slots, s));
    timer.stop();
    ctx->launches += 1;
    ctx->n_r2 = ctx->g.P;
    ctx->resid_fresh = false;
    ctx->r2_valid = true;
    return SENSAI_OK;
}

sensai_status run_hyper(sensai_ctx* ctx, cudaStream_t s)
{
    if (!ctx->frame_set) return fail(SENSAI_ESTATE, "no frame: call sensai_set_frame or pass a frame");
    sensai_status st = ensure_gamma_eps(ctx, s);
    if (st != SENSAI_OK) return st;
    st = ensure_code_stats(ctx, s);
    if (st != SENSAI_OK) return st;
    st = ensure_r2(ctx, s);
    if (st != SENSAI_OK) return st;
    const HyperArgs a = hyper_args(ctx);
    PhaseTimer timer(ctx, kPhaseHyper, s);
    SENSAI_CUDA(ctx, launch_hyper(a, s));
    timer.stop();
    ctx->launches += 1;
    return SENSAI_OK;
}

sensai_status clear_codes(sensai_ctx* ctx, cudaStream_t s)
{
    SENSAI_CUDA(ctx, cudaMemsetAsync(ctx->W, 0, sizeof(float) * (size_t)ctx->g.KB * kAtomBlock * ctx->g.Npad, s));
    SENSAI_CUDA(ctx, cudaMemsetAsync(ctx->Zb, 0, sizeof(uint32_t) * (size_t)ctx->g.K * ctx->g.NW, s));
    ctx->codes_valid = false;
    ctx->resid_valid = false;
    ctx->resid_fresh = false;
    ctx->r2_valid = false;
    return SENSAI_OK;
}

sensai_status reset_state(sensai_ctx* ctx, cudaStream_t s)
{
    sensai_status st = clear_codes(ctx, s);
    if (st != SENSAI_OK) return st;
    SENSAI_CUDA(ctx, launch_init_state(ctx->g, ctx->D, ctx->pi, ctx->lpi, ctx->sc, ctx->prm.seed, s));
    ctx->launches += 2;
    ctx->t = 0;
    ctx->ge_set = false;
    return SENSAI_OK;
}

sensai_status write_out(sensai_ctx* ctx, const void* src, void* dst, size_t bytes, cudaStream_t s)
{
    const bool dev = is_device_pointer(dst);
    SENSAI_CUDA(ctx, cudaMemcpyAsync(dst, src, bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    if (!dev) SENSAI_CUDA(ctx, cudaStreamSynchronize(s));
    return SENSAI_OK;
}

}  // namespace

// One metrics line per Gibbs iteration (sensai_trace): the draws of the
// iteration just finished, its active count and sums, the host time since
// the previous line, and the PSNR of the current reconstruction against the
// ground truth when one was given.  Synchronises the stream.
sensai_status trace_iteration(sensai_ctx* ctx, cudaStream_t s, const char* mode)
{
    if (!ctx->trace) return SENSAI_OK;
    DevScalars h{};
    SENSAI_CUDA(ctx, cudaMemcpyAsync(&h, ctx->sc, sizeof h, cudaMemcpyDeviceToHost, s));
    const bool have_clean = !ctx->trace_clean.empty();
    if (have_clean) {
        SENSAI_CUDA(ctx, launch_reconstruct(ctx->g, ctx->D, ctx->Dc, ctx->W, ctx->Y, ctx->out, &ctx->sc->status, s));
        ctx->launches += reconstruct_launches(ctx->g);
        SENSAI_CUDA(ctx, cudaMemcpyAsync(ctx->trace_rec.data(), ctx->out, sizeof(float) * ctx->trace_rec.size(),
                                         cudaMemcpyDeviceToHost, s));
    }
    SENSAI_CUDA(ctx, cudaStreamSynchronize(s));
    if (h.status != 0) return fail(SENSAI_ETIMEOUT, "a device-side wait timed out (status %d)", h.status);
    char psnr[40] = "null";
    if (have_clean) {
        double se = 0.0;
        for (size_t q = 0; q < ctx->trace_rec.size(); ++q) {
            const double d = (double)ctx->trace_rec[q] - (double)ctx->trace_clean[q];
            se += d * d;
        }
        const double mse = se / (double)ctx->trace_rec.size();
        if (mse > 0.0) snprintf(psnr, sizeof psnr, "%.17g", 10.0 * std::log10(1.0 / mse));
    }
    const auto now = std::chrono::steady_clock::now();
    const double wall_ms = std::chrono::duration<double, std::milli>(now - ctx->trace_last).count();
    ctx->trace_last = now;
    fprintf(ctx->trace,
            "{\"t\": %lld, \"mode\": \"%s\", \"gamma_s\": %.17g, \"gamma_eps\": %.17g, \"active\": %lld, "
            "\"active_per_patch\": %.17g, \"sum_s2\": %.17g, \"sum_r2\": %.17g, \"psnr_db\": %s, "
            "\"wall_ms\": %.3f}\n",
            (long long)(ctx->t - 1), mode, h.gamma_s, h.gamma_eps, (long long)h.n_active,
            (double)h.n_active / (double)ctx->g.N, h.sum_s2, h.sum_r2, psnr, wall_ms);
    fflush(ctx->trace);
    return SENSAI_OK;
}

extern "C" {

const char* sensai_last_error(void) { return g_last_error.c_str(); }

sensai_status sensai_create(const sensai_params* prm, const uint8_t* mask, sensai_ctx** out)
{
    g_last_error.clear();
    const FaultScope faults;
    if (!prm || !mask || !out) return fail(SENSAI_EINVAL, "null argument");
    *out = nullptr;
    const sensai_params& p = *prm;
    if (p.ndim < 1 || p.ndim > kMaxDim) return fail(SENSAI_EINVAL, "ndim must be 1..4 (got %d)", p.ndim);
    if (p.K < 1 || p.K > 1024) return fail(SENSAI_EINVAL, "K must be 1..1024 (got %d)", p.K);
    const int known_flags = SENSAI_FLAG_STREAM_DICTIONARY | SENSAI_FLAG_CHAIN_DICTIONARY | SENSAI_FLAG_GAMMA_S_FULL |
                            SENSAI_FLAG_DENSE_STATISTICS | SENSAI_FLAG_TF32_STATISTICS | SENSAI_SLICE_ATOMS(2040);
    if ((p.flags & ~known_flags) != 0) return fail(SENSAI_EINVAL, "unknown flags 0x%x", p.flags);
    if ((p.flags & SENSAI_SLICE_ATOMS(2040)) != 0 && !(p.flags & SENSAI_FLAG_STREAM_DICTIONARY))
        return fail(SENSAI_EINVAL, "SENSAI_SLICE_ATOMS needs SENSAI_FLAG_STREAM_DICTIONARY");
    if ((p.flags & (SENSAI_FLAG_DENSE_STATISTICS | SENSAI_FLAG_TF32_STATISTICS)) != 0) {
        Geom gk{};
        gk.K = p.K;
        if (!gram_available(gk))
            return fail(SENSAI_EINVAL, "the dense-statistics dictionary form needs K <= 128 (got %d)", p.K);
        if (p.flags & SENSAI_FLAG_CHAIN_DICTIONARY)
            return fail(SENSAI_EINVAL, "the dense-statistics and per-chain dictionary forms exclude each other");
    }
    if (!(p.c > 0 && p.d > 0 && p.e > 0 && p.f > 0)) return fail(SENSAI_EINVAL, "c, d, e, f must be > 0");
    Geom g{};
    g.ndim = p.ndim;
    g.K = p.K;
    long long P = 1, N = 1, nframe = 1;
    for (int d = 0; d < p.ndim; ++d) {
        if (p.M[d] < 1 || p.B[d] < 1 || p.B[d] > p.M[d] || p.stride[d] < 1)
            return fail(SENSAI_EINVAL, "dimension %d: need 1 <= B <= M and stride >= 1", d);
        if ((p.M[d] - p.B[d]) % p.stride[d] != 0)
            return fail(SENSAI_EINVAL, "dimension %d: (M - B) = %lld not divisible by stride %d", d,
                        (long long)(p.M[d] - p.B[d]), p.stride[d]);
        g.M[d] = p.M[d];
        g.B[d] = p.B[d];
        g.S[d] = p.stride[d];
        g.G[d] = (p.M[d] - p.B[d]) / p.stride[d] + 1;
        P *= p.B[d];
        N *= g.G[d];
        nframe *= p.M[d];
    }
    if (P > 1024) return fail(SENSAI_EINVAL, "patch size P = %lld exceeds 1024", P);
    if (N >= (1LL << 31)) return fail(SENSAI_EINVAL, "too many patches (%lld)", N);
    if (nframe >= (1LL << 31)) return fail(SENSAI_EINVAL, "frame too large (%lld pixels)", nframe);
    long long s = 1;
    for (int d = p.ndim - 1; d >= 0; --d) {
        g.fs[d] = s;
        s *= g.M[d];
    }
    g.P = (int)P;
    g.N = N;
    g.NW = (int)((N + 31) / 32);
    g.Npad = (long long)g.NW * 32;
    g.KB = (p.K + kAtomBlock - 1) / kAtomBlock;
    g.nframe = nframe;

    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return cuda_failure(nullptr, e, "cudaGetDevice", __LINE__);

    sensai_ctx* ctx = new (std::nothrow) sensai_ctx();
    if (!ctx) return fail(SENSAI_ENOMEM, "host allocation failed");
    ctx->device = device;
    ctx->g = g;
    ctx->prm = p;
    ctx->a_over_K = (p.a > 0 ? p.a : (double)p.K) / p.K;
    ctx->b_scaled = (p.b > 0 ? p.b : (double)N / 8.0) * (p.K - 1) / p.K;

    const cudaStream_t st0 = nullptr;
    uint8_t* mask_dev = nullptr;
    auto bail = [&](sensai_status status) {
        if (mask_dev) cudaFree(mask_dev);
        free_all(ctx);
        delete ctx;
        return status;
    };
#define CREATE_CUDA(call)                                                             \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess) return bail(cuda_failure(nullptr, e_, #call, __LINE__)); \
    } while (0)

    const long long nmw = (nframe + 31) / 32;
    CREATE_CUDA(dalloc(&mask_dev, (size_t)nframe));
    CREATE_CUDA(dalloc(&ctx->mask_bits, (size_t)nmw));
    CREATE_CUDA(dalloc(&ctx->imgoff, (size_t)P));
    CREATE_CUDA(dalloc(&ctx->nobs, (size_t)N));
    CREATE_CUDA(dalloc(&ctx->misc, 2));
    CREATE_CUDA(cudaMemcpy(mask_dev, mask, (size_t)nframe, cudaMemcpyHostToDevice));
    CREATE_CUDA(cudaMemset(ctx->misc, 0, 2 * sizeof(int)));
    CREATE_CUDA(launch_geometry(g, mask_dev, ctx->mask_bits, ctx->imgoff, ctx->nobs, ctx->misc, nullptr, st0));
    ctx->launches += 3;
    int misc[2] = {0, 0};
    CREATE_CUDA(cudaMemcpy(misc, ctx->misc, sizeof(misc), cudaMemcpyDeviceToHost));
    cudaFree(mask_dev);
    mask_dev = nullptr;
    ctx->maxobs = misc[0];
    if (ctx->maxobs > 256) {
        fail(SENSAI_EINVAL, "a patch observes %d pixels; at most 256 observed pixels per patch are supported",
             ctx->maxobs);
        return bail(SENSAI_EINVAL);
    }
    CREATE_CUDA(dalloc(&ctx->obs, (size_t)(ctx->maxobs > 0 ? ctx->maxobs : 1) * N));
    CREATE_CUDA(dalloc(&ctx->Ibits, (size_t)P * g.NW));
    CREATE_CUDA(dalloc(&ctx->Ipre, (size_t)P * g.NW));
    CREATE_CUDA(dalloc(&ctx->Icnt, (size_t)P));
    CREATE_CUDA(dalloc(&ctx->Rbase, (size_t)P + 1));
    CREATE_CUDA(launch_slots(g, ctx->mask_bits, ctx->imgoff, ctx->obs, ctx->Ibits, ctx->Ipre, ctx->Icnt,
                             ctx->Rbase, ctx->misc + 1, st0));
    ctx->launches += 4;
    int total = 0;
    CREATE_CUDA(cudaMemcpy(&total, ctx->Rbase + P, sizeof(int), cudaMemcpyDeviceToHost));
    CREATE_CUDA(cudaMemcpy(&ctx->max_slots, ctx->misc + 1, sizeof(int), cudaMemcpyDeviceToHost));
    ctx->n_observed = total;
    // residual layout: the pairs of the space-organised dictionary sweep when
    // it runs, else the per-pixel slots of the per-chain kernel
    CREATE_CUDA(dalloc(&ctx->pos, (size_t)(ctx->maxobs > 0 ? ctx->maxobs : 1) * N));
    ctx->gram = total > 0 && (p.flags & (SENSAI_FLAG_DENSE_STATISTICS | SENSAI_FLAG_TF32_STATISTICS));
    if (!ctx->gram && !(p.flags & SENSAI_FLAG_CHAIN_DICTIONARY))
        CREATE_CUDA(ds_build(g, mask, ctx->obs, ctx->nobs, device, ctx->pos, &ctx->R, &ctx->ds, st0));
    if (ctx->ds.grid > 0) {
        ctx->launches += 2;
    } else {
        CREATE_CUDA(dalloc(&ctx->Ilist, (size_t)total));
        CREATE_CUDA(launch_ilist(g, ctx->Ibits, ctx->Ipre, ctx->Rbase, ctx->Ilist, st0));
        CREATE_CUDA(dalloc(&ctx->R, (size_t)total));
        CREATE_CUDA(launch_pos_slots(g, ctx->obs, ctx->nobs, ctx->Ibits, ctx->Ipre, ctx->Rbase, ctx->pos, st0));
        ctx->launches += 2;
    }
    if (ctx->gram) {
        // the work items: each pixel's patch list in segments of at most
        // 2048 patches (one FP32 partial per segment)
        std::vector<int> hr((size_t)P + 1);
        CREATE_CUDA(cudaMemcpy(hr.data(), ctx->Rbase, sizeof(int) * hr.size(), cudaMemcpyDeviceToHost));
        std::vector<int4> items;
        std::vector<int> ps, pi;
        gram_plan_items(hr, (int)P, 2048, &items, &ps, &pi);
        ctx->n_items = (long long)items.size();
        CREATE_CUDA(dalloc(&ctx->Xlist, (size_t)total));
        CREATE_CUDA(dalloc(&ctx->items, items.size()));
        CREATE_CUDA(dalloc(&ctx->pitem_start, ps.size()));
        CREATE_CUDA(dalloc(&ctx->pitem_idx, pi.size()));
        CREATE_CUDA(dalloc(&ctx->Cpart, items.size() * 128 * 128));
        CREATE_CUDA(dalloc(&ctx->Ypart, items.size() * 2 * 128));
        CREATE_CUDA(dalloc(&ctx->C64, (size_t)P * 128 * 128));
        CREATE_CUDA(dalloc(&ctx->Y64, (size_t)P * 128));
        CREATE_CUDA(cudaMemcpy(ctx->items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice));
        CREATE_CUDA(cudaMemcpy(ctx->pitem_start, ps.data(), sizeof(int) * ps.size(), cudaMemcpyHostToDevice));
        CREATE_CUDA(cudaMemcpy(ctx->pitem_idx, pi.data(), sizeof(int) * pi.size(), cudaMemcpyHostToDevice));
        int sms_g = 0;
        CREATE_CUDA(cudaDeviceGetAttribute(&sms_g, cudaDevAttrMultiProcessorCount, device));
        ctx->gram_grid = (int)std::min<long long>(ctx->n_items, sms_g);
    }

    unsigned int split_units = 0;
    {
        // the code sweep's order: patches by decreasing |Omega_i|, so that
        // the 32 patches of a warp have nearly equal counts (a warp's loops
        // run to its largest count); obs, nobs and pos are rewritten by slot
        std::vector<uint16_t> hn((size_t)N);
        std::vector<int> hp((size_t)g.Npad);
        CREATE_CUDA(cudaMemcpy(hn.data(), ctx->nobs, sizeof(uint16_t) * (size_t)N, cudaMemcpyDeviceToHost));
        sweep_order_host(hn.data(), N, g.Npad, hp.data());
        // work units (32 slots) whose largest count exceeds the light
        // kernel's capacity: a prefix, slots being in decreasing order
        split_units = 0;
        while ((long long)split_units < g.NW && (long long)split_units * 32 < N &&
               hn[(size_t)hp[(size_t)split_units * 32]] > kSplitObs)
            ++split_units;
        CREATE_CUDA(dalloc(&ctx->perm, (size_t)g.Npad));
        CREATE_CUDA(cudaMemcpy(ctx->perm, hp.data(), sizeof(int) * (size_t)g.Npad, cudaMemcpyHostToDevice));
        const size_t rows = (size_t)(ctx->maxobs > 0 ? ctx->maxobs : 1);
        uint16_t *obs_s = nullptr, *nobs_s = nullptr;
        int* pos_s = nullptr;
        cudaError_t e1 = dalloc(&obs_s, rows * N);
        if (e1 == cudaSuccess) e1 = dalloc(&nobs_s, (size_t)N);
        if (e1 == cudaSuccess) e1 = dalloc(&pos_s, rows * N);
        if (e1 == cudaSuccess)
            e1 = launch_sweep_order(g, ctx->maxobs, ctx->perm, ctx->obs, ctx->nobs, ctx->pos, obs_s, nobs_s, pos_s,
                                    st0);
        if (e1 == cudaSuccess) e1 = cudaDeviceSynchronize();
        if (e1 != cudaSuccess) {
            cudaFree(obs_s);
            cudaFree(nobs_s);
            cudaFree(pos_s);
            return bail(cuda_failure(nullptr, e1, "sweep order", __LINE__));
        }
        std::swap(ctx->obs, obs_s);
        std::swap(ctx->nobs, nobs_s);
        std::swap(ctx->pos, pos_s);
        cudaFree(obs_s);
        cudaFree(nobs_s);
        cudaFree(pos_s);
        ctx->launches += 1;
    }

    CREATE_CUDA(dalloc(&ctx->x, (size_t)nframe));
    CREATE_CUDA(dalloc(&ctx->out, (size_t)nframe));
    CREATE_CUDA(dalloc(&ctx->mean_acc, (size_t)nframe));
    CREATE_CUDA(cudaMemset(ctx->mean_acc, 0, sizeof(double) * (size_t)nframe));
    CREATE_CUDA(dalloc(&ctx->D, (size_t)g.K * P));
    CREATE_CUDA(dalloc(&ctx->W, (size_t)g.KB * kAtomBlock * g.Npad));
    CREATE_CUDA(dalloc(&ctx->Zb, (size_t)g.K * g.NW));
    CREATE_CUDA(dalloc(&ctx->Y, (size_t)P * N));
    if (recon_tc_available(ctx->g)) CREATE_CUDA(dalloc(&ctx->Dc, recon_tc_operand_floats(ctx->g)));
    CREATE_CUDA(dalloc(&ctx->pi, (size_t)g.K));
    CREATE_CUDA(dalloc(&ctx->lpi, (size_t)g.K));
    CREATE_CUDA(dalloc(&ctx->m, (size_t)g.K + 1));   // [K] counts, then the draw kernel's arrival counter
    CREATE_CUDA(cudaMemset(ctx->m, 0, sizeof(int) * ((size_t)g.K + 1)));
    CREATE_CUDA(dalloc(&ctx->part_s2, (size_t)2 * g.NW));   // per 16- or 32-patch work unit
    int sms = 0;
    CREATE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    {
        size_t n = (size_t)(2 * (size_t)g.NW > (size_t)P ? 2 * (size_t)g.NW : (size_t)P);
        if (n < (size_t)sms) n = (size_t)sms;
        CREATE_CUDA(dalloc(&ctx->part_r2, n));
    }
    CREATE_CUDA(dalloc(&ctx->chunk_counter, 1));
    CREATE_CUDA(dalloc(&ctx->ge_part, (size_t)kInitGammaEpsScratch));
    CREATE_CUDA(dalloc(&ctx->sc, 1));
    {
        const bool stream = (p.flags & SENSAI_FLAG_STREAM_DICTIONARY) != 0;
        const int slice = ((p.flags >> 8) & 0xff) * kAtomBlock;
        if (!plan_sweep(g, ctx->maxobs, device, stream, slice, &ctx->sweep_plan)) {
            fail(SENSAI_EINVAL, "no launch configuration for the code sweep (K=%d, P=%d, max observed %d, slice %d)",
                 g.K, g.P, ctx->maxobs, slice);
            return bail(SENSAI_EINVAL);
        }
        if (ctx->sweep_plan.slice_atoms > 0) CREATE_CUDA(dalloc(&ctx->Dsl, (size_t)slice_capacity_floats(g)));
        SweepPlan& sp = ctx->sweep_plan;
        if (sp.slice_atoms == 0 && sp.lanes == 1 && ctx->maxobs > kSplitObs && split_units > 0 &&
            (long long)split_units < g.NW && !stream) {
            sp.split_units = split_units;
            sp.split_grid = std::min(sp.grid, (int)((split_units + 7) / 8));
            sp.light_grid = sweep_grid_size(g, kSplitObs, device);
            if (sp.light_grid > 0) {
                CREATE_CUDA(cudaStreamCreateWithFlags(&sp.side, cudaStreamNonBlocking));
                CREATE_CUDA(cudaEventCreateWithFlags(&sp.fork, cudaEventDisableTiming));
                CREATE_CUDA(cudaEventCreateWithFlags(&sp.join, cudaEventDisableTiming));
                CREATE_CUDA(dalloc(&sp.counter2, 1));
            } else {
                sp.split_units = 0;
            }
        }
    }
    if (reset_state(ctx, st0) != SENSAI_OK) return bail(SENSAI_ECUDA);
    CREATE_CUDA(cudaDeviceSynchronize());
#undef CREATE_CUDA
    *out = ctx;
    return SENSAI_OK;
}

void sensai_destroy(sensai_ctx* ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->serve) serve_destroy(ctx->serve);
    cudaDeviceSynchronize();
    clear_timers(ctx);
    if (ctx->trace) fclose(ctx->trace);
    free_all(ctx);
    delete ctx;
}

sensai_status sensai_set_frame(sensai_ctx* ctx, const float* frame, void* stream)
{
    sensai_status st = enter(ctx);
    if (st != SENSAI_OK) return st;
    if (!frame) return fail(SENSAI_EINVAL, "null frame");
    ctx->last_stream = (cudaStream_t)stream;
    return copy_frame(ctx, frame, (cudaStream_t)stream);
}

sensai_status sensai_reset(sensai_ctx* ctx, void* stream)
{
    sensai_status st = enter(ctx);
    if (st != SENSAI_OK) return st;
    ctx->last_stream = (cudaStream_t)stream;
    return reset_state(ctx, (cudaStream_t)stream);
}

sensai_status sensai_sweep_codes(sensai_ctx* ctx, void* stream)
{
    sensai_status st = enter(ctx);
    if (st != SENSAI_OK) return st;
    ctx->last_stream = (cudaStream_t)stream;
    return run_sweep(ctx, (cudaStream_t)stream);
}

sensai_status sensai_draw_dictionary(sensai_ctx* ctx, void* stream)
{
    sensai_status st = enter(ctx);
    if (st != SENSAI_OK) return st;
    ctx->last_stream = (cudaStream_t)stream;
    return run_dictionary(ctx, (cudaStream_t)stream);
}

sensai_status sensai_draw_hyper(sensai_ctx* ctx, void* stream)
{
    sensai_status st = enter(ctx);
    if (st != SENSAI_OK) return st;
    ctx->last_stream = (cudaStream_t)stream;
    return run_hyper(ctx, (cudaStream_t)stream);
}

sensai_status sensai_learn(sensai_ctx* ctx, const float* frame, int32_t iters, void* stream)
{
    sensai_status st = enter(ctx);
    if (st != SENSAI_OK) return st;
    if (iters < 0) return fail(SENSAI_EINVAL, "iters must be >= 0");
    const cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    if (frame) {
        st = copy_frame(ctx, frame, s);
        if (st != SENSAI_OK) return st;
    }
    if (!ctx->frame_set) return fail(SENSAI_ESTATE, "no frame: pass one or call sensai_set_frame");
    for (int it = 0; it < iters; ++it) {
        if ((st = run_sweep(ctx, s)) != SENSAI_OK) return st;
        if ((st = run_dictionary(ctx, s)) != SENSAI_OK) return st;
        if ((st = run_hyper(ctx, s)) != SENSAI_OK) return st;
        ctx->t += 1;
        if ((st = trace_iteration(ctx, s, "learn")) != SENSAI_OK) return st;
    }
    return SENSAI_OK;
}

sensai_status sensai_inpaint(sensai_ctx* ctx, const float* frame, int32_t sweeps, float* out, void* stream)
{
    sensai_status st = enter(ctx);
    if (st != SENSAI_OK) return st;
    if (!frame) return fail(SENSAI_EINVAL, "null frame");
    if (sweeps < 0) return fail(SENSAI_EINVAL, "sweeps must be >= 0");
    const cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    if ((st = copy_frame(ctx, frame, s)) != SENSAI_OK) return st;
    if ((st = clear_codes(ctx, s)) != SENSAI_OK) return st;
    for (int it = 0; it < sweeps; ++it) {
        if ((st = run_sweep(ctx, s)) != SENSAI_OK) return st;
        if ((st = run_hyper(ctx, s)) != SENSAI_OK) return st;
        ctx->t += 1;
        if ((st = trace_iteration(ctx, s, "inpaint")) != SENSAI_OK) return st;
    }
    if (!out) return SENSAI_OK;
    const bool dev = is_device_pointer(out);
    float* dst = dev ? out : ctx->out;
    {
        PhaseTimer timer(ctx, kPhaseRecon, s);
        SENSAI_CUDA(ctx, launch_reconstruct(ctx->g, ctx->D, ctx->Dc, ctx->W, ctx->Y, dst, &ctx->sc->status, s));
        timer.stop();
        ctx->launches += reconstruct_launches(ctx->g);
    }
    if (!dev) return write_out(ctx, ctx->out, out, sizeof(float) * (size_t)ctx->g.nframe, s);
    return SENSAI_OK;
}

sensai_status sensai_reconstruct(sensai_ctx* ctx, float* out, void* stream)
{
    sensai_status st = enter(ctx);
    if (st != SENSAI_OK) return st;
    if (!out) return fail(SENSAI_EINVAL, "null output");
    const cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    const bool dev = is_device_pointer(out);
    float* dst = dev ? out : ctx->out;
    {
        PhaseTimer timer(ctx, kPhaseRecon, s);
        SENSAI_CUDA(ctx, launch_reconstruct(ctx->g, ctx->D, ctx->Dc, ctx->W, ctx->Y, dst, &ctx->sc->status, s));
        timer.stop();
        ctx->launches += reconstruct_launches(ctx->g);
    }
    if (!dev) return write_out(ctx, ctx->out, out, sizeof(float) * (size_t)ctx->g.nframe, s);
    return SENSAI_OK;
}

sensai_status sensai_mean_reset(sensai_ctx* ctx, void* stream)
{
    sensai_status st = enter(ctx);
    if (st != SENSAI_OK) return st;
    const cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    SENSAI_CUDA(ctx, cudaMemsetAsync(ctx->mean_acc, 0, sizeof(double) * (size_t)ctx->g.nframe, s));
    ctx->mean_count = 0;
    return SENSAI_OK;
}

sensai_status sensai_mean_add(sensai_ctx* ctx, void* stream)
{
    sensai_status st = enter(ctx);
    if (st != SENSAI_OK) return st;
    const cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    {
        PhaseTimer timer(ctx, kPhaseRecon, s);
        SENSAI_CUDA(ctx, launch_reconstruct(ctx->g, ctx->D, ctx->Dc, ctx->W, ctx->Y, ctx->out, &ctx->sc->status, s));
        SENSAI_CUDA(ctx, launch_mean_accumulate(ctx->g.nframe, ctx->out, ctx->mean_acc, s));
        timer.stop();
        ctx->launches += reconstruct_launches(ctx->g) + 1;
    }
    ctx->mean_count += 1;
    return SENSAI_OK;
}

sensai_status sensai_mean_read(sensai_ctx* ctx, float* out, void* stream)
{
    sensai_status st = enter(ctx);
    if (st != SENSAI_OK) return st;
    if (!out) return fail(SENSAI_EINVAL, "null output");
    if (ctx->mean_count < 1) return fail(SENSAI_ESTATE, "no reconstruction added since the last sensai_mean_reset");
    const cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    const bool dev = is_device_pointer(out);
    float* dst = dev ? out : ctx->out;
    SENSAI_CUDA(ctx, launch_mean_finish(ctx->g.nframe, ctx->mean_acc, ctx->mean_count, dst, s));
    ctx->launches += 1;
    if (!dev) return write_out(ctx, ctx->out, out, sizeof(float) * (size_t)ctx->g.nframe, s);
    return SENSAI_OK;
}

sensai_status sensai_overlap_counts(sensai_ctx* ctx, int32_t* out, void* stream)
{
    sensai_status st = enter(ctx);
    if (st != SENSAI_OK) return st;
    if (!out) return fail(SENSAI_EINVAL, "null output");
    const cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    const bool dev = is_device_pointer(out);
    int* dst = dev ? out : (int*)ctx->out;
    SENSAI_CUDA(ctx, launch_overlap_counts(ctx->g, dst, s));
    ctx->launches += 1;
    if (!dev) return write_out(ctx, ctx->out, out, sizeof(int) * (size_t)ctx->g.nframe, s);
    return SENSAI_OK;
}

sensai_status sensai_get_dictionary(sensai_ctx* ctx, float* D)
{
    sensai_status st = enter(ctx);
    if (st != SENSAI_OK) return st;
    if (!D) return fail(SENSAI_EINVAL, "null dictionary");
    SENSAI_CUDA(ctx, cudaDeviceSynchronize());
    SENSAI_CUDA(ctx, cudaMemcpy(D, ctx->D, sizeof(float) * (size_t)ctx->g.K * ctx->g.P, cudaMemcpyDefault));
    return SENSAI_OK;
}

sensai_status sensai_set_dictionary(sensai_ctx* ctx, const float* D)
{
    sensai_status st = enter(ctx);
    if (st != SENSAI_OK) return st;
    if (!D) return fail(SENSAI_EINVAL, "null dictionary");
    SENSAI_CUDA(ctx, cudaDeviceSynchronize());
    SENSAI_CUDA(ctx, cudaMemcpy(ctx->D, D, sizeof(float) * (size_t)ctx->g.K * ctx->g.P, cudaMemcpyDefault));
    ctx->resid_valid = false;
    ctx->resid_fresh = false;
    ctx->r2_valid = false;
    return SENSAI_OK;
}

sensai_status sensai_get_state(sensai_ctx* ctx, sensai_state* state)
{
    sensai_status st = enter(ctx);
    if (st != SENSAI_OK) return st;
    if (!state) return fail(SENSAI_EINVAL, "null state");
    const Geom& g = ctx->g;
    SENSAI_CUDA(ctx, cudaDeviceSynchronize());
    if (state->D) SENSAI_CUDA(ctx, cudaMemcpy(state->D, ctx->D, sizeof(float) * (size_t)g.K * g.P, cudaMemcpyDefault));
    if (state->pi) SENSAI_CUDA(ctx, cudaMemcpy(state->pi, ctx->pi, sizeof(double) * g.K, cudaMemcpyDefault));
    if (state->Z || state->S) {
        uint8_t* z = nullptr;
        float* sv = nullptr;
        const size_t n = (size_t)g.N * g.K;
        SENSAI_CUDA(ctx, dalloc(&z, n));
        cudaError_t e = dalloc(&sv, n);
        if (e != cudaSuccess) {
            cudaFree(z);
            return cuda_failure(ctx, e, "dalloc", __LINE__);
        }
        e = launch_export_codes(g, ctx->W, ctx->Zb, ctx->perm, z, sv, nullptr);
        if (e == cudaSuccess && state->Z) e = cudaMemcpy(state->Z, z, n, cudaMemcpyDefault);
        if (e == cudaSuccess && state->S) e = cudaMemcpy(state->S, sv, n * sizeof(float), cudaMemcpyDefault);
        cudaFree(z);
        cudaFree(sv);
        if (e != cudaSuccess) return cuda_failure(ctx, e, "export codes", __LINE__);
    }
    DevScalars sc;
    SENSAI_CUDA(ctx, cudaMemcpy(&sc, ctx->sc, sizeof(sc), cudaMemcpyDeviceToHost));
    state->gamma_s = sc.gamma_s;
    state->gamma_eps = ctx->ge_set ? sc.gamma_eps : 0.0;
    state->iter = ctx->t;
    return SENSAI_OK;
}

sensai_status sensai_set_state(sensai_ctx* ctx, const sensai_state* state)
{
    sensai_status st = enter(ctx);
    if (st != SENSAI_OK) return st;
    if (!state) return fail(SENSAI_EINVAL, "null state");
    if ((state->Z == nullptr) != (state->S == nullptr)) return fail(SENSAI_EINVAL, "Z and S must be set together");
    if (!(state->gamma_s > 0)) return fail(SENSAI_EINVAL, "gamma_s must be > 0");
    if (state->iter < 0) return fail(SENSAI_EINVAL, "iter must be >= 0");
    if (state->pi)
        for (int k = 0; k < ctx->g.K; ++k)
            if (!(state->pi[k] > 0.0 && state->pi[k] < 1.0)) return fail(SENSAI_EINVAL, "pi[%d] must be in (0, 1)", k);
    const Geom& g = ctx->g;
    SENSAI_CUDA(ctx, cudaDeviceSynchronize());
    if (state->D) SENSAI_CUDA(ctx, cudaMemcpy(ctx->D, state->D, sizeof(float) * (size_t)g.K * g.P, cudaMemcpyDefault));
    if (state->pi) {
        SENSAI_CUDA(ctx, cudaMemcpy(ctx->pi, state->pi, sizeof(double) * g.K, cudaMemcpyDefault));
        SENSAI_CUDA(ctx, launch_logit(g.K, ctx->pi, ctx->lpi, nullptr));
    }
    if (state->Z) {
        uint8_t* z = nullptr;
        float* sv = nullptr;
        const size_t n = (size_t)g.N * g.K;
        SENSAI_CUDA(ctx, dalloc(&z, n));
        cudaError_t e = dalloc(&sv, n);
        if (e == cudaSuccess) e = cudaMemcpy(z, state->Z, n, cudaMemcpyDefault);
        if (e == cudaSuccess) e = cudaMemcpy(sv, state->S, n * sizeof(float), cudaMemcpyDefault);
        if (e == cudaSuccess) e = launch_import_codes(g, z, sv, ctx->perm, ctx->W, ctx->Zb, nullptr);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        cudaFree(z);
        if (sv) cudaFree(sv);
        if (e != cudaSuccess) return cuda_failure(ctx, e, "import codes", __LINE__);
    }
    DevScalars sc;
    SENSAI_CUDA(ctx, cudaMemcpy(&sc, ctx->sc, sizeof(sc), cudaMemcpyDeviceToHost));
    sc.gamma_s = state->gamma_s;
    if (state->gamma_eps > 0) {
        sc.gamma_eps = state->gamma_eps;
        sc.ge_set = 1;
        ctx->ge_set = true;
    }
    SENSAI_CUDA(ctx, cudaMemcpy(ctx->sc, &sc, sizeof(sc), cudaMemcpyHostToDevice));
    ctx->t = state->iter;
    ctx->codes_valid = false;
    ctx->resid_valid = false;
    ctx->resid_fresh = false;
    ctx->r2_valid = false;
    return SENSAI_OK;
}

sensai_status sensai_get_stats(sensai_ctx* ctx, sensai_stats* stats)
{
    sensai_status st = enter(ctx);
    if (st != SENSAI_OK) return st;
    if (!stats) return fail(SENSAI_EINVAL, "null stats");
    SENSAI_CUDA(ctx, cudaStreamSynchronize(ctx->last_stream));
    DevScalars sc;
    SENSAI_CUDA(ctx, cudaMemcpy(&sc, ctx->sc, sizeof(sc), cudaMemcpyDeviceToHost));
    stats->iter = ctx->t;
    stats->n_patches = ctx->g.N;
    stats->patch_size = ctx->g.P;
    stats->n_observed = ctx->n_observed;
    stats->n_active = sc.n_active;
    stats->max_observed = ctx->maxobs;
    stats->K = ctx->g.K;
    stats->sum_s2 = sc.sum_s2;
    stats->sum_r2 = sc.sum_r2;
    stats->gamma_s = sc.gamma_s;
    stats->gamma_eps = ctx->ge_set ? sc.gamma_eps : 0.0;
    stats->kernel_launches = ctx->launches;
    if (sc.status != 0) return fail(SENSAI_ETIMEOUT, "a device-side wait timed out (status %d)", sc.status);
    stats->changed_updates = (int64_t)sc.chg_n;
    stats->changed_observed = (int64_t)sc.chg_obs;
    stats->active_draws = (int64_t)sc.act_n;
    stats->rebuild_observed = (int64_t)sc.rb_obs;
    stats->slice_atoms = ctx->sweep_plan.slice_atoms;
    stats->slices = ctx->sweep_plan.slices;
    stats->dictionary_form = ctx->gram ? 3 : ctx->ds.grid > 0 ? (ctx->ds.staged ? 2 : 1) : 0;
    stats->dictionary_smem_kb = ctx->gram || ctx->ds.grid == 0 ? 0 : (int32_t)((ctx->ds.smem + 1023) / 1024);
    return SENSAI_OK;
}

sensai_status sensai_serve_start(sensai_ctx* ctx, const sensai_serve_params* sp)
{
    sensai_status st = enter(ctx);
    if (st != SENSAI_OK) return st;
    if (!sp) return fail(SENSAI_EINVAL, "null serve parameters");
    if (ctx->serve) return fail(SENSAI_EBUSY, "already serving");
    if (sp->slots < 1 || sp->slots > 64) return fail(SENSAI_EINVAL, "slots must be 1..64");
    if (sp->max_pixels < 1 || sp->max_pixels >= (1LL << 31)) return fail(SENSAI_EINVAL, "bad max_pixels");
    if (sp->max_observed < 1 || sp->max_observed > 256) return fail(SENSAI_EINVAL, "max_observed must be 1..256");
    if (!ctx->ge_set) return fail(SENSAI_ESTATE, "serving needs a learnt or set state (gamma_eps unset)");
    SENSAI_CUDA(ctx, cudaDeviceSynchronize());
    DevScalars sc;
    SENSAI_CUDA(ctx, cudaMemcpy(&sc, ctx->sc, sizeof(sc), cudaMemcpyDeviceToHost));
    ServeInit in{};
    in.device = ctx->device;
    in.base = ctx->g;
    in.D = ctx->D;
    in.pi = ctx->pi;
    in.gamma_s = sc.gamma_s;
    in.gamma_eps = sc.gamma_eps;
    in.a_over_K = ctx->a_over_K;
    in.b_param = ctx->prm.b;
    in.c = ctx->prm.c;
    in.d = ctx->prm.d;
    in.e = ctx->prm.e;
    in.f = ctx->prm.f;
    in.seed = ctx->prm.seed;
    in.t0 = (uint32_t)ctx->t;
    in.slots = sp->slots;
    in.max_pixels = sp->max_pixels;
    in.memory_budget = sp->memory_budget;
    in.max_observed = sp->max_observed;
    in.stream_dictionary = (ctx->prm.flags & SENSAI_FLAG_STREAM_DICTIONARY) != 0;
    in.slice_atoms = ((ctx->prm.flags >> 8) & 0xff) * kAtomBlock;
    in.full_s = (ctx->prm.flags & SENSAI_FLAG_GAMMA_S_FULL) != 0;
    ctx->serve = serve_create(in, &st);
    if (!ctx->serve) return fail(st, "could not allocate the serving slots");
    return SENSAI_OK;
}

sensai_status sensai_submit_frame(sensai_ctx* ctx, int32_t stream_id, uint64_t frame_id, const float* frame,
                                  const uint8_t* mask, const int64_t* M, int32_t sweeps, float* out,
                                  sensai_done_fn done, void* user)
{
    if (!ctx) return fail(SENSAI_EINVAL, "null context");
    if (!ctx->serve) return fail(SENSAI_ESTATE, "serving engine not started");
    const sensai_status st = serve_submit(ctx->serve, stream_id, frame_id, frame, mask, M, sweeps, out, done, user);
    if (st == SENSAI_EINVAL) return fail(st, "bad frame: shape, size above max_pixels or above the memory budget");
    if (st != SENSAI_OK) return fail(st, "serving engine stopped");
    return SENSAI_OK;
}

sensai_status sensai_serve_drain(sensai_ctx* ctx)
{
    if (!ctx) return fail(SENSAI_EINVAL, "null context");
    if (!ctx->serve) return fail(SENSAI_ESTATE, "serving engine not started");
    std::string msg;
    const sensai_status st = serve_drain(ctx->serve, &msg);
    if (st != SENSAI_OK) return fail(st, "%s", msg.c_str());
    return SENSAI_OK;
}

sensai_status sensai_serve_stop(sensai_ctx* ctx)
{
    if (!ctx) return fail(SENSAI_EINVAL, "null context");
    if (!ctx->serve) return fail(SENSAI_ESTATE, "serving engine not started");
    serve_destroy(ctx->serve);
    ctx->serve = nullptr;
    return SENSAI_OK;
}

sensai_status sensai_trace(sensai_ctx* ctx, const char* path, const float* clean)
{
    sensai_status st = enter(ctx);
    if (st != SENSAI_OK) return st;
    if (ctx->trace) fclose(ctx->trace);
    ctx->trace = nullptr;
    ctx->trace_clean.clear();
    ctx->trace_rec.clear();
    if (!path) return SENSAI_OK;
    const size_t n = (size_t)ctx->g.nframe;
    if (clean) {
        ctx->trace_clean.resize(n);
        ctx->trace_rec.resize(n);
        SENSAI_CUDA(ctx, cudaMemcpy(ctx->trace_clean.data(), clean, sizeof(float) * n, cudaMemcpyDefault));
    }
    FILE* f = fopen(path, "a");
    if (!f) {
        ctx->trace_clean.clear();
        ctx->trace_rec.clear();
        return fail(SENSAI_EINVAL, "cannot open the trace file %s", path);
    }
    ctx->trace = f;
    ctx->trace_last = std::chrono::steady_clock::now();
    return SENSAI_OK;
}

sensai_status sensai_profile(sensai_ctx* ctx, int32_t enable)
{
    sensai_status st = enter(ctx);
    if (st != SENSAI_OK) return st;
    if (enable) {
        SENSAI_CUDA(ctx, cudaDeviceSynchronize());
        clear_timers(ctx);
        const unsigned long long zero[4] = {0, 0, 0, 0};   // chg_n, chg_obs, act_n, rb_obs
        SENSAI_CUDA(ctx, cudaMemcpy(&ctx->sc->chg_n, zero, sizeof(zero), cudaMemcpyHostToDevice));
    }
    ctx->profiling = enable != 0;
    return SENSAI_OK;
}

sensai_status sensai_profile_read(sensai_ctx* ctx, double* ms, int64_t* counts)
{
    sensai_status st = enter(ctx);
    if (st != SENSAI_OK) return st;
    if (!ms || !counts) return fail(SENSAI_EINVAL, "null output");
    SENSAI_CUDA(ctx, cudaDeviceSynchronize());
    for (int ph = 0; ph < 4; ++ph) {
        double total = 0.0;
        for (auto& pr : ctx->timed[ph]) {
            float t = 0.0f;
            SENSAI_CUDA(ctx, cudaEventElapsedTime(&t, pr.first, pr.second));
            total += t;
        }
        ms[ph] = total;
        counts[ph] = (int64_t)ctx->timed[ph].size();
    }
    return SENSAI_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ batches --
//
// A batch learns n independent contexts together.  One Gibbs iteration of all
// instances is a handful of launches, each covering every instance:
//  * the code sweeps: one launch per kernel variant, CTAs divided among the
//    instances in proportion to their work, each instance's CTAs sharing its
//    patches through the instance's own chunk counter;
//  * the per-chain dictionary draws: one CTA per (instance, chain), one
//    launch per storage mode;
//  * the pi draws (one CTA per (instance, atom)) and the gamma draws (one CTA
//    per instance).
// The iteration is captured once into a CUDA graph and replayed per
// iteration.  The kernels read the iteration index from each context's device
// scalars and the gamma draws advance it, so every replay draws with fresh
// counters, and every context ends exactly where sensai_learn on it alone
// would.

namespace {

struct BatchClass {
    int key = 0;                 // sweep: template capacity; dictionary: storage mode
    bool streamed = false;       // sweep: dictionary streamed in slices
    std::vector<int> members;    // instance indices, in argument-array order
    size_t smem = 0;
    int grid = 0;
    int args_off = 0;            // first member in the class's argument array
    int table_off = 0;           // its CTA prefix table in the batch's table array
};

}  // namespace

constexpr int kBatchLanes = 8;   // side streams: launches of different classes overlap

struct sensai_batch {
    std::vector<sensai_ctx*> ctx;
    cudaStream_t origin = nullptr;       // the stream graphs are captured on and replayed from
    cudaStream_t side[kBatchLanes] = {};
    cudaEvent_t fork = nullptr, joins[kBatchLanes] = {};
    cudaEvent_t in = nullptr, out = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int divisor = 1;                     // code-sweep grid: 4 waves / divisor
    // device tables of the current graph
    SweepArgs* d_sweep = nullptr;
    DictArgs* d_dict = nullptr;
    HyperArgs* d_hyper = nullptr;
    unsigned int* d_counters = nullptr;  // per-instance chunk counters of the batched sweeps
    int* d_tables = nullptr;             // CTA prefix tables
    std::vector<BatchClass> sweeps, dicts;
    int pi_table = 0, gamma_table = 0, pi_grid = 0;
    long long launches_per_iter = 0;
};

namespace {

void batch_free_tables(sensai_batch* b)
{
    void* ptrs[] = {b->d_sweep, b->d_dict, b->d_hyper, b->d_counters, b->d_tables};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    b->d_sweep = nullptr;
    b->d_dict = nullptr;
    b->d_hyper = nullptr;
    b->d_counters = nullptr;
    b->d_tables = nullptr;
}

void batch_drop_graph(sensai_batch* b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    batch_free_tables(b);
}

// Per-instance arguments of the batched kernels, their classes and CTA
// partitions, uploaded to device tables.
sensai_status batch_build(sensai_batch* b)
{
    const int n = (int)b->ctx.size();
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->ctx[0]->device);
    if (e != cudaSuccess) return cuda_failure(nullptr, e, "cudaDeviceGetAttribute", __LINE__);
    if ((e = cudaMalloc((void**)&b->d_counters, sizeof(unsigned int) * n)) != cudaSuccess)
        return cuda_failure(nullptr, e, "batch counters", __LINE__);
    std::vector<SweepArgs> sa(n);
    std::vector<DictArgs> da(n);
    std::vector<HyperArgs> ha(n);
    for (int i = 0; i < n; ++i) {
        sensai_ctx* c = b->ctx[i];
        c->t_on_device = true;
        sa[i] = sweep_args(c);   // batched sweeps rebuild their residual themselves (same bits)
        da[i] = dict_args(c);
        ha[i] = hyper_args(c);
        c->t_on_device = false;
        sa[i].chunk_counter = b->d_counters + i;
        if (c->sweep_plan.slice_atoms > 0) {
            sa[i].Dsl = c->Dsl;
            sa[i].slice_atoms = c->sweep_plan.slice_atoms;
            sa[i].slices = c->sweep_plan.slices;
            sa[i].slice_stride = c->sweep_plan.slice_stride;
        }
        ha[i].n_s2 = c->g.NW * c->sweep_plan.lanes;   // the sweep's partials
        ha[i].n_r2 = c->g.P;                          // the per-chain dictionary draws' partials
    }
    // classes
    b->sweeps.clear();
    b->dicts.clear();
    for (int i = 0; i < n; ++i) {
        sensai_ctx* c = b->ctx[i];
        const bool streamed = c->sweep_plan.slice_atoms > 0;
        const int key = sweep_variant(c->maxobs > 0 ? c->maxobs : 1);
        BatchClass* cl = nullptr;
        for (BatchClass& x : b->sweeps)
            if (x.key == key && x.streamed == streamed) cl = &x;
        if (!cl) {
            b->sweeps.push_back(BatchClass{});
            cl = &b->sweeps.back();
            cl->key = key;
            cl->streamed = streamed;
        }
        cl->members.push_back(i);
        const size_t sm = streamed ? tiled_smem_bytes(c->g, c->sweep_plan.slice_atoms) : (size_t)sweep_smem_bytes(c->g);
        cl->smem = std::max(cl->smem, sm);
        size_t dsm = 0;
        const int mode = dict_mode(c->max_slots, &dsm);
        if (mode < 0) return fail(SENSAI_ECUDA, "no dictionary launch mode for instance %d", i);
        BatchClass* dl = nullptr;
        for (BatchClass& x : b->dicts)
            if (x.key == mode) dl = &x;
        if (!dl) {
            b->dicts.push_back(BatchClass{});
            dl = &b->dicts.back();
            dl->key = mode;
        }
        dl->members.push_back(i);
        dl->smem = std::max(dl->smem, dsm);
    }
    // CTA partitions and argument order
    std::vector<int> tables;
    std::vector<SweepArgs> sa_ord;
    std::vector<DictArgs> da_ord;
    for (BatchClass& cl : b->sweeps) {
        const int per_sm = cl.streamed ? sweep_tiled_multi_ctas_per_sm(cl.key, cl.smem)
                                       : sweep_multi_ctas_per_sm(cl.key, cl.smem);
        if (per_sm < 1) return fail(SENSAI_ECUDA, "no batched code-sweep configuration (capacity %d)", cl.key);
        const long long total = std::max<long long>((long long)cl.members.size(),
                                                    4LL * per_sm * sms / std::max(1, b->divisor));
        double work_sum = 0.0;
        std::vector<double> work;
        for (int i : cl.members) {
            const sensai_ctx* c = b->ctx[i];
            const double obs = (double)c->n_observed / std::max<long long>(1, c->g.N);
            work.push_back((double)c->g.N * c->g.K * (75.0 + 3.0 * obs));
            work_sum += work.back();
        }
        cl.args_off = (int)sa_ord.size();
        cl.table_off = (int)tables.size();
        int acc = 0;
        for (size_t m = 0; m < cl.members.size(); ++m) {
            const sensai_ctx* c = b->ctx[cl.members[m]];
            const long long units = (long long)c->g.NW * c->sweep_plan.lanes;
            const long long cap = (units + 7) / 8;     // 8 warps per CTA
            long long ctas = (long long)std::floor((double)total * work[m] / work_sum);
            ctas = std::max<long long>(1, std::min(ctas, cap));
            tables.push_back(acc);
            acc += (int)ctas;
            sa_ord.push_back(sa[cl.members[m]]);
        }
        tables.push_back(acc);
        cl.grid = acc;
    }
    for (BatchClass& cl : b->dicts) {
        cl.args_off = (int)da_ord.size();
        cl.table_off = (int)tables.size();
        int acc = 0;
        for (int i : cl.members) {
            tables.push_back(acc);
            acc += b->ctx[i]->g.P;
            da_ord.push_back(da[i]);
        }
        tables.push_back(acc);
        cl.grid = acc;
    }
    b->pi_table = (int)tables.size();
    int acc = 0;
    for (int i = 0; i < n; ++i) {
        tables.push_back(acc);
        acc += b->ctx[i]->g.K;
    }
    tables.push_back(acc);
    b->pi_grid = acc;
    b->gamma_table = (int)tables.size();
    for (int i = 0; i <= n; ++i) tables.push_back(i);
    // upload
    e = cudaMalloc((void**)&b->d_sweep, sizeof(SweepArgs) * n);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_dict, sizeof(DictArgs) * n);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_hyper, sizeof(HyperArgs) * n);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_tables, sizeof(int) * tables.size());
    if (e == cudaSuccess) e = cudaMemcpy(b->d_sweep, sa_ord.data(), sizeof(SweepArgs) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_dict, da_ord.data(), sizeof(DictArgs) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_hyper, ha.data(), sizeof(HyperArgs) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_tables, tables.data(), sizeof(int) * tables.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_failure(nullptr, e, "batch tables", __LINE__);
    return SENSAI_OK;
}

// Captures one iteration of every instance (the caller has run the eager
// setup: frame, gamma_eps, residual, iteration indices).
sensai_status batch_capture(sensai_batch* b)
{
    batch_drop_graph(b);
    sensai_status st = batch_build(b);
    if (st != SENSAI_OK) {
        batch_free_tables(b);
        return st;
    }
    const int n = (int)b->ctx.size();
    const cudaStream_t s = b->origin;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return cuda_failure(nullptr, e, "cudaStreamBeginCapture", __LINE__);
    long long launches = 0;
    e = cudaMemsetAsync(b->d_counters, 0, sizeof(unsigned int) * n, s);
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        const sensai_ctx* c = b->ctx[i];
        if (c->sweep_plan.slice_atoms > 0) {
            e = launch_slice_dictionary(c->g, c->D, c->Dsl, c->sweep_plan.slice_atoms, s);
            ++launches;
        }
    }
    // the classes of one phase run side by side (fork / join), phases in order
    auto fork = [&](size_t nclass) {
        if (e == cudaSuccess) e = cudaEventRecord(b->fork, s);
        for (size_t j = 0; j < std::min<size_t>(nclass, kBatchLanes) && e == cudaSuccess; ++j)
            e = cudaStreamWaitEvent(b->side[j], b->fork, 0);
    };
    auto join = [&](size_t nclass) {
        for (size_t j = 0; j < std::min<size_t>(nclass, kBatchLanes) && e == cudaSuccess; ++j) {
            e = cudaEventRecord(b->joins[j], b->side[j]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->joins[j], 0);
        }
    };
    fork(b->sweeps.size());
    for (size_t j = 0; j < b->sweeps.size() && e == cudaSuccess; ++j) {
        const BatchClass& cl = b->sweeps[j];
        const SweepArgs* args = b->d_sweep + cl.args_off;
        const int* table = b->d_tables + cl.table_off;
        const int m = (int)cl.members.size();
        const cudaStream_t ss = b->side[j % kBatchLanes];
        e = cl.streamed ? launch_sweep_tiled_multi(args, table, m, cl.key, cl.grid, cl.smem, ss)
                        : launch_sweep_multi(args, table, m, cl.key, cl.grid, cl.smem, ss);
        ++launches;
    }
    join(b->sweeps.size());
    fork(b->dicts.size());
    for (size_t j = 0; j < b->dicts.size() && e == cudaSuccess; ++j) {
        const BatchClass& cl = b->dicts[j];
        e = launch_dict_multi(b->d_dict + cl.args_off, b->d_tables + cl.table_off, (int)cl.members.size(), cl.key,
                              cl.smem, cl.grid, b->side[j % kBatchLanes]);
        ++launches;
    }
    join(b->dicts.size());
    if (e == cudaSuccess) {
        e = launch_hyper_multi(b->d_hyper, b->d_tables + b->pi_table, b->d_tables + b->gamma_table, n, b->pi_grid, s);
        launches += 2;
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e_end = cudaStreamEndCapture(s, &g);
    if (e == cudaSuccess) e = e_end;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        b->exec = nullptr;
        batch_free_tables(b);
        return cuda_failure(nullptr, e, "batch graph capture", __LINE__);
    }
    b->graph = g;
    b->launches_per_iter = launches;
    return SENSAI_OK;
}

// Eager per-instance setup on the origin stream, then the iteration indices.
sensai_status batch_prepare(sensai_batch* b)
{
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        sensai_ctx* c = b->ctx[i];
        sensai_status st = enter(c);
        if (st != SENSAI_OK) return st;
        if (!c->frame_set) return fail(SENSAI_ESTATE, "batch instance %zu has no frame", i);
        if ((st = ensure_gamma_eps(c, b->origin)) != SENSAI_OK) return st;
        if ((st = ensure_residual(c, b->origin)) != SENSAI_OK) return st;
        SENSAI_CUDA(c, launch_set_iteration(c->sc, (uint32_t)c->t, b->origin));
        c->launches += 1;
    }
    return SENSAI_OK;
}

void batch_advance(sensai_batch* b, int iters)
{
    for (sensai_ctx* c : b->ctx) {
        c->t += iters;
        c->codes_valid = true;
        c->resid_valid = true;
        c->resid_fresh = false;
        c->r2_valid = true;
        c->n_s2 = c->g.NW * c->sweep_plan.lanes;
        c->n_r2 = c->g.P;
    }
}

// Replays the graph iters times on the origin stream, ordered after `user`
// and before whatever the caller enqueues on `user` next.
sensai_status batch_replay(sensai_batch* b, int iters, cudaStream_t user)
{
    cudaError_t e = cudaEventRecord(b->in, user);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->origin, b->in, 0);
    if (e != cudaSuccess) return cuda_failure(nullptr, e, "batch stream ordering", __LINE__);
    sensai_status st = batch_prepare(b);
    if (st != SENSAI_OK) return st;
    if (!b->exec && (st = batch_capture(b)) != SENSAI_OK) return st;
    for (int it = 0; it < iters && e == cudaSuccess; ++it) e = cudaGraphLaunch(b->exec, b->origin);
    if (e == cudaSuccess) e = cudaEventRecord(b->out, b->origin);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(user, b->out, 0);
    if (e != cudaSuccess) return cuda_failure(nullptr, e, "cudaGraphLaunch", __LINE__);
    batch_advance(b, iters);
    return SENSAI_OK;
}

}  // namespace

extern "C" {

void sensai_batch_destroy(sensai_batch* b)
{
    if (!b) return;
    if (b->origin) cudaStreamSynchronize(b->origin);
    batch_drop_graph(b);
    cudaEvent_t evs[] = {b->in, b->out, b->fork};
    for (cudaEvent_t ev : evs)
        if (ev) cudaEventDestroy(ev);
    for (int j = 0; j < kBatchLanes; ++j) {
        if (b->joins[j]) cudaEventDestroy(b->joins[j]);
        if (b->side[j]) cudaStreamDestroy(b->side[j]);
    }
    if (b->origin) cudaStreamDestroy(b->origin);
    delete b;
}

sensai_status sensai_batch_create(sensai_ctx* const* ctxs, int32_t n, sensai_batch** out)
{
    if (!ctxs || !out || n < 1) return fail(SENSAI_EINVAL, "need n >= 1 contexts and an output pointer");
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) return fail(SENSAI_EINVAL, "null context %d", i);
        if (!(ctxs[i]->prm.flags & SENSAI_FLAG_CHAIN_DICTIONARY))
            return fail(SENSAI_EINVAL, "context %d does not use the per-chain dictionary kernel; create it with "
                        "SENSAI_FLAG_CHAIN_DICTIONARY", i);
        if (ctxs[i]->device != ctxs[0]->device) return fail(SENSAI_EINVAL, "contexts on different devices");
        if (ctxs[i]->prm.flags & SENSAI_FLAG_GAMMA_S_FULL)
            return fail(SENSAI_EINVAL, "context %d uses SENSAI_FLAG_GAMMA_S_FULL, which batches do not support", i);
        if (ctxs[i]->serve) return fail(SENSAI_EBUSY, "context %d is serving", i);
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return fail(SENSAI_EINVAL, "context %d appears twice", i);
    }
    sensai_status st = enter(ctxs[0]);
    if (st != SENSAI_OK) return st;
    sensai_batch* b = new (std::nothrow) sensai_batch();
    if (!b) return fail(SENSAI_ENOMEM, "host allocation failed");
    b->ctx.assign(ctxs, ctxs + n);
    cudaError_t e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (int j = 0; j < kBatchLanes && e == cudaSuccess; ++j) {
        e = cudaStreamCreateWithFlags(&b->side[j], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->joins[j], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        sensai_batch_destroy(b);
        return cuda_failure(nullptr, e, "batch resources", __LINE__);
    }
    *out = b;
    return SENSAI_OK;
}

sensai_status sensai_batch_learn(sensai_batch* b, int32_t iters, void* stream)
{
    if (!b) return fail(SENSAI_EINVAL, "null batch");
    if (iters < 0) return fail(SENSAI_EINVAL, "iters must be >= 0");
    if (iters == 0) return SENSAI_OK;
    return batch_replay(b, iters, (cudaStream_t)stream);
}

sensai_status sensai_batch_tune(sensai_batch* b, int32_t iters_per_trial, void* stream, int32_t* divisor)
{
    if (!b) return fail(SENSAI_EINVAL, "null batch");
    if (iters_per_trial < 1) return fail(SENSAI_EINVAL, "iters_per_trial must be >= 1");
    const cudaStream_t user = (cudaStream_t)stream;
    const int candidates[] = {1, 2, 4, 8, 16};
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    cudaError_t e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    if (e != cudaSuccess) return cuda_failure(nullptr, e, "cudaEventCreate", __LINE__);
    float best_ms = 0.0f;
    int best = 1;
    sensai_status st = SENSAI_OK;
    for (int cand : candidates) {
        b->divisor = cand;
        batch_drop_graph(b);
        // one warm-up replay (captures the graph), then the timed replays
        if ((st = batch_replay(b, 1, user)) != SENSAI_OK) break;
        if ((e = cudaEventRecord(t0, b->origin)) != cudaSuccess) break;
        for (int it = 0; it < iters_per_trial && e == cudaSuccess; ++it) e = cudaGraphLaunch(b->exec, b->origin);
        if (e == cudaSuccess) e = cudaEventRecord(t1, b->origin);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        if (e != cudaSuccess) break;
        batch_advance(b, iters_per_trial);
        if (cand == candidates[0] || ms < best_ms) {
            best_ms = ms;
            best = cand;
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (e == cudaSuccess) e = cudaEventRecord(b->out, b->origin);   // the caller's stream follows the trials
    if (e == cudaSuccess) e = cudaStreamWaitEvent(user, b->out, 0);
    if (st != SENSAI_OK) return st;
    if (e != cudaSuccess) return cuda_failure(nullptr, e, "batch tuning", __LINE__);
    b->divisor = best;
    batch_drop_graph(b);
    if (divisor) *divisor = best;
    return SENSAI_OK;
}

}  // extern "C"

extern "C" sensai_status sensai_selftest_wait(int32_t which)
{
    if (which != 0 && which != 1) return fail(SENSAI_EINVAL, "which must be 0 (grid barrier) or 1 (mbarrier)");
    int* status = nullptr;
    unsigned int* count = nullptr;
    cudaError_t e = cudaMalloc((void**)&status, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void**)&count, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(status, 0, sizeof(int));
    if (e == cudaSuccess)
        e = which == 0 ? launch_barrier_timeout_selftest(count, status, nullptr) : launch_mbar_timeout_selftest(status, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int st = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&st, status, sizeof(int), cudaMemcpyDeviceToHost);
    if (status) cudaFree(status);
    if (count) cudaFree(count);
    if (e != cudaSuccess) return cuda_failure(nullptr, e, "wait self-test", __LINE__);
    if (st == SENSAI_ETIMEOUT) return fail(SENSAI_ETIMEOUT, "the bounded %s wait gave up as designed",
                                          which == 0 ? "grid-barrier" : "mbarrier");
    return SENSAI_OK;
}
