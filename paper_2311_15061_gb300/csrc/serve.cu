// serve.cu -- live serving engine: inpainting of a continuous feed of frames
// with a transferred (fixed) dictionary.
//
// The paper's library reconstructs a live feed frame by frame while the
// microscope scans (Sec. "Introduction", Sec. "Visitors Experience"), using a
// dictionary learnt elsewhere (dictionary transfer, Sec. "SenseAI: Feature
// Summary").  Each frame is the same computation as sensai_inpaint: codes
// cleared, `sweeps` iterations of code sweep + pi / gamma draws at iteration
// index t0 + s, then overlap-add.
//
// Runtime: a fixed set of slots, each with its own CUDA stream, device
// buffers sized for the largest accepted frame and a worker thread.  Frames
// wait in one FIFO queue; the head is admitted when a slot is free and the
// device bytes of the frames in flight plus its own fit the memory budget, so
// requests that arrive while others run start as soon as room frees up and
// their kernels overlap on the device.  A frame's random numbers are keyed by
// h(h(h(seed) ^ stream_id) ^ frame_id) with h the SplitMix64 finaliser, so its
// result is the same alone and in any mix.
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <string>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.cuh"

namespace sensai {

// SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014).
static uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t serve_frame_seed(uint64_t seed, int32_t stream_id, uint64_t frame_id)
{
    uint64_t h = splitmix64(seed);
    h = splitmix64(h ^ (uint64_t)(uint32_t)stream_id);
    return splitmix64(h ^ frame_id);
}

struct ServeRequest {
    int32_t stream_id;
    uint64_t frame_id;
    const float* frame;
    const uint8_t* mask;
    float* out;
    int32_t sweeps;
    sensai_done_fn done;
    void* user;
    Geom g;
    size_t bytes;
};

struct ServeSlot {
    cudaStream_t stream = nullptr;
    float* x = nullptr;
    uint8_t* mask_bytes = nullptr;
    uint32_t* mask_bits = nullptr;
    int* imgoff = nullptr;
    uint16_t* nobs = nullptr;
    uint16_t* obs = nullptr;
    int* misc = nullptr;                 // [0] max |Omega_i|
    unsigned long long* total = nullptr; // sum |Omega_i|
    float* W = nullptr;
    uint32_t* Zb = nullptr;
    int* m = nullptr;
    double* part_s2 = nullptr;
    double* part_r2 = nullptr;
    unsigned int* counter = nullptr;
    DevScalars* sc = nullptr;
    double* pi = nullptr;
    float* lpi = nullptr;
    float* Y = nullptr;
    float* Dc = nullptr;                 // dictionary operands of the tensor-core reconstruction
    float* out = nullptr;
    float* Dsl = nullptr;                // dictionary slices (streamed code sweep)
    int* h_misc = nullptr;               // pinned readback
    unsigned long long* h_total = nullptr;
    DevScalars* h_sc = nullptr;          // pinned initial scalars
    std::thread worker;
};

struct ServeEngine {
    int device = 0;
    Geom base{};                 // ndim, B, S, K, P of the context
    int32_t max_observed = 0;
    bool stream_dictionary = false;
    bool full_s = false;                 // SENSAI_FLAG_GAMMA_S_FULL of the context
    int slice_atoms = 0;
    long long max_pixels = 0;
    long long budget = 0;
    long long in_flight = 0;
    double a_over_K = 0, b_param = 0;
    double c = 0, d = 0, e = 0, f = 0;
    uint64_t seed = 0;
    uint32_t t0 = 0;
    double gamma_s = 1, gamma_eps = 1;
    float* D = nullptr;          // snapshot of the dictionary [K][P]
    double* pi = nullptr;        // snapshot of pi [K]
    std::vector<ServeSlot*> slots;
    std::deque<ServeRequest> queue;
    int busy = 0;
    bool stop = false;
    sensai_status first_status = SENSAI_OK;   // first failure since the last drain
    std::string first_error;
    std::mutex mu;
    std::condition_variable cv_work, cv_idle;
};

// Device bytes a frame of geometry g occupies in a slot (what admission counts).
static size_t frame_bytes(const Geom& g, int max_observed)
{
    const size_t nmw = (size_t)((g.nframe + 31) / 32);
    size_t b = 0;
    b += sizeof(float) * 2 * (size_t)g.nframe + (size_t)g.nframe + sizeof(uint32_t) * nmw;   // x, out, mask
    b += sizeof(uint16_t) * (size_t)g.N * (1 + (size_t)max_observed);                       // nobs, obs
    b += sizeof(float) * (size_t)g.KB * kAtomBlock * (size_t)g.Npad;                        // W
    b += sizeof(uint32_t) * (size_t)g.K * g.NW + 4 * sizeof(double) * g.NW;                  // Zb, partials
    b += sizeof(float) * (size_t)g.P * (size_t)g.N;                                         // Y
    return b;
}

// Geometry of a frame of shape M with the context's patch shape and stride.
static bool frame_geom(const Geom& base, const int64_t* M, Geom* out)
{
    Geom g = base;
    long long N = 1, nframe = 1;
    for (int d = 0; d < base.ndim; ++d) {
        if (M[d] < base.B[d] || (M[d] - base.B[d]) % base.S[d] != 0) return false;
        g.M[d] = M[d];
        g.G[d] = (M[d] - base.B[d]) / base.S[d] + 1;
        N *= g.G[d];
        nframe *= M[d];
    }
    if (N >= (1LL << 31) || nframe >= (1LL << 31)) return false;
    long long s = 1;
    for (int d = base.ndim - 1; d >= 0; --d) {
        g.fs[d] = s;
        s *= g.M[d];
    }
    g.N = N;
    g.NW = (int)((N + 31) / 32);
    g.Npad = (long long)g.NW * 32;
    g.nframe = nframe;
    *out = g;
    return true;
}

}  // namespace sensai

namespace sensai {

static void free_slot(ServeSlot* s)
{
    void* dev[] = {s->x, s->mask_bytes, s->mask_bits, s->imgoff, s->nobs, s->obs, s->misc, s->total, s->W, s->Zb,
                   s->m, s->part_s2, s->part_r2, s->counter, s->sc, s->pi, s->lpi, s->Y, s->out, s->Dsl, s->Dc};
    for (void* p : dev)
        if (p) cudaFree(p);
    if (s->h_misc) cudaFreeHost(s->h_misc);
    if (s->h_total) cudaFreeHost(s->h_total);
    if (s->h_sc) cudaFreeHost(s->h_sc);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

template <typename T>
static cudaError_t slot_alloc(T** p, size_t count)
{
    return cudaMalloc((void**)p, sizeof(T) * (count > 0 ? count : 1));
}

// Buffers for the largest accepted frame (max_pixels pixels).
static cudaError_t alloc_slot(ServeEngine* e, ServeSlot* s)
{
    const Geom& b = e->base;
    const size_t px = (size_t)e->max_pixels;
    const size_t nw = (px + 31) / 32, npad = nw * 32;
    cudaError_t r;
#define SLOT_TRY(x)                       \
    do {                                  \
        if ((r = (x)) != cudaSuccess) return r; \
    } while (0)
    SLOT_TRY(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
    SLOT_TRY(slot_alloc(&s->x, px));
    SLOT_TRY(slot_alloc(&s->out, px));
    SLOT_TRY(slot_alloc(&s->mask_bytes, px));
    SLOT_TRY(slot_alloc(&s->mask_bits, nw));
    SLOT_TRY(slot_alloc(&s->imgoff, (size_t)b.P));
    SLOT_TRY(slot_alloc(&s->nobs, px));
    SLOT_TRY(slot_alloc(&s->obs, (size_t)e->max_observed * px));
    SLOT_TRY(slot_alloc(&s->misc, 2));
    SLOT_TRY(slot_alloc(&s->total, 1));
    SLOT_TRY(slot_alloc(&s->W, (size_t)b.KB * kAtomBlock * npad));
    SLOT_TRY(slot_alloc(&s->Zb, (size_t)b.K * nw));
    SLOT_TRY(slot_alloc(&s->m, (size_t)b.K + 1));   // [K] counts, then the draw kernel's arrival counter
    SLOT_TRY(cudaMemset(s->m, 0, sizeof(int) * ((size_t)b.K + 1)));
    SLOT_TRY(slot_alloc(&s->part_s2, 2 * nw));   // per 16- or 32-patch work unit
    SLOT_TRY(slot_alloc(&s->part_r2, 2 * nw));
    SLOT_TRY(slot_alloc(&s->counter, 1));
    SLOT_TRY(slot_alloc(&s->sc, 1));
    SLOT_TRY(slot_alloc(&s->pi, (size_t)b.K));
    SLOT_TRY(slot_alloc(&s->lpi, (size_t)b.K));
    SLOT_TRY(slot_alloc(&s->Y, (size_t)b.P * px));
    if (recon_tc_available(b)) SLOT_TRY(slot_alloc(&s->Dc, recon_tc_operand_floats(b)));
    SLOT_TRY(slot_alloc(&s->Dsl, (size_t)slice_capacity_floats(b)));
    SLOT_TRY(cudaMallocHost((void**)&s->h_misc, 2 * sizeof(int)));
    SLOT_TRY(cudaMallocHost((void**)&s->h_total, sizeof(unsigned long long)));
    SLOT_TRY(cudaMallocHost((void**)&s->h_sc, sizeof(DevScalars)));
#undef SLOT_TRY
    return cudaSuccess;
}

static void note_error(ServeEngine* e, sensai_status st, const char* what, const char* where)
{
    std::lock_guard<std::mutex> lk(e->mu);
    if (e->first_status != SENSAI_OK) return;
    char buf[384];
    snprintf(buf, sizeof(buf), "serving: %s in %s", what, where);
    e->first_status = st;
    e->first_error = buf;
}

// One frame on one slot: geometry, cleared codes, `sweeps` x (code sweep +
// pi / gamma draws), overlap-add, copy out.  Synchronous on the slot's stream.
static sensai_status process_frame(ServeEngine* e, ServeSlot* sl, const ServeRequest& q)
{
    const Geom& g = q.g;
    const cudaStream_t s = sl->stream;
    const uint64_t fseed = serve_frame_seed(e->seed, q.stream_id, q.frame_id);
    cudaError_t r;
#define FRAME_TRY(x)                                                                       \
    do {                                                                                   \
        if ((r = (x)) != cudaSuccess) {                                                    \
            cudaGetLastError();                                                            \
            note_error(e, r == cudaErrorMemoryAllocation ? SENSAI_ENOMEM : SENSAI_ECUDA,    \
                       cudaGetErrorString(r), #x);                                         \
            return r == cudaErrorMemoryAllocation ? SENSAI_ENOMEM : SENSAI_ECUDA;           \
        }                                                                                  \
    } while (0)
    FRAME_TRY(cudaMemcpyAsync(sl->x, q.frame, sizeof(float) * (size_t)g.nframe, cudaMemcpyHostToDevice, s));
    FRAME_TRY(cudaMemcpyAsync(sl->mask_bytes, q.mask, (size_t)g.nframe, cudaMemcpyHostToDevice, s));
    FRAME_TRY(cudaMemsetAsync(sl->misc, 0, 2 * sizeof(int), s));
    FRAME_TRY(cudaMemsetAsync(sl->total, 0, sizeof(unsigned long long), s));
    FRAME_TRY(launch_geometry(g, sl->mask_bytes, sl->mask_bits, sl->imgoff, sl->nobs, sl->misc, sl->total, s));
    FRAME_TRY(cudaMemcpyAsync(sl->h_misc, sl->misc, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    FRAME_TRY(cudaMemcpyAsync(sl->h_total, sl->total, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    FRAME_TRY(cudaStreamSynchronize(s));
    const int maxobs = sl->h_misc[0];
    if (maxobs > e->max_observed) {
        note_error(e, SENSAI_EINVAL, "a patch observes more pixels than max_observed", "frame geometry");
        return SENSAI_EINVAL;
    }
    const long long n_observed = (long long)*sl->h_total;
    FRAME_TRY(launch_fill_obs(g, sl->mask_bits, sl->imgoff, sl->obs, s));

    // cleared codes and the transferred pi / gamma
    FRAME_TRY(cudaMemsetAsync(sl->W, 0, sizeof(float) * (size_t)g.KB * kAtomBlock * (size_t)g.Npad, s));
    FRAME_TRY(cudaMemsetAsync(sl->Zb, 0, sizeof(uint32_t) * (size_t)g.K * g.NW, s));
    FRAME_TRY(cudaMemcpyAsync(sl->pi, e->pi, sizeof(double) * g.K, cudaMemcpyDeviceToDevice, s));
    FRAME_TRY(launch_logit(g.K, sl->pi, sl->lpi, s));
    std::memset(sl->h_sc, 0, sizeof(DevScalars));
    sl->h_sc->gamma_s = e->gamma_s;
    sl->h_sc->gamma_eps = e->gamma_eps;
    sl->h_sc->ge_set = 1;
    FRAME_TRY(cudaMemcpyAsync(sl->sc, sl->h_sc, sizeof(DevScalars), cudaMemcpyHostToDevice, s));

    SweepPlan plan{};
    if (!plan_sweep(g, maxobs, e->device, e->stream_dictionary, e->slice_atoms, &plan)) {
        note_error(e, SENSAI_ECUDA, "no launch configuration", "plan_sweep");
        return SENSAI_ECUDA;
    }
    const double b = e->b_param > 0 ? e->b_param : (double)g.N / 8.0;
    for (int sw = 0; sw < q.sweeps; ++sw) {
        SweepArgs a{};
        a.g = g;
        a.x = sl->x;
        a.obs = sl->obs;
        a.nobs = sl->nobs;
        a.imgoff = sl->imgoff;
        a.D = e->D;
        a.W = sl->W;
        a.Zb = sl->Zb;
        a.lpi = sl->lpi;
        a.sc = sl->sc;
        a.R = nullptr;   // inpainting keeps no per-pixel residual
        a.part_s2 = sl->part_s2;
        a.part_r2 = sl->part_r2;
        a.chunk_counter = sl->counter;
        a.sc_out = sl->sc;
        a.keys = philox_round_keys(fseed);
        a.t = e->t0 + (uint32_t)sw;
        FRAME_TRY(launch_code_sweep(a, plan, maxobs, sl->Dsl, s, nullptr));
        if (e->full_s) FRAME_TRY(launch_prior_s2(g, sl->Zb, nullptr, sl->sc, a.t, false, fseed, plan.lanes, sl->part_s2, s));
        HyperArgs h{};
        h.g = g;
        h.Zb = sl->Zb;
        h.m = sl->m;
        h.arrive = reinterpret_cast<unsigned int*>(sl->m + g.K);
        h.part_s2 = sl->part_s2;
        h.n_s2 = g.NW * plan.lanes;
        h.part_r2 = sl->part_r2;
        h.n_r2 = g.NW * plan.lanes;
        h.n_observed = n_observed;
        h.a_over_K = e->a_over_K;
        h.b_scaled = b * (g.K - 1) / g.K;
        h.c = e->c;
        h.d = e->d;
        h.e = e->e;
        h.f = e->f;
        h.pi = sl->pi;
        h.lpi = sl->lpi;
        h.sc = sl->sc;
        h.seed = fseed;
        h.t = e->t0 + (uint32_t)sw;
        h.full_s = e->full_s;
        FRAME_TRY(launch_hyper(h, s));
    }
    FRAME_TRY(launch_reconstruct(g, e->D, sl->Dc, sl->W, sl->Y, sl->out, &sl->sc->status, s));
    FRAME_TRY(cudaMemcpyAsync(q.out, sl->out, sizeof(float) * (size_t)g.nframe, cudaMemcpyDeviceToHost, s));
    FRAME_TRY(cudaMemcpyAsync(sl->h_misc + 1, &sl->sc->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    FRAME_TRY(cudaStreamSynchronize(s));
#undef FRAME_TRY
    if (sl->h_misc[1] != 0) {
        note_error(e, SENSAI_ETIMEOUT, "a device-side wait timed out", "frame kernels");
        return SENSAI_ETIMEOUT;
    }
    return SENSAI_OK;
}

}  // namespace sensai

namespace sensai {

static void worker_loop(ServeEngine* e, ServeSlot* sl)
{
    cudaSetDevice(e->device);
    for (;;) {
        ServeRequest q;
        {
            std::unique_lock<std::mutex> lk(e->mu);
            e->cv_work.wait(lk, [&] {
                return e->stop || (!e->queue.empty() && e->in_flight + (long long)e->queue.front().bytes <= e->budget);
            });
            if (e->queue.empty()) return;   // stop with nothing left
            q = e->queue.front();
            e->queue.pop_front();
            e->in_flight += (long long)q.bytes;
            ++e->busy;
        }
        const sensai_status st = process_frame(e, sl, q);
        {
            std::lock_guard<std::mutex> lk(e->mu);
            e->in_flight -= (long long)q.bytes;
        }
        e->cv_work.notify_all();
        if (q.done) q.done(q.user, q.frame_id, (int32_t)st);
        {
            std::lock_guard<std::mutex> lk(e->mu);
            --e->busy;
            if (e->busy == 0 && e->queue.empty()) e->cv_idle.notify_all();
        }
    }
}

ServeEngine* serve_create(const ServeInit& in, sensai_status* status)
{
    ServeEngine* e = new ServeEngine();
    e->device = in.device;
    e->base = in.base;
    e->max_observed = in.max_observed;
    e->stream_dictionary = in.stream_dictionary;
    e->slice_atoms = in.slice_atoms;
    e->full_s = in.full_s;
    e->max_pixels = in.max_pixels;
    e->a_over_K = in.a_over_K;
    e->b_param = in.b_param;
    e->c = in.c;
    e->d = in.d;
    e->e = in.e;
    e->f = in.f;
    e->seed = in.seed;
    e->t0 = in.t0;
    e->gamma_s = in.gamma_s;
    e->gamma_eps = in.gamma_eps;
    *status = SENSAI_OK;
    cudaError_t r = cudaSetDevice(in.device);
    if (r == cudaSuccess) r = preload_sweep_variants();   // no first-use loading while frames are timed
    const size_t dsz = sizeof(float) * (size_t)in.base.K * in.base.P;
    if (r == cudaSuccess) r = cudaMalloc((void**)&e->D, dsz);
    if (r == cudaSuccess) r = cudaMalloc((void**)&e->pi, sizeof(double) * in.base.K);
    if (r == cudaSuccess) r = cudaMemcpy(e->D, in.D, dsz, cudaMemcpyDeviceToDevice);
    if (r == cudaSuccess) r = cudaMemcpy(e->pi, in.pi, sizeof(double) * in.base.K, cudaMemcpyDeviceToDevice);
    // a frame of max_pixels pixels bounds every slot's footprint
    Geom worst = in.base;
    worst.N = in.max_pixels;
    worst.NW = (int)((in.max_pixels + 31) / 32);
    worst.Npad = (long long)worst.NW * 32;
    worst.nframe = in.max_pixels;
    const long long worst_bytes = (long long)frame_bytes(worst, in.max_observed);
    e->budget = in.memory_budget > 0 ? in.memory_budget : worst_bytes * in.slots;
    for (int i = 0; r == cudaSuccess && i < in.slots; ++i) {
        ServeSlot* sl = new ServeSlot();
        e->slots.push_back(sl);
        r = alloc_slot(e, sl);
    }
    if (r != cudaSuccess) {
        cudaGetLastError();
        *status = r == cudaErrorMemoryAllocation ? SENSAI_ENOMEM : SENSAI_ECUDA;
        for (ServeSlot* sl : e->slots) free_slot(sl);
        if (e->D) cudaFree(e->D);
        if (e->pi) cudaFree(e->pi);
        delete e;
        return nullptr;
    }
    for (ServeSlot* sl : e->slots) sl->worker = std::thread(worker_loop, e, sl);
    return e;
}

sensai_status serve_submit(ServeEngine* e, int32_t stream_id, uint64_t frame_id, const float* frame,
                           const uint8_t* mask, const int64_t* M, int32_t sweeps, float* out, sensai_done_fn done,
                           void* user)
{
    if (!frame || !mask || !out || !M || sweeps < 0) return SENSAI_EINVAL;
    ServeRequest q{};
    if (!frame_geom(e->base, M, &q.g) || q.g.nframe > e->max_pixels) return SENSAI_EINVAL;
    q.bytes = frame_bytes(q.g, e->max_observed);
    if ((long long)q.bytes > e->budget) return SENSAI_EINVAL;
    q.stream_id = stream_id;
    q.frame_id = frame_id;
    q.frame = frame;
    q.mask = mask;
    q.out = out;
    q.sweeps = sweeps;
    q.done = done;
    q.user = user;
    {
        std::lock_guard<std::mutex> lk(e->mu);
        if (e->stop) return SENSAI_ESTATE;
        e->queue.push_back(q);
    }
    e->cv_work.notify_all();
    return SENSAI_OK;
}

sensai_status serve_drain(ServeEngine* e, std::string* message)
{
    std::unique_lock<std::mutex> lk(e->mu);
    e->cv_idle.wait(lk, [&] { return e->queue.empty() && e->busy == 0; });
    const sensai_status st = e->first_status;
    if (message) *message = e->first_error;
    e->first_status = SENSAI_OK;
    e->first_error.clear();
    return st;
}

void serve_destroy(ServeEngine* e)
{
    serve_drain(e, nullptr);
    {
        std::lock_guard<std::mutex> lk(e->mu);
        e->stop = true;
    }
    e->cv_work.notify_all();
    for (ServeSlot* sl : e->slots)
        if (sl->worker.joinable()) sl->worker.join();
    cudaSetDevice(e->device);
    for (ServeSlot* sl : e->slots) free_slot(sl);
    if (e->D) cudaFree(e->D);
    if (e->pi) cudaFree(e->pi);
    delete e;
}

}  // namespace sensai
