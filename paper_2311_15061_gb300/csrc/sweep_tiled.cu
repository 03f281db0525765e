// sweep_tiled.cu -- the sparse-code sweep for dictionaries larger than shared
// memory (3-D video and spectral cubes: K = 256 atoms of P = 256 pixels is
// 257 KB in FP32).
//
// Same draws, same order and same arithmetic per atom as sweep.cu (both run
// sweep_block.cuh); only the dictionary's path differs.  A CTA takes work
// items of 8 consecutive 32-patch chunks, one per warp, and keeps every
// patch's residual in registers for the whole item.  The dictionary is
// streamed through two shared-memory slice buffers of KS atoms each, in the
// same [p][k] layout (odd pitch, zero row p = P) as the resident kernel.  A
// slice is one 1-D bulk copy (cp.async.bulk, the TMA engine) from a
// pre-laid-out global copy, completing on an mbarrier.  Per item the CTA
// passes over the slices twice: once to rebuild the residual from the stored
// weights and once for the atom-ordered sweep.  While the CTA works on one
// buffer, the copy of the next-but-one slice fills the other.  Slice
// boundaries are CTA barriers (the only ones).  Every mbarrier wait is
// bounded: on timeout the status word gets SENSAI_ETIMEOUT and the CTA stops.
#include "sweep_block.cuh"

namespace sensai {

constexpr int kTiledThreads = 256;
constexpr int kTiledWarps = kTiledThreads / 32;
constexpr long long kMbarSpins = 1LL << 20;   // try_wait polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Arrive (count 1) and announce the bytes the bulk copy will deliver.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of the barrier; false after kMbarSpins polls or
// kWaitLimitNs, whichever comes first (the global timer, a slow read, only
// once the first poll has failed).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    unsigned long long t0 = 0;
    for (long long spins = 0; spins < kMbarSpins; ++spins) {
        if (mbar_try_wait(bar, parity)) return true;
        if (spins == 0) t0 = global_ns();
        else if ((spins & 63) == 0 && global_ns() - t0 > kWaitLimitNs) break;
    }
    return false;
}

// Self-test of the bounded wait: an mbarrier that nothing completes.  One
// thread; writes SENSAI_ETIMEOUT to *status when the wait gives up.
__global__ void mbar_timeout_selftest_kernel(int* status)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *status = mbar_wait(&bar, 0) ? (int)SENSAI_OK : (int)SENSAI_ETIMEOUT;
}

cudaError_t launch_mbar_timeout_selftest(int* status, cudaStream_t s)
{
    mbar_timeout_selftest_kernel<<<1, 32, 0, s>>>(status);
    return cudaGetLastError();
}

// Slice s of the dictionary in its shared-memory layout: [P + 1][ldS] with
// ldS = KS + 1, column 0 zero and entry (p, 1 + kk) = d_{s KS + kk, p}; zero
// for p = P and atoms >= K.
__global__ void slice_dictionary_kernel(Geom g, const float* D, float* Dsl, int KS, int ldS, long long stride,
                                        int S)
{
    const long long total = (long long)S * stride;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(idx / stride);
        const long long e = idx - (long long)s * stride;
        const int p = (int)(e / ldS), kk = (int)(e - (long long)p * ldS) - kDictColumnOffset;
        const int k = s * KS + kk;
        float v = 0.0f;
        if (p < g.P && kk >= 0 && kk < KS && k < g.K) v = D[(long long)k * g.P + p];
        Dsl[idx] = v;
    }
}

template <int MAXOBS, int LANES>
__device__ __forceinline__ void tiled_body(const SweepArgs& a)
{
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ unsigned int item_s;
    __shared__ int abort_s;
    const int K = a.g.K, KB = a.g.KB;
    const int Kpad = KB * kAtomBlock;
    const int KS = a.slice_atoms, ldS = KS + kDictColumnOffset, S = a.slices;
    const long long stride = a.slice_stride;
    const uint32_t slice_bytes = (uint32_t)(stride * sizeof(float));
    const long long N = a.g.N, Npad = a.g.Npad;
    const int NW = a.g.NW;
    float* buf0 = smem;
    float* buf1 = smem + stride;
    float* lpi = smem + 2 * stride;        // Kpad
    const unsigned int units = (unsigned int)NW * LANES;   // 32-patch chunks, or 16-patch halves
    const long long nitems = (units + kTiledWarps - 1) / kTiledWarps;

    // logit(pi_k) + ln(gamma_s) / 2: the log-odds terms that do not depend on the patch
    const float half_log_gs = code_const(a.sc).half_log_gs;
    for (int k = threadIdx.x; k < Kpad; k += blockDim.x) lpi[k] = (k < K ? a.lpi[k] : 0.0f) + half_log_gs;
    if (threadIdx.x == 0) {
        abort_s = 0;
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        // uses 0 and 1 are slices 0 and 1 % S
        for (int b = 0; b < 2; ++b) {
            mbar_expect_tx(&bar[b], slice_bytes);
            bulk_copy_g2s(b ? buf1 : buf0, a.Dsl + (long long)(b % S) * stride, slice_bytes, &bar[b]);
        }
    }
    __syncthreads();

    const CodeConst c = code_const(a.sc);
    const uint32_t t_it = launch_t(a.t, a.t_dev, a.sc);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int half = LANES == 1 ? 0 : (lane & 1);
    CodeTally tl;
    // Use q of the slice buffers reads slice q % S from buffer q & 1 (each
    // item makes 2 S consecutive uses, or S when the residual is read from
    // the previous phase instead of rebuilt).  With S <= 2 both buffers keep
    // their first slices and are never refilled.
    long long q = 0;
    bool ok = true;

    for (;;) {
        if (threadIdx.x == 0) item_s = atomicAdd(a.chunk_counter, 1u);
        __syncthreads();
        const unsigned int item = item_s;
        __syncthreads();
        if (item >= (unsigned int)nitems) break;
        const unsigned int unit = item * kTiledWarps + warp;
        const bool warp_on = unit < units;
        const long long slot = (long long)unit * PatchLanes<LANES>::kPatchesPerWarp + lane / LANES;
        const long long i = warp_on ? slot_patch(a, slot) : N;
        LanePatch lp;
        lp.i = i;
        lp.valid = warp_on && i < N;
        lp.nobs = lp.valid ? (int)a.nobs[slot] : 0;
        lp.unit = unit;
        lp.lane = lane;
        const int nl = LANES == 1 ? lp.nobs : (lp.nobs + 1 - half) / 2;   // this lane's pixels
        lp.wmax = __reduce_max_sync(0xffffffffu, nl);
        const long long org = lp.valid ? patch_origin(a.g, i) : 0;
        const long long irec = warp_on ? i : 0;    // i < Npad: padding patches have zero records

        PixelAddr<MAXOBS> ad;
        ad.base = smem_addr(buf0) + 4u * kDictColumnOffset;
        ad.pitch = 4u * ldS;
        Resid<MAXOBS> r;
        const bool from_resid = a.R_in != nullptr;
        gather_patch<MAXOBS, LANES>(a, lp.valid ? slot : 0, nl, org, ad, r, half, from_resid);

        float s2 = 0.0f;
        begin_patch_counts(tl);
        W8 nb;
        AtomCarry carry;
        carry.dw = 0.0f;
        carry.cur = code_pair(i, 0, t_it, a.keys);
        for (int pass = from_resid ? 1 : 0; pass < 2 && ok; ++pass) {
            for (int sl = 0; sl < S; ++sl, ++q) {
                const int b = (int)(q & 1);
                float* Dbuf = b ? buf1 : buf0;
                const bool fresh = S > 2 || q < 2;   // a copy is pending on this buffer
                if (fresh && !mbar_wait(&bar[b], (uint32_t)((S > 2 ? (q >> 1) : 0) & 1))) {
                    atomicExch(&a.sc_out->status, (int)SENSAI_ETIMEOUT);
                    abort_s = 1;
                }
                __syncthreads();
                if (abort_s) { ok = false; break; }
                const int kb0 = sl * (KS / kAtomBlock);
                const int kb1 = min(KB, kb0 + KS / kAtomBlock);
                const uint32_t col0 = smem_addr(Dbuf) + 4u * kDictColumnOffset;
                if (warp_on) {
                    if (pass == 0) {
                        for (int kb = kb0; kb < kb1; ++kb) {
                            ad.rebase(col0 + 32u * (kb - kb0), lp.wmax);
                            const W8 wb = load_w8(a.W + ((long long)kb * Npad + irec) * kAtomBlock);
                            rebuild_block<MAXOBS>(ad, r, lp.wmax, wb);
                            tl.rb_obs += (unsigned int)nl * w8_nonzero(wb);
                        }
                    } else {
                        if (sl == 0) nb = load_w8(a.W + irec * kAtomBlock);
                        for (int kb = kb0; kb < kb1; ++kb) {
                            W8 wb = nb;
                            if (kb + 1 < KB) nb = load_w8(a.W + ((long long)(kb + 1) * Npad + irec) * kAtomBlock);
                            const int kbase = kb * kAtomBlock;
                            ad.rebase(col0 + 32u * (kb - kb0), lp.wmax);
                            const bool changed = code_block<MAXOBS, LANES, false>(
                                ad, r, lpi + kbase, lp, kbase, K, c, a.keys, t_it, a.Zb, NW, wb, carry, s2, tl);
                            if (half == 0 && changed && lp.valid)
                                store_w8(a.W + ((long long)kb * Npad + i) * kAtomBlock, wb.v[0], wb.v[1], wb.v[2],
                                         wb.v[3], wb.v[4], wb.v[5], wb.v[6], wb.v[7]);
                        }
                    }
                }
                __syncthreads();   // every warp is done with this buffer
                if (S > 2 && threadIdx.x == 0) {
                    mbar_expect_tx(&bar[b], slice_bytes);
                    bulk_copy_g2s(Dbuf, a.Dsl + (long long)((q + 2) % S) * stride, slice_bytes, &bar[b]);
                }
            }
        }
        if (!ok) break;
        end_patch_counts(tl, lp.nobs);
        if (warp_on) finish_patch<MAXOBS, LANES>(a, r, lp.wmax, nl, slot, unit, lane, s2);
    }
    // The copies still in flight land before the CTA exits: uses q and q + 1
    // when buffers are refilled, else the initial copies not yet waited for.
    if (ok && threadIdx.x == 0) {
        const long long u_end = S > 2 ? q + 2 : 2;
        for (long long u = q; u < u_end; ++u) {
            const int b = (int)(u & 1);
            if (!mbar_wait(&bar[b], (uint32_t)((S > 2 ? (u >> 1) : 0) & 1)))
                atomicExch(&a.sc_out->status, (int)SENSAI_ETIMEOUT);
        }
    }
    flush_counts(a, lane, tl);
}

template <int MAXOBS, int LANES>
__global__ void __launch_bounds__(kTiledThreads, (MAXOBS <= 48 && LANES == 1 ? 2 : 1)) sweep_tiled_kernel(const SweepArgs a)
{
    tiled_body<MAXOBS, LANES>(a);
}

// Batched instances in one launch (see sweep_multi_kernel); each instance
// streams its own dictionary slices.
template <int MAXOBS, int LANES>
__global__ void __launch_bounds__(kTiledThreads, (MAXOBS <= 48 && LANES == 1 ? 2 : 1))
    sweep_tiled_multi_kernel(const SweepArgs* __restrict__ args, const int* __restrict__ cta_start, int n)
{
    const SweepArgs& a = *stage_instance_args(args, cta_start, n);
    tiled_body<MAXOBS, LANES>(a);
}

template <int MAXOBS, int LANES = 1>
static void* tiled_ptr(bool multi)
{
    return multi ? (void*)sweep_tiled_multi_kernel<MAXOBS, LANES> : (void*)sweep_tiled_kernel<MAXOBS, LANES>;
}

static void* select_tiled(int maxobs, bool multi = false)
{
    if (maxobs > 96) {   // two lanes per patch: per-lane capacity 64 / 96 / 112 / 128
        if (maxobs <= 128) return tiled_ptr<64, 2>(multi);
        if (maxobs <= 192) return tiled_ptr<96, 2>(multi);
        if (maxobs <= 224) return tiled_ptr<112, 2>(multi);
        if (maxobs <= 256) return tiled_ptr<128, 2>(multi);
        return nullptr;
    }
    if (maxobs <= 8) return tiled_ptr<8>(multi);
    if (maxobs <= 16) return tiled_ptr<16>(multi);
    if (maxobs <= 24) return tiled_ptr<24>(multi);
    if (maxobs <= 32) return tiled_ptr<32>(multi);
    if (maxobs <= 40) return tiled_ptr<40>(multi);
    if (maxobs <= 48) return tiled_ptr<48>(multi);
    if (maxobs <= 64) return tiled_ptr<64>(multi);
    if (maxobs <= 72) return tiled_ptr<72>(multi);
    if (maxobs <= 80) return tiled_ptr<80>(multi);
    return tiled_ptr<96>(multi);
}

cudaError_t preload_tiled_variants()
{
    const int obs[] = {8, 16, 24, 32, 40, 48, 64, 72, 80, 96, 128, 192, 224, 256};
    for (int m : obs) {
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, select_tiled(m));
        if (e != cudaSuccess) return e;
    }
    cudaFuncAttributes fa;
    return cudaFuncGetAttributes(&fa, (void*)slice_dictionary_kernel);
}

long long slice_stride_floats(const Geom& g, int KS)
{
    const long long n = (long long)(g.P + 1) * (KS + kDictColumnOffset);
    return (n + 3) & ~3LL;   // whole 16-byte units: bulk copies move multiples of 16 bytes
}

size_t tiled_smem_bytes(const Geom& g, int KS)
{
    const int Kpad = g.KB * kAtomBlock;
    return sizeof(float) * (2 * (size_t)slice_stride_floats(g, KS) + Kpad);
}

// Largest slice (a multiple of 8 atoms, at most the padded K) whose two
// buffers fit the shared memory of one CTA at the variant's occupancy.
int tiled_slice_atoms(const Geom& g, int maxobs, int device)
{
    int per_sm_smem = 0, optin = 0;
    if (cudaDeviceGetAttribute(&per_sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device) != cudaSuccess)
        return 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) return 0;
    const int ctas = maxobs <= 48 ? 2 : 1;   // the variant's occupancy (two-lane variants: 1)
    const size_t reserve = 1024 + 64;   // per-CTA system reserve and the static barriers
    size_t budget = (size_t)per_sm_smem / ctas;
    budget = budget > reserve ? budget - reserve : 0;
    if (budget > (size_t)optin) budget = (size_t)optin;
    const int Kpad = g.KB * kAtomBlock;
    int best = 0;
    for (int KS = kAtomBlock; KS <= Kpad; KS += kAtomBlock)
        if (tiled_smem_bytes(g, KS) <= budget) best = KS;
    return best;
}

cudaError_t launch_slice_dictionary(const Geom& g, const float* D, float* Dsl, int KS, cudaStream_t s)
{
    const int S = (g.KB * kAtomBlock + KS - 1) / KS;
    const long long stride = slice_stride_floats(g, KS);
    const long long total = (long long)S * stride;
    const int threads = 256;
    long long blocks = (total + threads - 1) / threads;
    if (blocks > 1024) blocks = 1024;
    slice_dictionary_kernel<<<(unsigned int)blocks, threads, 0, s>>>(g, D, Dsl, KS, KS + kDictColumnOffset, stride,
                                                                    S);
    return cudaGetLastError();
}

int tiled_grid_size(const Geom& g, int maxobs, int KS, int device)
{
    void* fn = select_tiled(maxobs);
    if (!fn || KS < kAtomBlock) return 0;
    const int smem = (int)tiled_smem_bytes(g, KS);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 0;
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kTiledThreads, smem) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    if (per_sm < 1) return 0;
    const long long items = ((long long)g.NW * sweep_lanes(maxobs) + kTiledWarps - 1) / kTiledWarps;
    const long long grid = (long long)per_sm * sms;
    return (int)(grid < items ? grid : items);
}

cudaError_t launch_sweep_tiled_multi(const SweepArgs* args, const int* cta_start, int n, int maxobs, int grid,
                                     size_t smem, cudaStream_t s)
{
    void* fn = select_tiled(maxobs, true);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void* kargs[] = {(void*)&args, (void*)&cta_start, (void*)&n};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kTiledThreads), kargs, smem, s);
}

int sweep_tiled_multi_ctas_per_sm(int maxobs, size_t smem)
{
    void* fn = select_tiled(maxobs, true);
    int per_sm = 0;
    if (!fn || cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kTiledThreads, smem) != cudaSuccess)
        return 0;
    return per_sm;
}

cudaError_t launch_sweep_tiled(const SweepArgs& a, int maxobs, int grid, cudaStream_t s)
{
    void* fn = select_tiled(maxobs);
    if (!fn || !a.Dsl || a.slice_atoms < kAtomBlock || a.slices < 1) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(a.chunk_counter, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    const int smem = (int)tiled_smem_bytes(a.g, a.slice_atoms);
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    void* args[] = {(void*)&a};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kTiledThreads), args, (size_t)smem, s);
}

// Floats the slice buffer needs for any slice size of this geometry.
long long slice_capacity_floats(const Geom& g)
{
    const int Kpad = g.KB * kAtomBlock;
    long long best = 0;
    for (int KS = kAtomBlock; KS <= Kpad; KS += kAtomBlock) {
        const long long n = (long long)((Kpad + KS - 1) / KS) * slice_stride_floats(g, KS);
        if (n > best) best = n;
    }
    return best;
}

bool plan_sweep(const Geom& g, int maxobs, int device, bool force_stream, int force_slice_atoms, SweepPlan* out)
{
    SweepPlan p{};
    if (maxobs < 1) maxobs = 1;
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) return false;
    if (!force_stream && sweep_smem_bytes(g) <= optin) {
        p.grid = sweep_grid_size(g, maxobs, device);
        p.lanes = sweep_lanes(maxobs);
        *out = p;
        return p.grid > 0;
    }
    const int Kpad = g.KB * kAtomBlock;
    int KS = tiled_slice_atoms(g, maxobs, device);
    if (force_slice_atoms > 0) {
        if (force_slice_atoms % kAtomBlock != 0 || force_slice_atoms > Kpad || force_slice_atoms > KS) return false;
        KS = force_slice_atoms;
    }
    if (KS < kAtomBlock) return false;
    p.slice_atoms = KS;
    p.slices = (Kpad + KS - 1) / KS;
    p.slice_stride = slice_stride_floats(g, KS);
    p.grid = tiled_grid_size(g, maxobs, KS, device);
    p.lanes = sweep_lanes(maxobs);
    *out = p;
    return p.grid > 0;
}

cudaError_t launch_code_sweep(SweepArgs a, const SweepPlan& plan, int maxobs, float* Dsl, cudaStream_t s,
                              int* nlaunch)
{
    if (maxobs < 1) maxobs = 1;
    cudaError_t e;
    int n = 0;
    if (plan.slice_atoms == 0 && plan.split_units > 0) {
        e = launch_sweep_split(a, plan, maxobs, s);
        n = 2;
    } else if (plan.slice_atoms == 0) {
        e = launch_sweep(a, maxobs, plan.grid, s);
        n = 1;
    } else {
        if (!Dsl) return cudaErrorInvalidValue;
        e = launch_slice_dictionary(a.g, a.D, Dsl, plan.slice_atoms, s);
        if (e != cudaSuccess) return e;
        a.Dsl = Dsl;
        a.slice_atoms = plan.slice_atoms;
        a.slices = plan.slices;
        a.slice_stride = plan.slice_stride;
        e = launch_sweep_tiled(a, maxobs, plan.grid, s);
        n = 2;
    }
    if (e != cudaSuccess) return e;
    if (nlaunch) *nlaunch = n;
    return cudaSuccess;
}

}  // namespace sensai
