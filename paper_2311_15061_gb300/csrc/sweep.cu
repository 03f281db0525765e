// sweep.cu -- the sparse-code sweep (patch extraction fused in).
//
// For every patch i (in parallel) and every atom k in order (the sparse-coding
// step of the BPFA section), with r_i the residual of patch i on its observed
// pixels Omega_i:
//   n   = sum_{p in Omega_i} d_kp^2,   g = sum_{p in Omega_i} d_kp r_ip + w_ik n
//   lam = gamma_s + gamma_eps n
//   L   = logit(pi_k) + 1/2 ln(gamma_s / lam) + gamma_eps^2 g^2 / (2 lam)
//   z_ik = [ x_{k%2} < floor(sigmoid(L) 2^32) ],  x = Philox(i, floor(k/2), t, CODES)
//   s_ik = gamma_eps g / lam + lam^-1/2 BoxMuller_{k%2}(x2, x3)   if z_ik = 1
//   r_i -= d_k (w_new - w_old) on Omega_i
// (z with s integrated out, then s | z = 1; inactive weights are not stored).
//
// GB300 mapping: one thread owns one patch (above 96 observed pixels a lane
// pair, see sweep_block.cuh); a warp owns 32 consecutive, 32-aligned patches
// so the atom's activity bits of the warp form one 32-bit word (ballot).
// Warps pull 32-patch chunks from a global counter, so the tail of the grid is
// a single chunk per warp.  Weights are read and written in 8-atom blocks (one
// 256-bit access per lane, 1 KB per warp), the next block prefetched behind
// the current one, so no global load sits on the per-atom path.  The
// dictionary sits in shared memory as [p][k] with an odd row pitch plus one
// zero row (p = P) that padded observation slots point at, so the inner loops
// need no predicates.  The residual of the patch lives in registers (MAXOBS
// slots, chosen per problem from the largest |Omega_i|).  Patch extraction is
// fused: at the start of each sweep the residual of a patch's observed pixels
// is read from the layout the dictionary kernel keeps it in (or, where no
// residual is kept, the observed pixels are gathered from the frame and the
// residual rebuilt from the stored weights).  At the end the residual is
// written back, through the position table, for the dictionary kernel.  The per-block code is in sweep_block.cuh,
// shared with the streamed-dictionary kernel (sweep_tiled.cu); the batched
// kernel runs the same body on per-instance arguments.
#include "sweep_block.cuh"

namespace sensai {

constexpr int kSweepThreads = 256;
constexpr int kSweepWarps = kSweepThreads / 32;

template <int MAXOBS, int LANES>
__device__ __forceinline__ void sweep_body(const SweepArgs& a)
{
    extern __shared__ __align__(16) float smem[];
    const int K = a.g.K, P = a.g.P, KB = a.g.KB;
    const int Kpad = KB * kAtomBlock;
    const int ldK = Kpad + kDictColumnOffset;   // odd: rows fall in different banks
    const long long N = a.g.N, Npad = a.g.Npad;
    const int NW = a.g.NW;
    float* Ds = smem;                      // (P + 1) x ldK; row P, column 0 and atoms >= K are zero
    float* lpi = Ds + (P + 1) * ldK;       // Kpad
    __shared__ unsigned int chunk_slot[kSweepWarps];

    for (int idx = threadIdx.x; idx < (P + 1) * ldK; idx += blockDim.x) {
        const int p = idx / ldK, k = idx - p * ldK - kDictColumnOffset;
        Ds[idx] = (p < P && k >= 0 && k < K) ? a.D[(long long)k * P + p] : 0.0f;
    }
    const CodeConst c = code_const(a.sc);
    // logit(pi_k) + ln(gamma_s) / 2: the log-odds terms that do not depend on the patch
    for (int k = threadIdx.x; k < Kpad; k += blockDim.x) lpi[k] = (k < K ? a.lpi[k] : 0.0f) + c.half_log_gs;
    __syncthreads();

    const uint32_t t_it = launch_t(a.t, a.t_dev, a.sc);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int half = LANES == 1 ? 0 : (lane & 1);
    // 32-patch chunks, or 16-patch halves; a split launch takes a range
    const unsigned int units = a.unit_hi ? a.unit_hi : (unsigned int)NW * LANES;
    const uint32_t col0 = smem_addr(Ds) + 4u * kDictColumnOffset;   // atom 0's column, row 0
    CodeTally tl;

    for (;;) {
        if (lane == 0) chunk_slot[warp] = a.unit_lo + atomicAdd(a.chunk_counter, 1u);
        __syncwarp();
        const unsigned int unit = chunk_slot[warp];
        __syncwarp();
        if (unit >= units) break;
        const long long slot = (long long)unit * PatchLanes<LANES>::kPatchesPerWarp + lane / LANES;   // < Npad
        const long long i = slot_patch(a, slot);
        LanePatch lp;
        lp.i = i;
        lp.valid = i < N;
        lp.nobs = lp.valid ? (int)a.nobs[slot] : 0;
        lp.unit = unit;
        lp.lane = lane;
        const int nl = LANES == 1 ? lp.nobs : (lp.nobs + 1 - half) / 2;   // this lane's pixels
        lp.wmax = __reduce_max_sync(0xffffffffu, nl);
        const long long org = lp.valid ? patch_origin(a.g, i) : 0;

        PixelAddr<MAXOBS> ad;
        ad.base = col0;
        ad.pitch = 4u * ldK;
        Resid<MAXOBS> r;
        const bool from_resid = a.R_in != nullptr;
        gather_patch<MAXOBS, LANES>(a, slot, nl, org, ad, r, half, from_resid);

        // else the residual r = x - D w on the observed pixels, from the stored
        // weights (two blocks loaded ahead of their use)
        if (!from_resid) {
            W8 p0 = load_w8(a.W + (long long)i * kAtomBlock);
            W8 p1 = p0;
            if (KB > 1) p1 = load_w8(a.W + (Npad + i) * kAtomBlock);
            for (int kb = 0; kb < KB; ++kb) {
                const W8 wb = p0;
                p0 = p1;
                if (kb + 2 < KB) p1 = load_w8(a.W + ((long long)(kb + 2) * Npad + i) * kAtomBlock);
                ad.rebase(col0 + 32u * kb, lp.wmax);
                rebuild_block<MAXOBS>(ad, r, lp.wmax, wb);
                tl.rb_obs += (unsigned int)nl * w8_nonzero(wb);
            }
        }

        float s2 = 0.0f;
        begin_patch_counts(tl);
        AtomCarry carry;
        carry.dw = 0.0f;
        carry.cur = code_pair(i, 0, t_it, a.keys);
        W8 nb = load_w8(a.W + (long long)i * kAtomBlock);
        for (int kb = 0; kb < KB; ++kb) {
            W8 wb = nb;
            if (kb + 1 < KB)   // prefetch the next block behind this block's work
                nb = load_w8(a.W + ((long long)(kb + 1) * Npad + i) * kAtomBlock);
            const int kbase = kb * kAtomBlock;
            ad.rebase(col0 + 32u * kb, lp.wmax);
            const bool changed = code_block<MAXOBS, LANES, true>(ad, r, lpi + kbase, lp, kbase, K, c, a.keys, t_it,
                                                                 a.Zb, NW, wb, carry, s2, tl);
            if (half == 0 && changed)
                store_w8(a.W + ((long long)kb * Npad + i) * kAtomBlock, wb.v[0], wb.v[1], wb.v[2], wb.v[3], wb.v[4],
                         wb.v[5], wb.v[6], wb.v[7]);
        }
        apply_update<MAXOBS>(ad, r, lp.wmax, carry.dw);   // the last atom's rank-1 update
        end_patch_counts(tl, lp.nobs);
        finish_patch<MAXOBS, LANES>(a, r, lp.wmax, nl, slot, unit, lane, s2);
    }
    flush_counts(a, lane, tl);
}

// Resident CTAs per SM the register budget is set for: 2 up to 48 pixels,
// else 1.  (3 CTAs per SM for the 16-pixel kernel spill 76 bytes per
// thread and measured 3% slower than 2 without spills.)
template <int MAXOBS, int LANES>
constexpr int sweep_min_ctas()
{
    return LANES == 1 && MAXOBS <= 48 ? 2 : 1;
}

template <int MAXOBS, int LANES>
__global__ void __launch_bounds__(kSweepThreads, sweep_min_ctas<MAXOBS, LANES>()) sweep_kernel(const SweepArgs a)
{
    sweep_body<MAXOBS, LANES>(a);
}

// Batched instances in one launch: CTA b runs instance i with
// cta_start[i] <= b < cta_start[i + 1] (each instance has its own chunk
// counter, so its CTAs share its patches dynamically).  The instance's
// arguments are staged in shared memory.
template <int MAXOBS, int LANES>
__global__ void __launch_bounds__(kSweepThreads, (MAXOBS <= 48 && LANES == 1 ? 2 : 1))
    sweep_multi_kernel(const SweepArgs* __restrict__ args, const int* __restrict__ cta_start, int n)
{
    const SweepArgs& a = *stage_instance_args(args, cta_start, n);
    sweep_body<MAXOBS, LANES>(a);
}

// The residual x - D W of every patch on its observed pixels, rebuilt from
// the stored weights with the sweep's own rebuild (the same fused
// multiply-adds in the same atom order, so the bits equal those of a sweep
// that rebuilds it itself), written through the position table into R; the
// FP64 sum of its squares per work unit into part_r2.  Work units in a
// grid-stride loop.
template <int MAXOBS, int LANES>
__global__ void __launch_bounds__(kSweepThreads, (MAXOBS <= 48 && LANES == 1 ? 2 : 1)) rebuild_kernel(const SweepArgs a)
{
    extern __shared__ __align__(16) float smem[];
    const int K = a.g.K, P = a.g.P, KB = a.g.KB;
    const int Kpad = KB * kAtomBlock;
    const int ldK = Kpad + kDictColumnOffset;
    const long long N = a.g.N, Npad = a.g.Npad;
    float* Ds = smem;
    for (int idx = threadIdx.x; idx < (P + 1) * ldK; idx += blockDim.x) {
        const int p = idx / ldK, k = idx - p * ldK - kDictColumnOffset;
        Ds[idx] = (p < P && k >= 0 && k < K) ? a.D[(long long)k * P + p] : 0.0f;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int half = LANES == 1 ? 0 : (lane & 1);
    const unsigned int units = (unsigned int)a.g.NW * LANES;
    const uint32_t col0 = smem_addr(Ds) + 4u * kDictColumnOffset;
    for (unsigned int unit = blockIdx.x * kSweepWarps + warp; unit < units; unit += gridDim.x * kSweepWarps) {
        const long long slot = (long long)unit * PatchLanes<LANES>::kPatchesPerWarp + lane / LANES;
        const long long i = slot_patch(a, slot);
        const bool valid = i < N;
        const int nobs = valid ? (int)a.nobs[slot] : 0;
        const int nl = LANES == 1 ? nobs : (nobs + 1 - half) / 2;
        const int wmax = __reduce_max_sync(0xffffffffu, nl);
        const long long org = valid ? patch_origin(a.g, i) : 0;
        PixelAddr<MAXOBS> ad;
        ad.base = col0;
        ad.pitch = 4u * ldK;
        Resid<MAXOBS> r;
        gather_patch<MAXOBS, LANES>(a, slot, nl, org, ad, r, half, false);
        W8 nb = load_w8(a.W + (long long)i * kAtomBlock);
        for (int kb = 0; kb < KB; ++kb) {
            const W8 wb = nb;
            if (kb + 1 < KB) nb = load_w8(a.W + ((long long)(kb + 1) * Npad + i) * kAtomBlock);
            ad.rebase(col0 + 32u * kb, wmax);
            rebuild_block<MAXOBS>(ad, r, wmax, wb);
        }
        double r2 = 0.0;
#pragma unroll
        for (int g4 = 0; g4 < MAXOBS / 4; ++g4) {
            if (4 * g4 >= wmax) break;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int jj = 4 * g4 + u;
                if (jj < nl) {
                    const float v = r.get(jj);
                    a.R[a.pos[(long long)(jj * LANES + half) * N + slot]] = v;
                    r2 += (double)v * v;
                }
            }
        }
        r2 = warp_sum(r2);
        if (lane == 0) a.part_r2[unit] = r2;
    }
}

int sweep_block_size() { return kSweepThreads; }

int sweep_smem_bytes(const Geom& g)
{
    const int Kpad = g.KB * kAtomBlock;
    const int ldK = Kpad + kDictColumnOffset;
    return (int)(sizeof(float) * ((size_t)(g.P + 1) * ldK + Kpad));
}

// Kernel variants: 0 the sweep, 1 the batched sweep, 2 the residual rebuild.
template <int MAXOBS, int LANES = 1>
static void* kernel_ptr(int kind)
{
    if (kind == 1) return (void*)sweep_multi_kernel<MAXOBS, LANES>;
    if (kind == 2) return (void*)rebuild_kernel<MAXOBS, LANES>;
    return (void*)sweep_kernel<MAXOBS, LANES>;
}

int sweep_lanes(int maxobs) { return maxobs > 96 ? 2 : 1; }

static void* select_kernel(int maxobs, int multi = 0)
{
    if (maxobs > 96) {   // two lanes per patch: per-lane capacity 64 / 96 / 112 / 128
        if (maxobs <= 128) return kernel_ptr<64, 2>(multi);
        if (maxobs <= 192) return kernel_ptr<96, 2>(multi);
        if (maxobs <= 224) return kernel_ptr<112, 2>(multi);
        if (maxobs <= 256) return kernel_ptr<128, 2>(multi);
        return nullptr;
    }
    if (maxobs <= 8) return kernel_ptr<8>(multi);
    if (maxobs <= 12) return kernel_ptr<12>(multi);
    if (maxobs <= 16) return kernel_ptr<16>(multi);
    if (maxobs <= 24) return kernel_ptr<24>(multi);
    if (maxobs <= 32) return kernel_ptr<32>(multi);
    if (maxobs <= 40) return kernel_ptr<40>(multi);
    if (maxobs <= 48) return kernel_ptr<48>(multi);
    if (maxobs <= 64) return kernel_ptr<64>(multi);
    if (maxobs <= 72) return kernel_ptr<72>(multi);
    if (maxobs <= 80) return kernel_ptr<80>(multi);
    return kernel_ptr<96>(multi);
}

// Variant key: equal keys run the same kernel template.
int sweep_variant(int maxobs)
{
    const int caps[] = {8, 12, 16, 24, 32, 40, 48, 64, 72, 80, 96, 128, 192, 224, 256};
    for (int c : caps)
        if (maxobs <= c) return c;
    return 0;
}

cudaError_t launch_sweep_multi(const SweepArgs* args, const int* cta_start, int n, int maxobs, int grid,
                               size_t smem, cudaStream_t s)
{
    void* fn = select_kernel(maxobs, 1);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void* kargs[] = {(void*)&args, (void*)&cta_start, (void*)&n};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kSweepThreads), kargs, smem, s);
}

int sweep_multi_ctas_per_sm(int maxobs, size_t smem)
{
    void* fn = select_kernel(maxobs, 1);
    int per_sm = 0;
    if (!fn || cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kSweepThreads, smem) != cudaSuccess)
        return 0;
    return per_sm;
}

// Loads every variant now: with lazy module loading the first launch of a
// variant would otherwise pay for it (a latency spike when serving).
cudaError_t preload_sweep_variants()
{
    const int obs[] = {8, 12, 16, 24, 32, 40, 48, 64, 72, 80, 96, 128, 192, 224, 256};
    for (int m : obs) {
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, select_kernel(m));
        if (e != cudaSuccess) return e;
        e = cudaFuncGetAttributes(&fa, select_kernel(m, 2));
        if (e != cudaSuccess) return e;
    }
    return preload_tiled_variants();
}

int sweep_grid_size(const Geom& g, int maxobs, int device)
{
    void* fn = select_kernel(maxobs);
    if (!fn) return 0;
    const int smem = sweep_smem_bytes(g);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 0;
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kSweepThreads, smem) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    if (per_sm < 1) return 0;
    long long units = (long long)g.NW * sweep_lanes(maxobs);
    long long warps_per_cta = kSweepThreads / 32;
    long long want = (units + warps_per_cta - 1) / warps_per_cta;
    long long grid = (long long)per_sm * sms;
    return (int)(grid < want ? grid : want);
}

cudaError_t launch_sweep(const SweepArgs& a, int maxobs, int grid, cudaStream_t s)
{
    void* fn = select_kernel(maxobs);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(a.chunk_counter, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    const int smem = sweep_smem_bytes(a.g);
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    void* args[] = {(void*)&a};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kSweepThreads), args, (size_t)smem, s);
}

// The split sweep: units [0, split_units) on s with the kernel for maxobs,
// the rest concurrently on plan.side with the kernel for kSplitObs pixels
// (shorter pixel loops, fewer registers), forked from and joined to s by
// events.  The heavy
// launch goes first so its few CTAs are resident before the light kernel
// fills the GPU.
cudaError_t launch_sweep_split(const SweepArgs& a, const SweepPlan& plan, int maxobs, cudaStream_t s)
{
    SweepArgs heavy = a, light = a;
    heavy.unit_lo = 0;
    heavy.unit_hi = plan.split_units;
    light.unit_lo = plan.split_units;
    light.unit_hi = (unsigned int)a.g.NW;
    light.chunk_counter = plan.counter2;
    cudaError_t e = cudaEventRecord(plan.fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(plan.side, plan.fork, 0);
    if (e == cudaSuccess) e = launch_sweep(heavy, maxobs, plan.split_grid, s);
    if (e == cudaSuccess) e = launch_sweep(light, kSplitObs, plan.light_grid, plan.side);
    if (e == cudaSuccess) e = cudaEventRecord(plan.join, plan.side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, plan.join, 0);
    return e;
}

cudaError_t launch_rebuild(const SweepArgs& a, int maxobs, int grid, cudaStream_t s)
{
    void* fn = select_kernel(maxobs, 2);
    if (!fn || !a.R || !a.part_r2) return cudaErrorInvalidValue;
    const int smem = sweep_smem_bytes(a.g);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    void* args[] = {(void*)&a};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kSweepThreads), args, (size_t)smem, s);
}

}  // namespace sensai
