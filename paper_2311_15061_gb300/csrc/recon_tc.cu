// recon_tc.cu -- the per-patch reconstructions Y = W D on the tensor cores.
//
// The overlap-add estimate of the frame (the paper's reconstruction from the
// learned dictionary and codes, section "BPFA") first needs every patch's
// reconstruction y_i = sum_k z_ik s_ik d_k: a dense N x K by K x P product
// whose left factor is the weight records (0 where z_ik = 0).
//
// A CTA of 128 threads computes tiles of 128 patches with tcgen05.  Per
// 8-atom block: A = the tile's weight records (128 x 8, row r = patch) and
// B = the block's dictionary columns (Np x 8, Np = P rounded up to 16), both
// in shared memory in the canonical no-swizzle K-major layout (core matrices
// of 8 rows x 16 bytes; 128 B between the two core matrices along K, 256 B
// between 8-row groups).  Each factor is split into a TF32 head and an FP32
// tail (x = hi + lo, hi = x with the low 13 mantissa bits cleared); the three
// products hi*hi + hi*lo + lo*hi give FP32-level accuracy (the dropped lo*lo
// is below 2^-20 relative).  The B operands of every block (heads and tails)
// are written once per call by operand_kernel, in that layout.  A ring of
// shared-memory slots holds, per iteration, the tile's 128 raw weight records
// of the block (4 KB, contiguous in the [KB][Npad][8] layout) and the block's
// B operands; thread 0 fills each slot with two bulk copies several
// iterations ahead.  Each iteration, thread r splits its raw record into row
// r of the A heads and tails, and thread 0 issues the MMAs (kind::tf32,
// M = 128, N = Np, K = 8) into a TMEM accumulator of 128 lanes x Np columns,
// commits them to the slot's mbarrier and refills the previous iteration's
// slot once its MMAs have completed.  At the end of a tile the accumulator
// rows are read back with tcgen05.ld (warp w, thread r: patch 32 w + r) and
// stored as coalesced rows of Y [P][N].
//
// Every wait is bounded.  On a timeout the status word gets SENSAI_ETIMEOUT,
// the CTA stops, waits once more (bounded) for its copies and MMAs in flight
// and frees its TMEM.
#include "internal.cuh"

namespace sensai {

constexpr int kRTM = 128;                  // patches per tile (the MMA's M)
constexpr int kRTThreads = 128;            // one thread per tile row
constexpr int kATile = kRTM * kAtomBlock;  // floats of one A operand (128 x 8)
constexpr long long kRTSpins = 1LL << 20;  // try_wait polls before giving up
constexpr int kRTMaxStages = 8;           // deepest copy ring

__device__ __forceinline__ uint32_t rt_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, no swizzle: start address, the byte
// distance between core matrices along K (128) and between 8-row groups
// (256), descriptor version 1.
__device__ __forceinline__ uint64_t rt_desc(const void* p)
{
    uint64_t d = (uint64_t)((rt_smem(p) >> 4) & 0x3FFF);
    d |= (uint64_t)(128u >> 4) << 16;
    d |= (uint64_t)(256u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor: F32 accumulator, TF32 A and B, both K-major, no
// negation, M = 128, N = n.
__device__ __forceinline__ uint32_t rt_idesc(int n)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kRTM >> 4) << 24);
}

// Offset in floats of element (row, k) of an R x 8 operand in that layout.
__device__ __forceinline__ int rt_off(int row, int k)
{
    return (row >> 3) * 64 + (k >> 2) * 32 + (row & 7) * 4 + (k & 3);
}

__device__ __forceinline__ float tf32_head(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// Bounded wait for a phase; the global timer (a slow read) only once the
// first try has failed.
__device__ __forceinline__ bool rt_wait(uint64_t* bar, uint32_t parity)
{
    unsigned long long t0 = 0;
    for (long long spins = 0; spins < kRTSpins; ++spins) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(rt_smem(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (spins == 0) t0 = global_ns();
        else if ((spins & 63) == 0 && global_ns() - t0 > kWaitLimitNs) break;
    }
    return false;
}

__device__ __forceinline__ void rt_mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}


__device__ __forceinline__ void rt_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(rt_smem(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void rt_bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     rt_smem(dst)),
                 "l"(src), "r"(bytes), "r"(rt_smem(bar))
                 : "memory");
}

// The CTA's next (tile, block) in its sequence: blocks of a tile in order,
// tiles strided by the grid.
__device__ __forceinline__ void rt_advance(long long* tile, int* kb, int KB)
{
    if (++*kb == KB) {
        *kb = 0;
        *tile += gridDim.x;
    }
}

// Latest iteration <= last that used ring slot s of `stages` (negative if none).
__device__ __forceinline__ long long rt_latest(long long last, int s, int stages)
{
    if (last < 0) return -1;
    return last - (((last - s) % stages) + stages) % stages;
}

// B operands of every 8-atom block: Dc [KB][head, tail][Np x 8] floats in the
// canonical layout, zero past P and past K.
__global__ void operand_kernel(Geom g, const float* D, float* Dc, int np)
{
    const int bsz = np * kAtomBlock;
    const long long total = (long long)g.KB * bsz;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int kb = (int)(idx / bsz), e = (int)(idx - (long long)kb * bsz);
        const int k = e / np, p = e - k * np;   // consecutive threads: consecutive pixels
        const int ka = kb * kAtomBlock + k;
        const float x = (p < g.P && ka < g.K) ? D[(long long)ka * g.P + p] : 0.0f;
        const float xh = tf32_head(x);
        float* dst = Dc + (long long)kb * 2 * bsz;
        dst[rt_off(p, k)] = xh;
        dst[bsz + rt_off(p, k)] = x - xh;
    }
}

// Dynamic shared memory: A [2 buffers][head, tail][128 x 8] floats, then a
// ring of `stages` slots, each [raw records 128 x 8][B head, tail: Np x 8]
// floats, filled by bulk copies.  Iteration u of the CTA's sequence (tile,
// block) writes A buffer u & 1 and reads ring slot u % stages; its copies and
// its MMAs complete phase u / stages of that slot's two mbarriers.  The copies
// of iteration u are issued stages - 1 iterations ahead.
__global__ void __launch_bounds__(kRTThreads) recon_tc_kernel(Geom g, const float* Dc, const float* W, float* Y,
                                                              int np, int tmem_cols, int stages, int* status)
{
    extern __shared__ __align__(128) float rsm[];
    __shared__ __align__(8) uint64_t copy_bar[kRTMaxStages];
    __shared__ __align__(8) uint64_t mma_bar[kRTMaxStages];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_s, copy_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int P = g.P, KB = g.KB;
    const long long N = g.N, Npad = g.Npad;
    const int bsz = np * kAtomBlock;
    const int slot_floats = kATile + 2 * bsz;
    const uint32_t bbytes = (uint32_t)(2 * bsz * sizeof(float));
    float* As = rsm;
    float* Ring = rsm + 4 * kATile;
    const long long tiles = (Npad + kRTM - 1) / kRTM;
    const long long my_tiles = (long long)blockIdx.x < tiles ? (tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const long long n_u = my_tiles * KB;

    if (tid == 0) {
        abort_s = 0;
        copy_fail = 0;
        for (int s = 0; s < stages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(rt_smem(&copy_bar[s])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(rt_smem(&mma_bar[s])) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(rt_smem(&tmem_slot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = rt_idesc(np);

    // Thread 0: the copies of iteration v, the tile's raw records of block kb
    // (only the rows below Npad) and the block's dictionary operands.
    long long last_copy = -1, last_mma = -1;
    auto issue = [&](long long v) {
        const long long tile = blockIdx.x + (v / KB) * (long long)gridDim.x;
        const int kb = (int)(v % KB);
        const long long i0 = tile * kRTM;
        const long long rows = Npad - i0 < kRTM ? Npad - i0 : kRTM;   // a multiple of 32
        const uint32_t wbytes = (uint32_t)(rows * kAtomBlock * sizeof(float));
        const int s = (int)(v % stages);
        float* slot = Ring + (long long)s * slot_floats;
        rt_expect_tx(&copy_bar[s], wbytes + bbytes);
        rt_bulk_g2s(slot, W + wblock(g, kb, i0), wbytes, &copy_bar[s]);
        rt_bulk_g2s(slot + kATile, Dc + (long long)kb * 2 * bsz, bbytes, &copy_bar[s]);
        last_copy = v;
    };
    if (tid == 0)
        for (long long v = 0; v < stages - 1 && v < n_u; ++v) issue(v);

    long long ct = blockIdx.x;
    int ckb = 0;
    for (long long u = 0; u < n_u; ++u) {
        const int a = (int)(u & 1);
        const int s = (int)(u % stages);
        const uint32_t par = (uint32_t)((u / stages) & 1);
        const float* slot = Ring + (long long)s * slot_floats;
        __syncthreads();   // A[a] is free: thread 0 saw the MMAs of u - 2 complete
        if (abort_s) break;
        if (!rt_wait(&copy_bar[s], par)) {   // every thread reads the slot
            atomicExch(status, (int)SENSAI_ETIMEOUT);
            copy_fail = 1;
        }
        // row tid: its record, split into head and tail
        const bool live = ct * kRTM + tid < Npad;
        float* ah = As + (a * 2 + 0) * kATile;
        float* al = As + (a * 2 + 1) * kATile;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float4 x = live ? reinterpret_cast<const float4*>(slot)[tid * 2 + h] : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 vh, vl;
            vh.x = tf32_head(x.x);
            vh.y = tf32_head(x.y);
            vh.z = tf32_head(x.z);
            vh.w = tf32_head(x.w);
            vl.x = x.x - vh.x;
            vl.y = x.y - vh.y;
            vl.z = x.z - vh.z;
            vl.w = x.w - vh.w;
            *reinterpret_cast<float4*>(ah + rt_off(tid, 4 * h)) = vh;
            *reinterpret_cast<float4*>(al + rt_off(tid, 4 * h)) = vl;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (copy_fail) break;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const float* bh = slot + kATile;
            const float* bl = bh + bsz;
            rt_mma(tmem, rt_desc(ah), rt_desc(bh), idesc, ckb > 0 ? 1u : 0u);
            rt_mma(tmem, rt_desc(ah), rt_desc(bl), idesc, 1u);
            rt_mma(tmem, rt_desc(al), rt_desc(bh), idesc, 1u);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             rt_smem(&mma_bar[s]))
                         : "memory");
            last_mma = u;
            // the MMAs of u - 1 are complete: their A buffer and ring slot are free
            if (u >= 1 && !rt_wait(&mma_bar[(u - 1) % stages], (uint32_t)(((u - 1) / stages) & 1))) {
                atomicExch(status, (int)SENSAI_ETIMEOUT);
                abort_s = 1;
            } else if (u + stages - 1 < n_u) {
                issue(u + stages - 1);   // into the slot of u - 1
            }
        }
        if (ckb == KB - 1) {
            // the tile's accumulation is complete before it is read
            if (tid == 0 && !abort_s && !rt_wait(&mma_bar[s], par)) {
                atomicExch(status, (int)SENSAI_ETIMEOUT);
                abort_s = 1;
            }
            __syncthreads();
            if (abort_s) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const long long i = ct * kRTM + warp * 32 + lane;
            for (int c0 = 0; c0 < np; c0 += 16) {
                uint32_t v[16];
                const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                      "=r"(v[14]), "=r"(v[15])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (i < N) {
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        if (c0 + q < P) Y[(long long)(c0 + q) * N + i] = __uint_as_float(v[q]);
                }
            }
            // the next tile's first MMA (after the next barrier) overwrites the accumulator
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        }
        rt_advance(&ct, &ckb, KB);
    }
    // Every copy and MMA has landed before the TMEM is freed: no-ops after a
    // normal finish, the second bounded wait after a timeout.
    if (tid == 0) {
        for (int s = 0; s < stages; ++s) {
            const long long vc = rt_latest(last_copy, s, stages), vm = rt_latest(last_mma, s, stages);
            if (vc >= 0) (void)rt_wait(&copy_bar[s], (uint32_t)((vc / stages) & 1));
            if (vm >= 0) (void)rt_wait(&mma_bar[s], (uint32_t)((vm / stages) & 1));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

// Np and the TMEM columns for P; false if the tensor-core form does not
// apply (P > 256: the MMA's N is at most 256).
static bool recon_tc_shape(const Geom& g, int* np, int* cols)
{
    if (g.P < 1 || g.P > 256 || g.K < 1) return false;
    *np = (g.P + 15) & ~15;
    *cols = *np <= 32 ? 32 : *np <= 64 ? 64 : *np <= 128 ? 128 : 256;
    return true;
}

bool recon_tc_available(const Geom& g)
{
    int np, cols;
    return recon_tc_shape(g, &np, &cols);
}

size_t recon_tc_operand_floats(const Geom& g)
{
    int np = 0, cols = 0;
    if (!recon_tc_shape(g, &np, &cols)) return 0;
    return (size_t)g.KB * 2 * (size_t)np * kAtomBlock;
}

cudaError_t launch_recon_tc(const Geom& g, const float* D, float* Dc, const float* W, float* Y, int* status,
                            cudaStream_t s)
{
    int np = 0, cols = 0;
    if (!recon_tc_shape(g, &np, &cols) || !Dc) return cudaErrorInvalidValue;
    int dev = 0, sms = 0, smem_sm = 0, reserved = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (e != cudaSuccess) return e;
    // Every resident CTA holds `cols` of the SM's 512 TMEM columns.  The ring
    // is as deep as lets 512 / cols CTAs share an SM (2 to 8 slots), and the
    // shared-memory request is padded so that no more fit: no TMEM allocation
    // of the launch waits on another.
    const int max_ctas = 512 / cols;
    const long long a_bytes = 4LL * kATile * (long long)sizeof(float);
    const long long slot_bytes = (long long)sizeof(float) * (kATile + 2LL * np * kAtomBlock);
    const long long budget = (long long)smem_sm / max_ctas - reserved - 256;
    long long stages = (budget - a_bytes) / slot_bytes;
    if (stages < 2) stages = 2;
    if (stages > kRTMaxStages) stages = kRTMaxStages;
    const long long need = a_bytes + stages * slot_bytes;
    const long long floor_bytes = (long long)smem_sm / (max_ctas + 1) + 1;
    const long long smem = need > floor_bytes ? need : floor_bytes;
    e = cudaFuncSetAttribute((void*)recon_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)   // the whole unified L1 / shared array as shared memory
        e = cudaFuncSetAttribute((void*)recon_tc_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    cudaFuncAttributes fa;
    int threads_sm = 0, blocks_sm = 0;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, (const void*)recon_tc_kernel);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&threads_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&blocks_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev);
    if (e != cudaSuccess) return e;
    // Resident CTAs per SM from shared memory, registers and threads (the
    // occupancy calculator assumes one CTA per SM for a kernel that allocates
    // tensor memory).  Shared memory alone keeps it at most max_ctas.
    const long long per_cta = smem + (long long)fa.sharedSizeBytes + reserved;
    long long per_sm = (long long)smem_sm / per_cta;
    const long long by_regs = 65536 / ((long long)(fa.numRegs > 0 ? fa.numRegs : 1) * kRTThreads);
    if (by_regs < per_sm) per_sm = by_regs;
    if (threads_sm / kRTThreads < per_sm) per_sm = threads_sm / kRTThreads;
    if (blocks_sm < per_sm) per_sm = blocks_sm;
    if (per_sm < 1 || ((long long)smem_sm / per_cta) * cols > 512) return cudaErrorInvalidConfiguration;
    const long long total = (long long)g.KB * np * kAtomBlock;
    operand_kernel<<<(unsigned int)((total + 255) / 256), 256, 0, s>>>(g, D, Dc, np);
    const long long tiles = (g.Npad + kRTM - 1) / kRTM;
    long long grid = (long long)per_sm * sms;
    if (grid > tiles) grid = tiles;
    recon_tc_kernel<<<(unsigned int)grid, kRTThreads, (size_t)smem, s>>>(g, Dc, W, Y, np, cols, (int)stages, status);
    return cudaGetLastError();
}

}  // namespace sensai
