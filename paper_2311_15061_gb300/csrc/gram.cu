// gram.cu -- the dictionary step in its dense-statistics form, with the
// statistics contracted on the tensor cores (the dictionary-learning step of
// the BPFA section).
//
// Neither dictionary sum couples different within-patch pixels p, and the
// atom-ordered conditional of d_kp given every other atom needs, for pixel
// p, only
//   C_p = sum_{i observes p} w_i w_i^T   (the K x K Gram of the weights),
//   Y_p = sum_{i observes p} w_i x_ip    (K correlations with the frame)
// and the current column d_p.  With u = C_p d_p kept current,
//   A_kp = Y_kp - u_k + C_p[k,k] d_kp,  Lambda_kp = P + gamma_eps C_p[k,k],
//   d_kp = gamma_eps A_kp / Lambda_kp + xi_kp / sqrt(Lambda_kp),
// then u += C_p[:,k] (d_new - d_old): atom by atom in order, the same
// conditional as the residual form (tests/test_oracle_dense_statistics.py
// pins the equality), with no pass over the residual at all.
//
// gram_kernel -- the statistics.  Work items are (pixel p, a segment of the
// patches observing p), segment-major so that concurrent items read weight
// records of neighbouring patches (L2 reuse).  An item is cut into chunks of
// 32 patches.  With w = h + l split into a TF32 head h (the top 19 bits, what
// the tensor core reads) and an FP32 tail l, per 8 patches of a chunk two
// tcgen05.mma kind::tf32 (M = N = 128 atoms, K = 8 patches; A in tensor
// memory, B = H K-major in shared memory) accumulate
//   T' += H H^T + (2L) H^T,
// i.e. one product with the K dimension doubled, [H | 2L] [H | H]^T, into a
// 128-column tensor-memory accumulator.  Since H H^T is symmetric,
// C = (T' + T'^T) / 2 = H H^T + L H^T + H L^T: the h h + l h + h l products,
// the dropped l l below 2^-20 relative (FP32-level).  With
// SENSAI_FLAG_TF32_STATISTICS only H H^T is formed (TF32-level).
// The tensor core's FP32 accumulation rounds toward minus infinity (each
// step aligns the addends to the largest with one guard bit and floors; an
// in-bounds probe on this GPU showed it), a bias that grows with the steps
// accumulated.  So the accumulator is drained every 4 chunks (16 steps of 8
// patches) into running sums added in FP32 round-to-nearest: a simulation of
// that arithmetic on the 128x128 K = 64 workload gives <= 2e-6 relative on
// the drawn atoms.
// Warp roles (448 threads, one CTA per SM):
//  * warp 13, loader: per chunk, the 32 patch indices and frame values
//    (loaded a chunk ahead) into one slot of an 8-slot shared ring;
//  * warps 0-7, converters: every chunk, warp w the 32 atoms of TMEM lane
//    quarter w % 4 and the patches 16 (w / 4) .. + 15: lane l (atom
//    32 (w % 4) + l) loads its weight of each patch straight from W, a chunk
//    ahead of use (8 lanes read one 32-byte record block: 4 full sectors
//    per warp instruction), splits it into h and l, writes its row of
//    A = [H | 2L] into tensor memory (tcgen05.st) and its row of B = H into
//    one of two shared-memory stages (K-major, no swizzle; an 8-row group
//    pitch of 272 bytes), and accumulates Y_p for its atom in FP32;
//  * warp 12, lane 0: issues the MMAs (a wait per chunk, 8 MMAs with A in
//    tensor memory, a commit) into two accumulators in turn, one per group
//    of 4 chunks;
//  * warps 8-11, epilogue: warp w reads TMEM lanes 32 (w % 4) .., i.e. the
//    rows of 32 atoms, adds each group's accumulator into running sums kept
//    in tensor memory and frees it; at the end of an item it writes T'^T
//    (coalesced) as the item's FP32 partial.
// Every wait is bounded; a timeout sets SENSAI_ETIMEOUT in the status word,
// every role stops (each warp's decision is its lane 0's, broadcast), the
// MMAs in flight are waited for and TMEM is freed.
//
// gram_reduce_kernel -- the compensated sums of every pixel's item partials,
// in item order; gram_draw_kernel -- one CTA per pixel p: symmetrises the
// sum into C_p and makes the K atom-ordered draws in FP64.
#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace sensai {

constexpr int kGAtoms = 128;                    // M = N: atoms, K padded to 128
constexpr int kGStep = 8;                       // patches per MMA (tf32 K)
constexpr int kGChunk = 32;                     // patches per chunk (4 MMA steps)
constexpr int kGConverters = 8;                 // warps 0-7: lane quarter w % 4, patch half w / 4
constexpr int kGHalf = 16;                      // patches per converter warp and chunk
constexpr int kGEpilogue0 = 8;                  // warps 8-11
constexpr int kGMmaWarp = 12;
constexpr int kGLoaderWarp = 13;
constexpr int kGThreads = 32 * (kGLoaderWarp + 1);
constexpr int kGRawSlots = 8;                   // ring of the chunks' patch indices and frame values
constexpr int kGStages = 2;                     // operand stages (A in TMEM, B in shared memory)
constexpr int kGGroup = 4;                      // chunks per accumulator drain
constexpr int kGRingWords = 2 * kGChunk;        // one chunk's patch indices, then its frame values
constexpr int kGSboBytes = 272;                 // 8-row group pitch (256 B of data + 16 B)
constexpr int kGOpFloats = (kGAtoms / 8) * kGSboBytes / 4;   // one 128 x 8 operand: 1088 floats
constexpr int kGStageFloats = (kGChunk / kGStep) * kGOpFloats;   // B = H of a chunk: 4 operands
constexpr int kGTmemCols = 4 * kGAtoms;         // two accumulators, the A stages, the running sums
constexpr int kGACol0 = 2 * kGAtoms;            // stage s's A operands: columns kGACol0 + 64 s ..
constexpr int kGAStageCols = 2 * kGChunk;       // H (32 patch columns), then 2L (32)
constexpr int kGSumCol = kGACol0 + kGStages * kGAStageCols;   // the running sums' 128 columns
static_assert(kGSumCol + kGAtoms <= kGTmemCols, "tensor memory columns");
constexpr long long kGSpins = 1LL << 22;

// Every converter warp takes part in every chunk (its quarter of the atoms),
// so each waits on every phase of every barrier in order.
static_assert(kGConverters == 8 && kGEpilogue0 % 4 == 0, "warp w accesses TMEM lane quarter w % 4");


__device__ __forceinline__ uint32_t gm_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// No-swizzle K-major descriptor (8-row x 16-byte core matrices; 128 B between
// the two core matrices along K, kGSboBytes between 8-row groups), version 1.
__device__ __forceinline__ uint64_t gm_desc(const void* p)
{
    uint64_t d = (uint64_t)((gm_smem(p) >> 4) & 0x3FFF);
    d |= (uint64_t)(128u >> 4) << 16;
    d |= (uint64_t)((uint32_t)kGSboBytes >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// F32 accumulator, TF32 A and B, both K-major, M = N = 128.
__device__ __forceinline__ uint32_t gm_idesc()
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kGAtoms >> 3) << 17) | ((uint32_t)(kGAtoms >> 4) << 24);
}

__device__ __forceinline__ float gm_head(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

__device__ __forceinline__ void gm_bar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(gm_smem(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void gm_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(gm_smem(bar)) : "memory");
}

// Bounded wait for a phase.  Between tries the thread sleeps, the sleep
// doubling from 32 ns up to kGSleepCapNs: a waiting warp then takes almost no
// issue slots from the warps doing the work on its scheduler (a try that
// fails returns at once on this GPU, so an undelayed poll loop issues about
// one instruction per cycle).  Gives up after kWaitLimitNs; the global timer
// is read only every 16 tries.
constexpr unsigned int kGSleepCapNs = 256;

__device__ __forceinline__ bool gm_wait(uint64_t* bar, uint32_t parity)
{
    unsigned long long t0 = 0;
    unsigned int ns = 32;
    for (long long spins = 0; spins < kGSpins; ++spins) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(gm_smem(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (spins == 0) t0 = global_ns();
        else if ((spins & 15) == 0 && global_ns() - t0 > kWaitLimitNs) break;
        __nanosleep(ns);
        ns = ns < kGSleepCapNs ? 2 * ns : kGSleepCapNs;
    }
    return false;
}

__device__ __forceinline__ void gm_mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// D (+)= A B^T with A (M = 128 rows, one per TMEM lane; K = 8 columns) in
// tensor memory and B described in shared memory.
__device__ __forceinline__ void gm_mma_tmem_a(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// 16 consecutive accumulator columns of this warp's 32 lanes.
__device__ __forceinline__ void gm_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ void gm_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(gm_smem(bar))
                 : "memory");
}

// 32 consecutive accumulator columns of this warp's 32 lanes.
__device__ __forceinline__ void gm_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

// Stores 32 consecutive columns of this warp's 32 lanes; tcgen05.wait::st
// (gm_st_wait) orders them before later tensor-memory reads.
__device__ __forceinline__ void gm_st32(uint32_t taddr, const float (&v)[32])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
        "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
        "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
        "r"(__float_as_uint(v[15])), "r"(__float_as_uint(v[16])), "r"(__float_as_uint(v[17])),
        "r"(__float_as_uint(v[18])), "r"(__float_as_uint(v[19])), "r"(__float_as_uint(v[20])),
        "r"(__float_as_uint(v[21])), "r"(__float_as_uint(v[22])), "r"(__float_as_uint(v[23])),
        "r"(__float_as_uint(v[24])), "r"(__float_as_uint(v[25])), "r"(__float_as_uint(v[26])),
        "r"(__float_as_uint(v[27])), "r"(__float_as_uint(v[28])), "r"(__float_as_uint(v[29])),
        "r"(__float_as_uint(v[30])), "r"(__float_as_uint(v[31]))
        : "memory");
}

__device__ __forceinline__ void gm_st16(uint32_t taddr, const float* v)
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
        "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
        "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
        "r"(__float_as_uint(v[15]))
        : "memory");
}

__device__ __forceinline__ void gm_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ int gm_chunks(int cnt) { return (cnt + kGChunk - 1) / kGChunk; }

// The chunks of this CTA's items in order: item it, chunk c of it, and the
// running chunk number u.  Every role walks the same sequence.
struct ChunkWalk {
    long long it;
    int c, nch;
    long long u;
    __device__ void start(const GramArgs& a)
    {
        it = blockIdx.x;
        c = 0;
        u = 0;
        nch = it < a.n_items ? gm_chunks(a.items[it].z) : 0;
    }
    __device__ bool valid(const GramArgs& a) const { return it < a.n_items; }
    __device__ void next(const GramArgs& a)
    {
        ++u;
        if (++c == nch) {
            c = 0;
            it += gridDim.x;
            nch = it < a.n_items ? gm_chunks(a.items[it].z) : 0;
        }
    }
};

// Item it: pixel items[it].x, patches Ilist[items[it].y .. + items[it].z).
__global__ void __launch_bounds__(kGThreads, 1)
    gram_kernel(const __grid_constant__ GramArgs a)
{
    extern __shared__ __align__(1024) float gsm[];
    __shared__ __align__(8) uint64_t full_bar[kGStages];     // stage written (a converter warp)
    __shared__ __align__(8) uint64_t empty_bar[kGStages];    // stage read (the MMA commit)
    __shared__ __align__(8) uint64_t raw_full[kGRawSlots];   // ring slot written (the loader)
    __shared__ __align__(8) uint64_t raw_empty[kGRawSlots];  // ring slot read (every converter warp)
    __shared__ __align__(8) uint64_t accf_bar[2];          // a group's MMAs complete
    __shared__ __align__(8) uint64_t acce_bar[2];          // a group's accumulator drained
    __shared__ __align__(8) uint64_t done_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int K = a.g.K;
    const bool split = !a.tf32;
    // 1024-byte aligned whatever the dynamic segment's base (tensor copies
    // and the MMA operands want aligned shared addresses)
    float* stages = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(gsm) + 1023) & ~(uintptr_t)1023);
    float* ring = stages + kGStages * kGStageFloats;       // [kGRawSlots][kGRingWords]

    if (tid == 0) {
        abort_s = 0;
        for (int s = 0; s < kGStages; ++s) {
            gm_bar_init(&full_bar[s], kGConverters);   // lane 0 of every converter warp
            gm_bar_init(&empty_bar[s], 1);             // the MMA commit
        }
        for (int r = 0; r < kGRawSlots; ++r) {
            gm_bar_init(&raw_full[r], 1);              // the loader
            gm_bar_init(&raw_empty[r], kGConverters);
        }
        for (int b = 0; b < 2; ++b) {
            gm_bar_init(&accf_bar[b], 1);
            gm_bar_init(&acce_bar[b], 4);   // lane 0 of every epilogue warp
        }
        gm_bar_init(&done_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(gm_smem(&tmem_slot)),
                     "r"(kGTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const long long Npad = a.g.Npad;

    // lane 0 of the warp waits; the warp leaves with lane 0's decision
    auto warp_wait = [&](uint64_t* bar, uint32_t parity) {
        int ok = 1;
        if (lane == 0) {
            ok = !abort_s && gm_wait(bar, parity);
            if (!ok && !abort_s) {
                atomicExch(a.status, (int)SENSAI_ETIMEOUT);
                abort_s = 1;
            }
        }
        return __shfl_sync(0xffffffffu, ok, 0) != 0;
    };

    ChunkWalk wk;
    wk.start(a);
    if (warp < kGConverters) {
        // ----------------------------------------------------- converters --
        // warp w, every chunk: lane l holds atom a = 32 (w % 4) + l of the
        // chunk's patches 16 (w / 4) .. + 15, loaded from W one chunk ahead
        // (one 4-byte load per patch: 8 lanes read a 32-byte record block, 4
        // full sectors per instruction); writes its row of the A operands H
        // and 2L into tensor memory (TMEM lane a, one column per patch) and
        // its row of B = H into the chunk's shared-memory stage, and
        // accumulates Y_pa over its patches
        const int q = warp & 3, hf = warp >> 2;
        const int atom = 32 * q + lane;
        const bool live = atom < K;
        const float* wcol = a.W + (long long)(atom >> 3) * Npad * kAtomBlock + (atom & 7);
        // float offset of (row atom, patches 4 c4 .. + 3) in a 128 x 8 operand
        const int b_base = (atom >> 3) * (kGSboBytes / 4) + (atom & 7) * 4;
        const uint32_t tm_lanes = tmem + ((uint32_t)(32 * q) << 16);
        float y = 0.0f;
        bool ok = true;
        float pre[kGHalf];   // the next chunk's weights of this lane's atom
        // issues the loads of chunk c (its ring slot is waited for first)
        auto fetch = [&](const ChunkWalk& c) {
            const int rs = (int)(c.u % kGRawSlots);
            ok = warp_wait(&raw_full[rs], (uint32_t)((c.u / kGRawSlots) & 1));
            if (!ok) return;
            const int* ri = reinterpret_cast<const int*>(ring + rs * kGRingWords) + kGHalf * hf;
            const int nv = min(kGChunk, a.items[c.it].z - c.c * kGChunk) - kGHalf * hf;
#pragma unroll
            for (int j = 0; j < kGHalf; ++j)
                pre[j] = (j < nv && live) ? __ldg(wcol + (long long)ri[j] * kAtomBlock) : 0.0f;
        };
        if (wk.valid(a)) fetch(wk);
        for (; wk.valid(a) && ok; wk.next(a)) {
            const int nvalid = min(kGChunk, a.items[wk.it].z - wk.c * kGChunk) - kGHalf * hf;
            const int rs = (int)(wk.u % kGRawSlots);
            const int st = (int)(wk.u % kGStages);
            float cur[kGHalf];
#pragma unroll
            for (int j = 0; j < kGHalf; ++j) cur[j] = pre[j];
            const float* rx = ring + rs * kGRingWords + kGChunk + kGHalf * hf;
#pragma unroll
            for (int j = 0; j < kGHalf; ++j) y = fmaf(cur[j], j < nvalid ? rx[j] : 0.0f, y);
            __syncwarp();
            if (lane == 0) gm_arrive(&raw_empty[rs]);   // indices and frame values read
            {
                ChunkWalk nx = wk;
                nx.next(a);
                if (nx.valid(a)) fetch(nx);   // in flight during this chunk's conversion
                if (!ok) break;
            }
            if (!(ok = warp_wait(&empty_bar[st], (uint32_t)(((wk.u / kGStages) & 1) ^ 1)))) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t acol = (uint32_t)(kGACol0 + st * kGAStageCols + kGHalf * hf);
            float* stg = stages + (size_t)st * kGStageFloats;
            float h[kGHalf], l2[kGHalf];
#pragma unroll
            for (int j = 0; j < kGHalf; ++j) {
                h[j] = gm_head(cur[j]);
                l2[j] = 2.0f * (cur[j] - h[j]);   // exact: h is w truncated, doubling is exact
            }
            gm_st16(tm_lanes + acol, h);
            if (split) gm_st16(tm_lanes + acol + kGChunk, l2);
#pragma unroll
            for (int c4 = 0; c4 < kGHalf / 4; ++c4) {   // patch quad 4 hf + c4: operand (4 hf + c4) / 2
                const int qd = 4 * hf + c4;
                *reinterpret_cast<float4*>(stg + (qd >> 1) * kGOpFloats + b_base + (qd & 1) * 32) =
                    make_float4(h[4 * c4], h[4 * c4 + 1], h[4 * c4 + 2], h[4 * c4 + 3]);
            }
            gm_st_wait();
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) gm_arrive(&full_bar[st]);
            if (wk.c == wk.nch - 1) {
                // the end of an item: this warp's share of Y_p for its atom
                a.Ypart[((size_t)wk.it * 2 + hf) * kGAtoms + atom] = y;
                y = 0.0f;
            }
        }
    } else if (warp == kGLoaderWarp) {
        // ---------------------------------------------------------- loader --
        // per chunk: the 32 patch indices and frame values (loaded a chunk
        // ahead) into one ring slot
        int idx = 0;
        float xv = 0.0f;
        auto load_lane = [&](const ChunkWalk& c, int& i_out, float& x_out) {
            i_out = 0;
            x_out = 0.0f;
            if (!c.valid(a)) return;
            const int4 item = a.items[c.it];
            const int e = c.c * kGChunk + lane;
            if (e < item.z) {
                i_out = __ldg(a.Ilist + item.y + e);
                x_out = __ldg(a.Xlist + item.y + e);
            }
        };
        ChunkWalk cur = wk;
        load_lane(cur, idx, xv);
        while (cur.valid(a)) {
            ChunkWalk nxt = cur;
            nxt.next(a);
            int idx_n;
            float xv_n;
            load_lane(nxt, idx_n, xv_n);
            const int rs = (int)(cur.u % kGRawSlots);
            if (!warp_wait(&raw_empty[rs], (uint32_t)(((cur.u / kGRawSlots) & 1) ^ 1))) break;
            reinterpret_cast<int*>(ring + rs * kGRingWords)[lane] = idx;
            ring[rs * kGRingWords + kGChunk + lane] = xv;
            __syncwarp();
            if (lane == 0) gm_arrive(&raw_full[rs]);
            cur = nxt;
            idx = idx_n;
            xv = xv_n;
        }
    } else if (warp == kGMmaWarp) {
        // ---------------------------------------------------- MMA issuer --
        if (lane == 0) {
            const uint32_t idesc = gm_idesc();
            long long gc = 0;   // groups (accumulator uses)
            bool ok = true;
            while (wk.valid(a) && ok) {
                const int cnt = a.items[wk.it].z;
                const int c1 = min(wk.c + kGGroup, wk.nch);
                const int buf = (int)(gc & 1);
                if (abort_s || !gm_wait(&acce_bar[buf], (uint32_t)(((gc >> 1) & 1) ^ 1))) {   // drained
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t acc_tmem = tmem + (uint32_t)(buf * kGAtoms);
                uint32_t acc = 0;
                for (int c = wk.c; c < c1; ++c, wk.next(a)) {
                    const int s = (int)(wk.u % kGStages);
                    if (abort_s || !gm_wait(&full_bar[s], (uint32_t)((wk.u / kGStages) & 1))) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const float* stg = stages + (size_t)s * kGStageFloats;
                    const uint32_t acol = tmem + (uint32_t)(kGACol0 + s * kGAStageCols);
                    const int nvalid = min(kGChunk, cnt - c * kGChunk);
                    for (int kb = 0; kb * kGStep < nvalid; ++kb) {
                        const uint64_t bh = gm_desc(stg + kb * kGOpFloats);
                        gm_mma_tmem_a(acc_tmem, acol + (uint32_t)(kb * kGStep), bh, idesc, acc);   // H H^T
                        acc = 1;
                        if (split)   // 2L H^T
                            gm_mma_tmem_a(acc_tmem, acol + (uint32_t)(kGChunk + kb * kGStep), bh, idesc, 1u);
                    }
                    gm_commit(&empty_bar[s]);
                }
                if (!ok) break;
                gm_commit(&accf_bar[buf]);
                ++gc;
            }
            if (!ok && !abort_s) {
                atomicExch(a.status, (int)SENSAI_ETIMEOUT);
                abort_s = 1;
            }
            // every MMA issued has completed before TMEM is freed
            gm_commit(&done_bar);
            if (!gm_wait(&done_bar, 0)) atomicExch(a.status, (int)SENSAI_ETIMEOUT);
        }
    } else if (warp >= kGEpilogue0 && warp < kGEpilogue0 + 4) {
        // ------------------------------------------------------- epilogue --
        const int quarter = warp & 3;              // TMEM lanes 32 quarter ..
        const int row = quarter * 32 + lane;       // atom of the accumulator rows
        const uint32_t lanes = tmem + ((uint32_t)(quarter * 32) << 16);
        long long gc = 0;
        bool ok = true;
        while (wk.valid(a) && ok) {
            float* cpart = a.Cpart + (size_t)wk.it * kGAtoms * kGAtoms;
            bool first = true;
            // the item's groups of kGGroup chunks: the running sums in tensor
            // memory; the last group's total is the item's partial T^T
            while (ok) {
                const int c1 = min(wk.c + kGGroup, wk.nch);
                const bool last = c1 == wk.nch;
                const int buf = (int)(gc & 1);
                ok = warp_wait(&accf_bar[buf], (uint32_t)((gc >> 1) & 1));
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
                for (int cb = 0; cb < kGAtoms / 32; ++cb) {
                    float v[32];
                    gm_ld32(lanes + (uint32_t)(buf * kGAtoms + cb * 32), v);
                    if (!first) {
                        float sm[32];
                        gm_ld32(lanes + (uint32_t)(kGSumCol + cb * 32), sm);
#pragma unroll
                        for (int q = 0; q < 32; ++q) v[q] = sm[q] + v[q];
                    }
                    if (last) {
                        // column `row` of the transposed partial (coalesced)
#pragma unroll
                        for (int q = 0; q < 32; ++q) cpart[(size_t)(cb * 32 + q) * kGAtoms + row] = v[q];
                    } else {
                        gm_st32(lanes + (uint32_t)(kGSumCol + cb * 32), v);
                    }
                }
                if (!last) gm_st_wait();
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) gm_arrive(&acce_bar[buf]);
                ++gc;
                first = false;
                for (int c = wk.c; c < c1; ++c) wk.next(a);
                if (last) break;
            }
        }
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kGTmemCols) : "memory");
}

// Compensated FP32 summation: (s, c) with s + c the running sum; TwoSum
// (Knuth) gives the rounding error of each addition exactly, so the result
// is as accurate as an FP64 sum of these few FP32 terms, at FP32 speed (the
// FP64 units of this GPU are a small fraction of its FP32 rate).
__device__ __forceinline__ void gm_sum2(float& s, float& c, float v)
{
    const float t = s + v;
    const float bp = t - s;
    const float e = (s - (t - bp)) + (v - bp);
    s = t;
    c += e;
}

// S_p = sum of pixel p's item partials T^T and Y_p, in item order, by
// compensated FP32 summation, stored in FP64.  One thread per element,
// every item's load in flight at once.
__global__ void __launch_bounds__(256) gram_reduce_kernel(GramArgs a)
{
    const int p = blockIdx.x;
    const int idx = blockIdx.y * blockDim.x + threadIdx.x;   // r * 128 + t
    const int i0 = a.pitem_start[p], i1 = a.pitem_start[p + 1];
    float s = 0.0f, c = 0.0f;
    int j = i0;
    for (; j + 8 <= i1; j += 8) {
        float v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = a.Cpart[(size_t)a.pitem_idx[j + q] * kGAtoms * kGAtoms + idx];
#pragma unroll
        for (int q = 0; q < 8; ++q) gm_sum2(s, c, v[q]);
    }
    for (; j < i1; ++j) gm_sum2(s, c, a.Cpart[(size_t)a.pitem_idx[j] * kGAtoms * kGAtoms + idx]);
    a.C64[(size_t)p * kGAtoms * kGAtoms + idx] = (double)s + (double)c;
    if (blockIdx.y == 0 && threadIdx.x < kGAtoms) {
        const int t = threadIdx.x;
        float ys = 0.0f, yc = 0.0f;
        for (int jj = i0; jj < i1; ++jj) {
            const size_t it = (size_t)a.pitem_idx[jj];
            gm_sum2(ys, yc, a.Ypart[(it * 2 + 0) * kGAtoms + t]);
            gm_sum2(ys, yc, a.Ypart[(it * 2 + 1) * kGAtoms + t]);
        }
        a.Y64[(size_t)p * kGAtoms + t] = (double)ys + (double)yc;
    }
}

// One CTA per pixel p (128 threads, thread = atom): C_p = (S_p + S_p^T) / 2,
// then the atom-ordered draws in FP64 from C_p, Y_p and the current column.
__global__ void __launch_bounds__(kGAtoms) gram_draw_kernel(GramArgs a)
{
    extern __shared__ __align__(16) double cs[];   // [128][129] C_p
    __shared__ double delta[kGAtoms];
    __shared__ double dcol[kGAtoms];
    const int p = blockIdx.x;
    const int t = threadIdx.x;
    const int K = a.g.K, P = a.g.P;
    const double* cg = a.C64 + (size_t)p * kGAtoms * kGAtoms;
#pragma unroll 16
    for (int r = 0; r < kGAtoms; ++r) cs[r * (kGAtoms + 1) + t] = cg[(size_t)r * kGAtoms + t];
    __syncthreads();
    // thread t symmetrises the pairs (r, t), r < t: each unordered pair once
    for (int r = 0; r < t; ++r) {
        const double v = 0.5 * (cs[r * (kGAtoms + 1) + t] + cs[t * (kGAtoms + 1) + r]);
        cs[r * (kGAtoms + 1) + t] = v;
        cs[t * (kGAtoms + 1) + r] = v;
    }
    const double y = a.Y64[(size_t)p * kGAtoms + t];
    const uint32_t t_it = launch_t(a.t, a.t_dev, a.sc);
    const double ge = a.sc->gamma_eps;
    double d = t < K ? (double)a.D[(long long)t * P + p] : 0.0;
    dcol[t] = d;
    __syncthreads();
    // per atom, independent of the order: gain gamma_eps / Lambda and noise
    // xi / sqrt(Lambda), Lambda = P + gamma_eps C_kk
    const double ckk = cs[t * (kGAtoms + 1) + t];
    const double lam = (double)P + ge * ckk;
    const double gain = ge / lam;
    double noise = 0.0;
    if (t < K) {
        const uint4 blk = philox4x32_10(make_uint4((uint32_t)p, (uint32_t)t, t_it, kTagDict), seed_key(a.seed));
        noise = normal64(blk.x, blk.y) / sqrt(lam);
    }
    // u = C_p d_p
    double u = 0.0;
    for (int b = 0; b < kGAtoms; ++b) u = fma(cs[t * (kGAtoms + 1) + b], dcol[b], u);
    // the draws in atom order: A_k = Y_k - u_k + C_kk d_k excludes atom k
    for (int k = 0; k < K; ++k) {
        if (t == k) {
            const double A = y - u + ckk * d;
            const double dn = fma(gain, A, noise);
            delta[k] = dn - d;
            d = dn;
            a.D[(long long)k * P + p] = (float)dn;
        }
        __syncthreads();
        u = fma(cs[t * (kGAtoms + 1) + k], delta[k], u);
    }
}

// ------------------------------------------------------------ host side --

// The work items: for every pixel p, its patch list cut into segments of at
// most `seg` patches; items ordered segment-major.  pitem: p -> its items.
void gram_plan_items(const std::vector<int>& Rbase, int P, int seg, std::vector<int4>* items,
                     std::vector<int>* pitem_start, std::vector<int>* pitem_idx)
{
    items->clear();
    int max_segs = 0;
    for (int p = 0; p < P; ++p) max_segs = std::max(max_segs, (Rbase[p + 1] - Rbase[p] + seg - 1) / seg);
    std::vector<std::vector<int>> per_p(P);
    for (int s = 0; s < max_segs; ++s)
        for (int p = 0; p < P; ++p) {
            // pixel p's list in nseg near-equal segments of at most seg patches
            const int cnt = Rbase[p + 1] - Rbase[p];
            const int nseg = (cnt + seg - 1) / seg;
            if (s >= nseg) continue;
            const int start = (int)((long long)cnt * s / nseg), end = (int)((long long)cnt * (s + 1) / nseg);
            per_p[p].push_back((int)items->size());
            items->push_back(make_int4(p, Rbase[p] + start, end - start, 0));
        }
    pitem_start->assign(P + 1, 0);
    pitem_idx->clear();
    for (int p = 0; p < P; ++p) {
        (*pitem_start)[p] = (int)pitem_idx->size();
        for (int it : per_p[p]) pitem_idx->push_back(it);
    }
    (*pitem_start)[P] = (int)pitem_idx->size();
}

size_t gram_smem_bytes()
{
    return 1024 + sizeof(float) * ((size_t)kGStages * kGStageFloats + (size_t)kGRawSlots * kGRingWords);
}

// Xlist[e] = x[origin(Ilist[e]) + imgoff[p]] for the entries of pixel p.
__global__ void xlist_kernel(Geom g, const int* Ilist, const int* Rbase, const int* imgoff, const float* x,
                             float* Xlist)
{
    const int p = blockIdx.y;
    const int e = Rbase[p] + blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= Rbase[p + 1]) return;
    Xlist[e] = x[patch_origin(g, Ilist[e]) + imgoff[p]];
}

cudaError_t launch_xlist(const Geom& g, const int* Ilist, const int* Rbase, int max_slots, const int* imgoff,
                         const float* x, float* Xlist, cudaStream_t s)
{
    dim3 grid((unsigned int)((max_slots + 255) / 256 > 0 ? (max_slots + 255) / 256 : 1), (unsigned int)g.P);
    xlist_kernel<<<grid, 256, 0, s>>>(g, Ilist, Rbase, imgoff, x, Xlist);
    return cudaGetLastError();
}

cudaError_t launch_gram(const GramArgs& a, int grid, cudaStream_t s)
{
    const size_t smem = gram_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute((void*)gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    gram_kernel<<<grid, kGThreads, smem, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    gram_reduce_kernel<<<dim3((unsigned int)a.g.P, kGAtoms * kGAtoms / 256), 256, 0, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t dsmem = sizeof(double) * (size_t)kGAtoms * (kGAtoms + 1);
    e = cudaFuncSetAttribute((void*)gram_draw_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsmem);
    if (e != cudaSuccess) return e;
    gram_draw_kernel<<<a.g.P, kGAtoms, dsmem, s>>>(a);
    return cudaGetLastError();
}

bool gram_available(const Geom& g) { return g.K >= 1 && g.K <= kGAtoms; }

}  // namespace sensai
