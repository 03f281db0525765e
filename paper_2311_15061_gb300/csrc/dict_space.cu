// dict_space.cu -- the dictionary sweep organised by space.
//
// Same draws as dict.cu: the atom-ordered conjugate Gaussian of every d_kp, in
// 8-atom blocks with the in-block Gram correction.  The work is split over
// the frame instead of over pixel chains.  A pair (u, q) -- an observed
// frame pixel u and a within-patch pixel q such that u - q is a patch origin
// -- is one residual slot of chain q.
//
// Layout (planned once per context, on the host and by the two planning
// kernels below):
//  * the observed pixels are split into one spatial box per CTA, balanced by
//    count (recursive bisection).  Inside a box they are ordered tile by tile
//    (tiles of min(B_d, 8) pixels per dimension), raster order within a tile;
//  * a thread owns one chain q and every G-th pixel of its CTA's list
//    (G = 512 / P groups), so at any moment the CTA works on a few
//    neighbouring pixels, whose covering patches are neighbours in the
//    patch grid;
//  * the patches holding any pixel of a box form its neighbourhood, a box
//    of the patch grid.  When two neighbourhood-sized buffers fit in shared
//    memory for every CTA, the kernel is staged: each 8-atom block's 32-byte
//    weight records of the neighbourhood are copied into shared memory (the
//    record halves in separate arrays, so a warp reading neighbouring
//    records reads consecutive words), and a pair's index is its position
//    in the neighbourhood.  Otherwise the records are read through L1;
//  * pair jp of thread t in CTA c is element base_c + jp * 512 + t of the
//    residual array R and of the patch-index array pidx.  Threads of a warp
//    therefore touch consecutive words; the sweep writes its residuals
//    straight into this layout through a (pixel, patch) -> pair table.
//
// Per 8-atom block: (1) every thread applies the previous block's update to
// its residual pairs (shared memory when they fit, else global memory) and
// accumulates G_k = sum w_k r and the in-block Gram C_kl over them; (2) the
// CTA sums its threads per chain in a fixed order and publishes the partial;
// (3) grid barrier; (4) CTA c sums the partials (stored chain-major, so one
// owner reads one contiguous block) of chains c, c + grid, ...
// over all CTAs in a fixed order (compensated FP32: FP64 arithmetic runs at a
// small fraction of the FP32 rate on this part) and draws the block's 8 atoms
// at those pixels; (5) grid barrier; (6) every thread reads its chain's 8
// updates.
// One cooperative launch, one CTA per SM; the barrier spins are bounded and
// report SENSAI_ETIMEOUT through the status word instead of hanging.
#include "internal.cuh"

#include <algorithm>
#include <vector>

namespace sensai {

constexpr int kDSThreads = 512;
constexpr int kDSGram = kAtomBlock * (kAtomBlock + 1) / 2;   // 36
constexpr int kDSRed = kAtomBlock + kDSGram;                  // 44
constexpr int kDSRedPad = kDSRed + 1;                          // smem row pitch (odd)
constexpr long long kBarrierSpins = 1LL << 24;               // x ~64 ns sleep: ~1 s

// Grid barrier on a monotonic arrival counter (zeroed by the host before
// every launch): barrier number n of the launch waits until the counter reaches
// (n + 1) * nblocks.  Thread 0 arrives with a release reduction (no round
// trip) after the block barrier, so the CTA's earlier writes are published
// (release is cumulative over what the block barrier ordered before it), and
// polls with acquire loads.  Returns false (and sets *status) if it does not
// complete within the spin and time limits.
// The two halves, for a CTA that works between its arrival and its wait:
// grid_arrive by one thread after a block barrier, grid_wait by the same
// thread (1 = complete, 0 = gave up and set *status).
__device__ __forceinline__ void grid_arrive(unsigned int* count)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
}

__device__ int grid_wait(unsigned int* count, unsigned int target, int* status)
{
    unsigned long long t0 = 0;   // the global timer (a slow read) once a poll has failed
    long long spins = 0;
    for (;;) {
        unsigned int v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
        if (v >= target) return 1;
        if (spins == 0) t0 = global_ns();
        if (++spins > kBarrierSpins || ((spins & 255) == 0 && global_ns() - t0 > kWaitLimitNs)) {
            atomicExch(status, (int)SENSAI_ETIMEOUT);
            return 0;
        }
        __nanosleep(32);
    }
}

__device__ bool grid_barrier(unsigned int* count, unsigned int target, int* status)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        grid_arrive(count);
        ok_s = grid_wait(count, target, status);
    }
    __syncthreads();
    return ok_s != 0;
}

// Self-test of the bounded grid barrier: one CTA waits for an arrival count
// that nothing reaches (target = 2 with one CTA) and must give up with
// SENSAI_ETIMEOUT in *status.
__global__ void barrier_timeout_selftest_kernel(unsigned int* count, int* status)
{
    grid_barrier(count, 2u, status);
}

cudaError_t launch_barrier_timeout_selftest(unsigned int* count, int* status, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    barrier_timeout_selftest_kernel<<<1, 64, 0, s>>>(count, status);
    return cudaGetLastError();
}

// Within-patch multi-index of chain q.
__device__ __forceinline__ void chain_index(const Geom& g, int q, int* qd)
{
    for (int d = g.ndim - 1; d >= 0; --d) {
        qd[d] = q % g.B[d];
        q /= g.B[d];
    }
}

// Patch whose pixel qd is frame pixel u, or -1.
__device__ __forceinline__ long long pair_patch(const Geom& g, long long u, const int* qd)
{
    int cd[kMaxDim];
    for (int d = g.ndim - 1; d >= 0; --d) {
        cd[d] = (int)(u % g.M[d]);
        u /= g.M[d];
    }
    long long i = 0;
    for (int d = 0; d < g.ndim; ++d) {
        int av = cd[d] - qd[d];
        if (av < 0) return -1;
        if (g.S[d] != 1) {
            if (av % g.S[d]) return -1;
            av /= g.S[d];
        }
        if (av >= g.G[d]) return -1;
        i = i * g.G[d] + av;
    }
    return i;
}

// Planning pass 1: pairs per thread and the largest count per CTA.
__global__ void __launch_bounds__(kDSThreads) ds_count_kernel(Geom g, const int* order, const int* start, int* np,
                                                              int* npmax)
{
    __shared__ int wmax[kDSThreads / 32];
    const int c = blockIdx.x, t = threadIdx.x;
    const int G = kDSThreads / g.P;
    const bool active = t < G * g.P;
    int n = 0;
    if (active) {
        const int grp = t / g.P, q = t % g.P;
        int qd[kMaxDim];
        chain_index(g, q, qd);
        const int lo = start[c], L = start[c + 1] - lo;
        for (int j = grp; j < L; j += G)
            if (pair_patch(g, order[lo + j], qd) >= 0) ++n;
    }
    np[(size_t)c * kDSThreads + t] = n;
    const int m = __reduce_max_sync(0xffffffffu, n);
    if ((t & 31) == 0) wmax[t >> 5] = m;
    __syncthreads();
    if (t == 0) {
        int mx = 0;
        for (int w = 0; w < kDSThreads / 32; ++w) mx = max(mx, wmax[w]);
        npmax[c] = mx;
    }
}

// Position of patch i inside CTA c's staged neighbourhood nb[c] = {origin
// a0[kMaxDim], extents E[kMaxDim]} of the patch grid (row-major).
__device__ __forceinline__ int local_record(const Geom& g, long long i, const int* nb)
{
    int l = 0, mul = 1;
    for (int d = g.ndim - 1; d >= 0; --d) {
        const int a = (int)(i % g.G[d]);
        i /= g.G[d];
        l += (a - nb[d]) * mul;
        mul *= nb[kMaxDim + d];
    }
    return l;
}

// Planning pass 2: the patch of every pair (its neighbourhood position when
// the weights are staged) and, for the sweep, the pair of every (observed
// pixel j, patch i): pos[j][i].
__global__ void __launch_bounds__(kDSThreads) ds_fill_kernel(Geom g, const int* order, const int* start,
                                                             const long long* base, const uint16_t* obs,
                                                             const uint16_t* nobs, const int* nb, int* pidx,
                                                             int* pos)
{
    const int c = blockIdx.x, t = threadIdx.x;
    const int G = kDSThreads / g.P;
    if (t >= G * g.P) return;
    const int grp = t / g.P, q = t % g.P;
    int qd[kMaxDim];
    chain_index(g, q, qd);
    const int lo = start[c], L = start[c + 1] - lo;
    long long idx = base[c] + t;
    for (int j = grp; j < L; j += G) {
        const long long i = pair_patch(g, order[lo + j], qd);
        if (i < 0) continue;
        pidx[idx] = nb ? local_record(g, i, nb + (size_t)c * 2 * kMaxDim) : (int)i;
        const int no = nobs[i];
        for (int jj = 0; jj < no; ++jj)
            if (obs[(long long)jj * g.N + i] == q) {
                pos[(long long)jj * g.N + i] = (int)idx;
                break;
            }
        idx += kDSThreads;
    }
}

// s + e += x by Knuth's TwoSum: s takes the rounded sum, e collects its exact
// rounding error.
__device__ __forceinline__ void two_sum_acc(float& s, float& e, float x)
{
    const float t = s + x;
    const float bp = t - s;
    e += (s - (t - bp)) + (x - bp);
    s = t;
}

// One 8-atom block's weight records for this CTA's patch neighbourhood, by
// cp.async copies of 16 bytes: the first half of every record (atoms 0-3 of
// the block) to buf[0, half), the second half to buf[half, 2 half), both in
// neighbourhood order, so that a warp reading a run of neighbouring records
// reads consecutive shared-memory words.  Consecutive threads copy
// consecutive 16-byte pieces of a neighbourhood row.
__device__ __forceinline__ void ds_stage(float* buf, int half, const float* Wblk, const int* rowbase, int nrec,
                                         int elast)
{
    const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(buf);
    for (int c = threadIdx.x; c < 2 * nrec; c += kDSThreads) {
        const int rec = c >> 1, h = c & 1;
        const int r = rec / elast;
        const float* src = Wblk + ((long long)rowbase[r] + (rec - r * elast)) * kAtomBlock + h * 4;
        const uint32_t dst = s0 + (uint32_t)(((size_t)h * half + (size_t)rec * 4) * sizeof(float));
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// Waits for this thread's staging copies (plain loads: they always complete).
__device__ __forceinline__ void ds_stage_wait()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// Record l of a staged block.
__device__ __forceinline__ W8 lds_w8_split(const float* buf, int half, int l)
{
    const float4 lo = *reinterpret_cast<const float4*>(buf + (size_t)l * 4);
    const float4 hi = *reinterpret_cast<const float4*>(buf + half + (size_t)l * 4);
    W8 w;
    w.v[0] = lo.x;
    w.v[1] = lo.y;
    w.v[2] = lo.z;
    w.v[3] = lo.w;
    w.v[4] = hi.x;
    w.v[5] = hi.y;
    w.v[6] = hi.z;
    w.v[7] = hi.w;
    return w;
}

// RHO_SMEM: the residual pairs live in shared memory during the launch.
// STAGED: each block's weight records for the CTA's neighbourhood are copied
// to shared memory (two buffers: block b in buffer b & 1, the next block
// copied while the CTAs reduce and draw the current one) instead of being
// read through L1 from global memory.
// Dynamic shared memory: [buffer 0][buffer 1][red, unless it shares the
// buffer of the previous block][rowbase][xis][rho_s].
template <bool RHO_SMEM, bool STAGED>
__global__ void __launch_bounds__(kDSThreads, 1) dict_space_kernel(const DictSpaceArgs a)
{
    extern __shared__ __align__(16) float dyn[];
    __shared__ float dold8[kAtomBlock];
    __shared__ float gain8[kAtomBlock], noise8[kAtomBlock];
    __shared__ float fin[kDSRed];
    __shared__ float tmp_s[kDSRed][11], tmp_e[kDSRed][11];
    __shared__ float r2_s[kDSThreads / 32];
    const Geom& g = a.g;
    const int P = g.P, K = g.K, KB = g.KB;
    const long long Npad = g.Npad;
    const int c = blockIdx.x, ncta = gridDim.x;
    const int G = kDSThreads / P;                    // groups of P threads
    const int t = threadIdx.x;
    const bool active = t < G * P;
    const int grp = active ? t / P : 0, q = active ? t % P : 0;
    const int lane = t & 31, warp = t >> 5;
    constexpr int T = kDSThreads;

    float* bufs = dyn;                                               // 2 x buf_floats (staged)
    float* red_sep = dyn + 2 * (size_t)a.buf_floats;                 // [G-1][P][kDSRedPad] or empty
    int* rowbase = reinterpret_cast<int*>(red_sep + a.red_sep_floats);   // [rows_max] (staged)
    float* xis = reinterpret_cast<float*>(rowbase + a.rows_max);     // [own_max][K] normals of owned chains
    float* rho_s = xis + (size_t)a.own_max * K;                      // [max_np][T] staged residual pairs
    const long long base = a.base[c];
    const int np = a.np[(size_t)c * T + t];                         // 0 for idle threads
    const int* pid = a.pidx + base + t;                             // pair jp: pid[jp * T]
    float* rho = RHO_SMEM ? rho_s + t : a.R + base + t;            // pair jp: rho[jp * T]

    // the neighbourhood of the CTA's box in the patch grid: nrec records in
    // rows of elast; rowbase[r] = global index of row r's first record
    int nrec = 0, elast = 1;
    if (STAGED) {
        const int* nbc = a.nb + (size_t)c * 2 * kMaxDim;
        nrec = 1;
        for (int d = 0; d < g.ndim; ++d) nrec *= nbc[kMaxDim + d];
        elast = max(1, nbc[kMaxDim + g.ndim - 1]);
        const int rows = nrec / elast;
        for (int r = t; r < rows; r += T) {
            long long i = nbc[g.ndim - 1], mul = g.G[g.ndim - 1];
            int rr = r;
            for (int d = g.ndim - 2; d >= 0; --d) {
                const int e = nbc[kMaxDim + d];
                i += (long long)(nbc[d] + rr % e) * mul;
                rr /= e;
                mul *= g.G[d];
            }
            rowbase[r] = (int)i;
        }
        __syncthreads();
        if (KB > 0) ds_stage(bufs, a.half_floats, a.W, rowbase, nrec, elast);
    }
    if (RHO_SMEM)
        for (int jp = 0; jp < np; ++jp) rho[(size_t)jp * T] = a.R[base + t + (long long)jp * T];
    for (int idx = t; idx < a.own_max * K; idx += blockDim.x) {
        const int o = idx / K, k = idx % K;
        const int ch = c + o * ncta;
        if (ch < P) {
            const uint4 blk = philox4x32_10(make_uint4((uint32_t)ch, (uint32_t)k, a.t, kTagDict), seed_key(a.seed));
            xis[idx] = (float)normal64(blk.x, blk.y);
        }
    }
    __syncthreads();

    const double ge = a.sc->gamma_eps;
    const float gef = (float)ge;
    float dq[kAtomBlock];
#pragma unroll
    for (int k = 0; k < kAtomBlock; ++k) dq[k] = 0.0f;

    // staged: the record index and residual of a pair are loaded four pairs
    // ahead; the first four of a pass are loaded before the barriers that
    // precede it
    int hp0 = 0, hp1 = 0, hp2 = 0, hp3 = 0;
    float hr0 = 0.0f, hr1 = 0.0f, hr2 = 0.0f, hr3 = 0.0f;
#define DS_HEAD(J_, PX, RX)                                                \
    do {                                                                   \
        if ((J_) < np) {                                                   \
            PX = pid[(size_t)(J_) * T];                                    \
            RX = rho[(size_t)(J_) * T];                                    \
        }                                                                  \
    } while (0)
    if (STAGED) {
        DS_HEAD(0, hp0, hr0);
        DS_HEAD(1, hp1, hr1);
        DS_HEAD(2, hp2, hr2);
        DS_HEAD(3, hp3, hr3);
    }

    for (int kb = 0; kb <= KB; ++kb) {
        if (STAGED) {   // block kb has landed in buffer kb & 1
            ds_stage_wait();
            __syncthreads();
        }
        float acc[kDSRed];
#pragma unroll
        for (int v = 0; v < kDSRed; ++v) acc[v] = 0.0f;
        const bool has_prev = kb > 0, has_cur = kb < KB;
#define DS_ACCUMULATE(R_, V)                                               \
        do {                                                               \
            _Pragma("unroll") for (int k = 0; k < kAtomBlock; ++k) {       \
                acc[k] = fmaf(V.v[k], R_, acc[k]);                         \
                _Pragma("unroll") for (int l = 0; l <= k; ++l)             \
                    acc[kAtomBlock + k * (k + 1) / 2 + l] =                \
                        fmaf(V.v[k], V.v[l], acc[kAtomBlock + k * (k + 1) / 2 + l]); \
            }                                                              \
        } while (0)
        if (STAGED) {
            const float* sprev = bufs + (size_t)((kb + 1) & 1) * a.buf_floats;   // block kb - 1
            const float* scur = bufs + (size_t)(kb & 1) * a.buf_floats;          // block kb
            const int half = a.half_floats;
#define DS_PAIR(J_, PX, RX)                                                \
            do {                                                           \
                const int l_ = PX;                                         \
                float r_ = RX;                                             \
                DS_HEAD((J_) + 4, PX, RX);                                 \
                if (has_prev) {                                            \
                    const W8 u_ = lds_w8_split(sprev, half, l_);           \
                    _Pragma("unroll") for (int k = 0; k < kAtomBlock; ++k) \
                        r_ = fmaf(-dq[k], u_.v[k], r_);                    \
                    rho[(size_t)(J_) * T] = r_;                            \
                }                                                          \
                if (has_cur) {                                             \
                    const W8 v_ = lds_w8_split(scur, half, l_);            \
                    DS_ACCUMULATE(r_, v_);                                 \
                }                                                          \
            } while (0)
            for (int jp = 0; jp < np; jp += 4) {
                DS_PAIR(jp, hp0, hr0);
                if (jp + 1 < np) DS_PAIR(jp + 1, hp1, hr1);
                if (jp + 2 < np) DS_PAIR(jp + 2, hp2, hr2);
                if (jp + 3 < np) DS_PAIR(jp + 3, hp3, hr3);
            }
#undef DS_PAIR
        } else {
            const float* qprev = a.W + (long long)(kb > 0 ? kb - 1 : 0) * Npad * kAtomBlock;
            const float* qcur = a.W + (long long)(kb < KB ? kb : 0) * Npad * kAtomBlock;
            // two pairs in flight: the loads of one are issued before the other
            // is applied (alternating register sets, no copies of pending loads)
            W8 ua, va, ub, vb;
            float ra = 0.0f, rb = 0.0f;
            // each register set's next patch index is loaded one loop iteration
            // (two pairs) before the weight loads that use it
            int pa = np > 0 ? pid[0] : 0, pb = np > 1 ? pid[(size_t)T] : 0;
#define DS_LOAD(J_, R_, U, V, PX)                                          \
            do {                                                           \
                const long long i_ = PX;                                   \
                PX = (J_) + 2 < np ? pid[(size_t)((J_) + 2) * T] : 0;      \
                R_ = rho[(size_t)(J_) * T];                                \
                if (has_prev) U = load_w8(qprev + i_ * kAtomBlock);        \
                if (has_cur) V = load_w8(qcur + i_ * kAtomBlock);          \
            } while (0)
#define DS_APPLY(J_, R_, U, V)                                             \
            do {                                                           \
                if (has_prev) {                                            \
                    _Pragma("unroll") for (int k = 0; k < kAtomBlock; ++k) \
                        R_ = fmaf(-dq[k], U.v[k], R_);                     \
                    rho[(size_t)(J_) * T] = R_;                            \
                }                                                          \
                if (has_cur) DS_ACCUMULATE(R_, V);                         \
            } while (0)
            if (np > 0) DS_LOAD(0, ra, ua, va, pa);
            for (int jp = 0; jp < np; jp += 2) {
                if (jp + 1 < np) DS_LOAD(jp + 1, rb, ub, vb, pb);
                DS_APPLY(jp, ra, ua, va);
                if (jp + 1 >= np) break;
                if (jp + 2 < np) DS_LOAD(jp + 2, ra, ua, va, pa);
                DS_APPLY(jp + 1, rb, ub, vb);
            }
#undef DS_LOAD
#undef DS_APPLY
        }
#undef DS_ACCUMULATE
        if (kb == KB) break;

        // per chain: sum the groups in order and publish the CTA partial
        // part[q][c][v].  With several groups the sums are staged in shared
        // memory (group 0 overwrites its own row of slot 0 after reading it)
        // and the whole CTA stores them as P contiguous 44-word runs.  When
        // staged, the scratch may be the buffer of block kb - 1, which the
        // pass has just finished reading.
        const bool red_in_buf = STAGED && a.red_sep_floats == 0;
        float* red = red_in_buf ? bufs + (size_t)((kb + 1) & 1) * a.buf_floats : red_sep;
        if (red_in_buf) __syncthreads();
        if (active && grp > 0) {
#pragma unroll
            for (int v = 0; v < kDSRed; ++v) red[((size_t)(grp - 1) * P + q) * kDSRedPad + v] = acc[v];
        }
        __syncthreads();
        if (active && grp == 0) {
            for (int h = 1; h < G; ++h) {
#pragma unroll
                for (int v = 0; v < kDSRed; ++v) acc[v] += red[((size_t)(h - 1) * P + q) * kDSRedPad + v];
            }
            if (G > 1) {
#pragma unroll
                for (int v = 0; v < kDSRed; ++v) red[(size_t)q * kDSRedPad + v] = acc[v];
            } else {
#pragma unroll
                for (int v = 0; v < kDSRed; ++v) a.part[((size_t)q * ncta + c) * kDSRed + v] = acc[v];
            }
        }
        if (G > 1) {
            __syncthreads();
            for (int e = t; e < P * kDSRed; e += T) {
                const int qq = e / kDSRed, v = e - qq * kDSRed;
                a.part[((size_t)qq * ncta + c) * kDSRed + v] = red[(size_t)qq * kDSRedPad + v];
            }
        }
        // grid barrier: arrive once the whole CTA has published; then, before
        // waiting, copy block kb + 1 into buffer (kb + 1) & 1 (free now that
        // every thread is past the pass and the publish) and load the head
        // of the next pass, all of which overlaps the other CTAs' arrivals
        __shared__ int ok_s;
        __syncthreads();
        if (t == 0) grid_arrive(a.bar);
        if (STAGED) {
            if (kb + 1 < KB)
                ds_stage(bufs + (size_t)((kb + 1) & 1) * a.buf_floats, a.half_floats,
                         a.W + (long long)(kb + 1) * Npad * kAtomBlock, rowbase, nrec, elast);
            DS_HEAD(0, hp0, hr0);
            DS_HEAD(1, hp1, hr1);
            DS_HEAD(2, hp2, hr2);
            DS_HEAD(3, hp3, hr3);
        }
        if (t == 0) ok_s = grid_wait(a.bar, (unsigned int)(2 * kb + 1) * ncta, &a.sc->status);
        __syncthreads();
        if (!ok_s) {
            if (STAGED) ds_stage_wait();
            return;
        }

        // chains c, c + grid, ...: fixed-order compensated sums of the CTA
        // partials, then the 8 sequential draws
        for (int ch = c; ch < P; ch += ncta) {
            // 11 groups of CTAs per value; each thread's loads are issued
            // together (independent), then summed in order
            const int per = (ncta + 10) / 11;
            if (t < kDSRed * 11) {
                const int v = t % kDSRed, h = t / kDSRed;
                const int c0 = h * per, c1 = min(ncta, (h + 1) * per);
                float sum = 0.0f, err = 0.0f;
                for (int cb = c0; cb < c1; cb += 16) {
                    float x[16];
#pragma unroll
                    for (int u = 0; u < 16; ++u)
                        x[u] = (cb + u < c1) ? __ldcg(&a.part[((size_t)ch * ncta + cb + u) * kDSRed + v]) : 0.0f;
#pragma unroll
                    for (int u = 0; u < 16; ++u) two_sum_acc(sum, err, x[u]);
                }
                tmp_s[v][h] = sum;
                tmp_e[v][h] = err;
            }
            if (t < kAtomBlock && kb * kAtomBlock + t < K) dold8[t] = a.D[(long long)(kb * kAtomBlock + t) * P + ch];
            __syncthreads();
            if (t < kDSRed) {
                float sum = 0.0f, err = 0.0f;
                for (int h = 0; h < 11; ++h) {
                    two_sum_acc(sum, err, tmp_s[t][h]);
                    err += tmp_e[t][h];
                }
                fin[t] = sum + err;
            }
            __syncthreads();
            const float* xo = xis + (size_t)((ch - c) / ncta) * K;
            if (t < kAtomBlock) {
                // per atom, in parallel: gamma_eps / Lambda and the noise term Lambda^-1/2 xi
                const int k = kb * kAtomBlock + t;
                const float ckk = fin[kAtomBlock + t * (t + 1) / 2 + t];
                const float prec = (float)P + gef * ckk;
                gain8[t] = gef / prec;
                noise8[t] = k < K ? xo[k] * rsqrtf(prec) : 0.0f;
            }
            __syncthreads();
            if (t == 0) {
                // the 8 sequential draws in FP32 on the reduced sums
                float dl[kAtomBlock];
                for (int kk = 0; kk < kAtomBlock; ++kk) {
                    const int k = kb * kAtomBlock + kk;
                    dl[kk] = 0.0f;
                    if (k >= K) continue;
                    const float d_old = dold8[kk];
                    const float ckk = fin[kAtomBlock + kk * (kk + 1) / 2 + kk];
                    float num = fin[kk] + d_old * ckk;                    // sum w_k r^{-k}
                    for (int l = 0; l < kk; ++l) num = fmaf(-dl[l], fin[kAtomBlock + kk * (kk + 1) / 2 + l], num);
                    const float dnew = fmaf(gain8[kk], num, noise8[kk]);
                    a.D[(long long)k * P + ch] = dnew;
                    dl[kk] = dnew - d_old;
                }
                for (int kk = 0; kk < kAtomBlock; ++kk) a.delta[ch * kAtomBlock + kk] = dl[kk];
            }
            __syncthreads();
        }
        if (!grid_barrier(a.bar, (unsigned int)(2 * kb + 2) * ncta, &a.sc->status)) {
            if (STAGED) ds_stage_wait();
            return;
        }
        if (active) {
#pragma unroll
            for (int k = 0; k < kAtomBlock; ++k) dq[k] = __ldcg(&a.delta[q * kAtomBlock + k]);
        }
    }

#undef DS_HEAD
    // write the residual back; this CTA's share of sum ||r||^2
    float r2 = 0.0f;
    for (int jp = 0; jp < np; ++jp) {
        const float v = rho[(size_t)jp * T];
        if (RHO_SMEM) a.R[base + t + (long long)jp * T] = v;
        r2 = fmaf(v, v, r2);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r2 += __shfl_down_sync(0xffffffffu, r2, o);
    if (lane == 0) r2_s[warp] = r2;
    __syncthreads();
    if (t == 0) {
        double s = 0.0;
        for (int w = 0; w < kDSThreads / 32; ++w) s += (double)r2_s[w];
        a.part_r2[c] = s;
    }
}

// ------------------------------------------------------------ host planning --

namespace {

struct Box {
    int lo[kMaxDim], hi[kMaxDim];
};

// Calls f(u, coords) for the pixels of [lo, hi) in raster order.
template <class F>
void for_box(const Geom& g, const int* lo, const int* hi, F f)
{
    const int nd = g.ndim;
    int cd[kMaxDim];
    for (int d = 0; d < nd; ++d) {
        if (lo[d] >= hi[d]) return;
        cd[d] = lo[d];
    }
    for (;;) {
        long long u = 0;
        for (int d = 0; d < nd; ++d) u = u * g.M[d] + cd[d];
        f(u, cd);
        int d = nd - 1;
        while (d >= 0) {
            if (++cd[d] < hi[d]) break;
            cd[d] = lo[d];
            --d;
        }
        if (d < 0) return;
    }
}

// Recursive bisection into n boxes with balanced observed counts: cut the
// longest side where the lower part holds n1 / n of the box's pixels.
void split_boxes(const Geom& g, const uint8_t* mask, const Box& b, int n, std::vector<Box>& out)
{
    if (n == 1) {
        out.push_back(b);
        return;
    }
    int dim = 0;
    for (int d = 1; d < g.ndim; ++d)
        if (b.hi[d] - b.lo[d] > b.hi[dim] - b.lo[dim]) dim = d;
    const int ext = b.hi[dim] - b.lo[dim];
    const int n1 = n / 2;
    if (ext < 2) {   // cannot cut: the remaining boxes are empty
        out.push_back(b);
        Box e = b;
        e.hi[dim] = e.lo[dim];
        for (int k = 1; k < n; ++k) out.push_back(e);
        return;
    }
    std::vector<long long> slab(ext, 0);
    long long total = 0;
    for_box(g, b.lo, b.hi, [&](long long u, const int* cd) {
        if (mask[u]) {
            ++slab[cd[dim] - b.lo[dim]];
            ++total;
        }
    });
    const long long target = total * n1 / n;
    int cut = 1;
    long long acc = slab[0];
    while (cut < ext - 1 && acc < target) acc += slab[cut++];
    Box lo = b, hi = b;
    lo.hi[dim] = b.lo[dim] + cut;
    hi.lo[dim] = b.lo[dim] + cut;
    split_boxes(g, mask, lo, n1, out);
    split_boxes(g, mask, hi, n - n1, out);
}

// Observed pixels of each box, tile by tile, raster order inside a tile.
void order_pixels(const Geom& g, const uint8_t* mask, int ncta, std::vector<int>& order, std::vector<int>& start,
                  std::vector<Box>& boxes)
{
    Box all;
    for (int d = 0; d < g.ndim; ++d) {
        all.lo[d] = 0;
        all.hi[d] = (int)g.M[d];
    }
    boxes.clear();
    split_boxes(g, mask, all, ncta, boxes);
    int tile[kMaxDim];
    for (int d = 0; d < g.ndim; ++d) tile[d] = std::max(1, std::min(g.B[d], 8));
    order.clear();
    start.assign(1, 0);
    for (const Box& b : boxes) {
        Box tg;   // tile grid of the box
        for (int d = 0; d < g.ndim; ++d) {
            tg.lo[d] = 0;
            tg.hi[d] = b.hi[d] > b.lo[d] ? (b.hi[d] - b.lo[d] + tile[d] - 1) / tile[d] : 0;
        }
        for_box(g, tg.lo, tg.hi, [&](long long, const int* tc) {
            int lo[kMaxDim], hi[kMaxDim];
            for (int d = 0; d < g.ndim; ++d) {
                lo[d] = b.lo[d] + tc[d] * tile[d];
                hi[d] = std::min(b.hi[d], lo[d] + tile[d]);
            }
            for_box(g, lo, hi, [&](long long u, const int*) {
                if (mask[u]) order.push_back((int)u);
            });
        });
        start.push_back((int)order.size());
    }
}

size_t ds_fixed_smem()
{
    return sizeof(float) * (kDSRed + 2 * kDSRed * 11 + 3 * kAtomBlock + kDSThreads / 32) + 256;
}

// The patch-grid neighbourhood of box b: the patches holding any of its
// pixels, origin o[d] and extents o[kMaxDim + d].  Returns the record count.
long long box_neighbourhood(const Geom& g, const Box& b, int* o)
{
    long long n = 1;
    for (int d = 0; d < g.ndim; ++d) {
        int a0 = 0, a1 = -1;
        if (b.hi[d] > b.lo[d]) {
            const long long lo = (long long)b.lo[d] - g.B[d] + 1;   // first pixel a patch may start at
            a0 = lo <= 0 ? 0 : (int)((lo + g.S[d] - 1) / g.S[d]);
            a1 = (int)std::min<long long>(g.G[d] - 1, (b.hi[d] - 1) / g.S[d]);
        }
        o[d] = a0;
        o[kMaxDim + d] = std::max(0, a1 - a0 + 1);
        n *= o[kMaxDim + d];
    }
    return n;
}

void* ds_kernel_fn(const DictSpacePlan& p)
{
    if (p.staged) return p.rho_smem ? (void*)dict_space_kernel<true, true> : (void*)dict_space_kernel<false, true>;
    return p.rho_smem ? (void*)dict_space_kernel<true, false> : (void*)dict_space_kernel<false, false>;
}

}  // namespace

void ds_free(DictSpacePlan* p)
{
    void* ptrs[] = {p->order, p->start, p->np, p->base, p->pidx, p->part, p->delta, p->bar, p->nb};
    for (void* v : ptrs)
        if (v) cudaFree(v);
    *p = DictSpacePlan{};
}

cudaError_t ds_build(const Geom& g, const uint8_t* mask, const uint16_t* obs, const uint16_t* nobs, int device,
                     int* pos, float** R, DictSpacePlan* plan, cudaStream_t s)
{
    *plan = DictSpacePlan{};
    *R = nullptr;
    const int P = g.P;
    if (P > kDSThreads) return cudaSuccess;
    int optin = 0, sms = 0, coop = 0;
    cudaError_t e;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device)) != cudaSuccess) return e;
    if (!coop) return cudaSuccess;
    const int grid = sms;
    const int G = kDSThreads / P;
    const int own = (P + grid - 1) / grid;
    const size_t red_floats = (size_t)(G - 1) * P * kDSRedPad;
    const size_t base_smem = sizeof(float) * (red_floats + (size_t)own * g.K);
    if (base_smem + ds_fixed_smem() > (size_t)optin) return cudaSuccess;

    std::vector<int> order, start;
    std::vector<Box> boxes;
    order_pixels(g, mask, grid, order, start, boxes);
    if (order.empty()) return cudaSuccess;

    DictSpacePlan p{};
#define DS_TRY(x)                  \
    do {                           \
        if ((e = (x)) != cudaSuccess) { \
            ds_free(&p);           \
            return e;              \
        }                          \
    } while (0)
    DS_TRY(cudaMalloc((void**)&p.order, sizeof(int) * order.size()));
    DS_TRY(cudaMalloc((void**)&p.start, sizeof(int) * start.size()));
    DS_TRY(cudaMalloc((void**)&p.np, sizeof(int) * (size_t)grid * kDSThreads));
    DS_TRY(cudaMalloc((void**)&p.base, sizeof(long long) * (size_t)grid));
    DS_TRY(cudaMemcpy(p.order, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice));
    DS_TRY(cudaMemcpy(p.start, start.data(), sizeof(int) * start.size(), cudaMemcpyHostToDevice));
    int* npmax_d = nullptr;
    DS_TRY(cudaMalloc((void**)&npmax_d, sizeof(int) * (size_t)grid));
    ds_count_kernel<<<grid, kDSThreads, 0, s>>>(g, p.order, p.start, p.np, npmax_d);
    std::vector<int> npmax(grid);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(npmax.data(), npmax_d, sizeof(int) * grid, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(npmax_d);
    if (e != cudaSuccess) {
        ds_free(&p);
        return e;
    }
    std::vector<long long> base(grid);
    long long total = 0;
    for (int c = 0; c < grid; ++c) {
        base[c] = total;
        total += (long long)npmax[c] * kDSThreads;
        p.max_np = std::max(p.max_np, npmax[c]);
    }
    if (total >= (1LL << 31)) {   // the sweep's pair table holds int32 indices
        ds_free(&p);
        return cudaSuccess;
    }
    DS_TRY(cudaMemcpy(p.base, base.data(), sizeof(long long) * grid, cudaMemcpyHostToDevice));

    // Staging: every CTA's neighbourhood in two buffers of the largest (the
    // group-sum scratch shares the buffer of the previous block when it fits).
    std::vector<int> nbh((size_t)grid * 2 * kMaxDim, 0);
    long long nrec_max = 0, rows_max = 0;
    for (int c = 0; c < grid; ++c) {
        int* o = &nbh[(size_t)c * 2 * kMaxDim];
        const long long n = box_neighbourhood(g, boxes[c], o);
        const int el = o[kMaxDim + g.ndim - 1];
        nrec_max = std::max(nrec_max, n);
        rows_max = std::max(rows_max, el > 0 ? n / el : 0LL);
    }
    const long long half = (nrec_max * 4 + 31) / 32 * 32;
    const size_t stage_red = red_floats <= (size_t)(2 * half) ? 0 : red_floats;
    const size_t rows_pad = (size_t)(rows_max + 3) / 4 * 4;
    const size_t staged_smem = sizeof(float) * ((size_t)(4 * half) + stage_red + rows_pad + (size_t)own * g.K);
    p.staged = nrec_max > 0 && staged_smem + ds_fixed_smem() <= (size_t)optin;
    if (p.staged) {
        p.half_floats = (int)half;
        p.buf_floats = (int)(2 * half);
        p.red_sep_floats = (int)stage_red;
        p.rows_max = (int)rows_pad;
        DS_TRY(cudaMalloc((void**)&p.nb, sizeof(int) * nbh.size()));
        DS_TRY(cudaMemcpy(p.nb, nbh.data(), sizeof(int) * nbh.size(), cudaMemcpyHostToDevice));
    } else {
        p.red_sep_floats = (int)red_floats;
    }
    DS_TRY(cudaMalloc((void**)&p.pidx, sizeof(int) * (size_t)(total > 0 ? total : 1)));
    float* Rd = nullptr;
    DS_TRY(cudaMalloc((void**)&Rd, sizeof(float) * (size_t)(total > 0 ? total : 1)));
    e = cudaMemsetAsync(Rd, 0, sizeof(float) * (size_t)(total > 0 ? total : 1), s);
    if (e == cudaSuccess) {
        ds_fill_kernel<<<grid, kDSThreads, 0, s>>>(g, p.order, p.start, p.base, obs, nobs, p.nb, p.pidx, pos);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(Rd);
        ds_free(&p);
        return e;
    }
    // the residual pairs in shared memory: beside staged weights when they
    // fit; else when that leaves >= 64 KB of L1 for the weight records
    const size_t rho_bytes = sizeof(float) * (size_t)p.max_np * kDSThreads;
    if (p.staged)
        p.rho_smem = staged_smem + rho_bytes + ds_fixed_smem() <= (size_t)optin;
    else
        p.rho_smem = base_smem + rho_bytes + ds_fixed_smem() <= (size_t)160 * 1024;
    p.smem = (p.staged ? staged_smem : base_smem) + (p.rho_smem ? rho_bytes : 0);
    void* fn = ds_kernel_fn(p);
    int per_sm = 0;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kDSThreads, p.smem);
    if (e == cudaSuccess && per_sm >= 1) {
        e = cudaMalloc((void**)&p.part, sizeof(float) * (size_t)grid * kDSRed * P);
        if (e == cudaSuccess) e = cudaMalloc((void**)&p.delta, sizeof(float) * (size_t)P * kAtomBlock);
        if (e == cudaSuccess) e = cudaMalloc((void**)&p.bar, 2 * sizeof(unsigned int));
        if (e == cudaSuccess) e = cudaMemset(p.bar, 0, 2 * sizeof(unsigned int));
    }
    if (e != cudaSuccess || per_sm < 1) {
        cudaFree(Rd);
        ds_free(&p);
        return e;
    }
#undef DS_TRY
    p.grid = grid;
    p.own_max = own;
    p.pairs = total;
    *plan = p;
    *R = Rd;
    return cudaSuccess;
}

cudaError_t launch_dict_space(const DictSpaceArgs& args_in, const DictSpacePlan& p, cudaStream_t s)
{
    DictSpaceArgs a = args_in;
    a.nb = p.nb;
    a.half_floats = p.half_floats;
    a.buf_floats = p.buf_floats;
    a.red_sep_floats = p.red_sep_floats;
    a.rows_max = p.rows_max;
    void* fn = ds_kernel_fn(p);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(a.bar, 0, sizeof(unsigned int), s);   // the barrier counts from zero each launch
    if (e != cudaSuccess) return e;
    void* args[] = {(void*)&a};
    return cudaLaunchCooperativeKernel(fn, dim3(p.grid), dim3(kDSThreads), args, p.smem, s);
}

}  // namespace sensai
