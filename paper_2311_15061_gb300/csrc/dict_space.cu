// dict_space.cu -- the dictionary sweep organised by space.
//
// Same draws as dict.cu (the atom-ordered conjugate Gaussian of every d_kp,
// in 8-atom blocks with the in-block Gram correction), but the work is split
// over the frame instead of over pixel chains.  A pair (u, q) -- an observed
// frame pixel u and a within-patch pixel q such that u - q is a patch origin
// -- is one residual slot of chain q.  CTA c owns a contiguous range of
// observed pixels in raster order; inside it, a thread owns one chain q and a
// sub-range of those pixels, so its pairs are consecutive slots of chain q
// (slots are ranked by patch index, which grows with u).  For one pixel u the
// ~P patches covering it form a small neighbourhood of the patch grid, whose
// 32-byte weight records are contiguous rows that the next pixels reuse: the
// gathers of the per-chain kernel become local, mostly L1-resident reads, and
// every SM takes part.
//
// Per 8-atom block: (1) every thread accumulates G_k = sum w_k r and the
// in-block Gram C_kl over its pairs (after applying the previous block's
// update); (2) the CTA sums its threads per chain in a fixed order and
// publishes the partial; (3) grid barrier; (4) CTA c sums the partials of
// chains c, c + grid, ... over all CTAs in a fixed order (FP64) and draws the
// block's 8 atoms at those pixels; (5) grid barrier; (6) every thread reads
// its chain's 8 updates.
// One cooperative launch, one CTA per SM; the barrier spins are bounded and
// report SENSAI_ETIMEOUT through the status word instead of hanging.
#include "internal.cuh"

namespace sensai {

constexpr int kDSThreads = 512;
constexpr int kDSGram = kAtomBlock * (kAtomBlock + 1) / 2;   // 36
constexpr int kDSRed = kAtomBlock + kDSGram;                  // 44
constexpr int kDSRedPad = kDSRed + 1;                          // smem row pitch (odd)
constexpr long long kBarrierSpins = 1LL << 24;               // x ~64 ns sleep: ~1 s

// Sense-free grid barrier on a (count, generation) pair: the last CTA to
// arrive resets the count and bumps the generation.  Returns false (and sets
// *status) if the generation does not move within the spin limit.
__device__ bool grid_barrier(unsigned int* count, unsigned int* gen, unsigned int nblocks, int* status)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned int* vgen = gen;
        const unsigned int g0 = *vgen;
        __threadfence();
        const unsigned int arrived = atomicAdd(count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            long long spins = 0;
            while (*vgen == g0) {
                if (++spins > kBarrierSpins) {
                    atomicExch(status, (int)SENSAI_ETIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

__global__ void __launch_bounds__(kDSThreads, 1) dict_space_kernel(const DictSpaceArgs a)
{
    extern __shared__ float dyn[];
    __shared__ float dold8[kAtomBlock];
    __shared__ double fin[kDSRed];
    __shared__ double tmp[kDSRed][11];
    __shared__ int scan_s[kDSThreads / 32];
    __shared__ float r2_s[kDSThreads / 32];
    const Geom& g = a.g;
    const int P = g.P, K = g.K, KB = g.KB, nd = g.ndim;
    const long long Npad = g.Npad;
    const int c = blockIdx.x, ncta = gridDim.x;
    const int G = kDSThreads / P;                    // groups of P threads
    const int t = threadIdx.x;
    const bool active = t < G * P;
    const int grp = active ? t / P : 0, q = active ? t % P : 0;
    const int lane = t & 31, warp = t >> 5;

    // this CTA's observed pixels and this thread's sub-range of them
    const long long n0 = (long long)a.n_obs_px * c / ncta, n1 = (long long)a.n_obs_px * (c + 1) / ncta;
    const int L = (int)(n1 - n0);
    const int s0 = (int)((long long)L * grp / G), s1 = active ? (int)((long long)L * (grp + 1) / G) : s0;
    int* coord = reinterpret_cast<int*>(dyn);                      // [L][nd] multi-indices
    float* red = reinterpret_cast<float*>(coord + (size_t)a.max_tile * nd);   // [G-1][P][44]
    float* rho = red + (size_t)(kDSThreads / P - 1) * P * kDSRedPad;          // this CTA's pairs
    int* pidx = reinterpret_cast<int*>(rho + (size_t)a.max_tile * P);         // their patch indices
    float* xis = reinterpret_cast<float*>(pidx + (size_t)a.max_tile * P);     // normals of owned chains
    for (int j = t; j < L; j += blockDim.x) {
        long long u = a.obs_px[n0 + j];
        for (int d = nd - 1; d >= 0; --d) {
            coord[j * nd + d] = (int)(u % g.M[d]);
            u /= g.M[d];
        }
    }
    int qd[kMaxDim];
    {
        int rem = q;
        for (int d = nd - 1; d >= 0; --d) {
            qd[d] = rem % g.B[d];
            rem /= g.B[d];
        }
    }
    __syncthreads();

    // patch index of pair (tile pixel j, chain q), or -1
    auto patch_of = [&](int j) -> long long {
        long long i = 0;
        for (int d = 0; d < nd; ++d) {
            int av = coord[j * nd + d] - qd[d];
            if (av < 0) return -1;
            if (g.S[d] != 1) {
                if (av % g.S[d]) return -1;
                av /= g.S[d];
            }
            if (av >= g.G[d]) return -1;
            i = i * g.G[d] + av;
        }
        return i;
    };

    // count this thread's pairs; exclusive scan gives its residual offset
    int np = 0;
    long long first_i = -1;
    for (int j = s0; j < s1; ++j) {
        const long long i = patch_of(j);
        if (i >= 0) {
            if (np == 0) first_i = i;
            ++np;
        }
    }
    int incl = np;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) scan_s[warp] = incl;
    __syncthreads();
    int wbase = 0;
    for (int w = 0; w < warp; ++w) wbase += scan_s[w];
    const int ro = wbase + incl - np;           // offset of this thread's pairs in rho
    int slot0 = 0;
    if (np > 0) {
        const long long wd = (long long)q * g.NW + (first_i >> 5);
        slot0 = a.Rbase[q] + (int)a.Ipre[wd] + __popc(a.Ibits[wd] & ((1u << (first_i & 31)) - 1u));
        int jp = 0;
        for (int j = s0; j < s1; ++j) {
            const long long i = patch_of(j);
            if (i < 0) continue;
            rho[ro + jp] = a.R[slot0 + jp];
            pidx[ro + jp] = (int)i;
            ++jp;
        }
    }
    // normals of this CTA's chains (c, c + grid, ...), off the sequential path
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

    for (int kb = 0; kb <= KB; ++kb) {
        float acc[kDSRed];
#pragma unroll
        for (int v = 0; v < kDSRed; ++v) acc[v] = 0.0f;
        const float* qprev = a.W + (long long)(kb > 0 ? kb - 1 : 0) * Npad * kAtomBlock;
        const float* qcur = a.W + (long long)(kb < KB ? kb : 0) * Npad * kAtomBlock;
        // two pairs in flight: the loads of one are issued before the other
        // is applied (alternating register sets, no copies of pending loads)
        const bool has_prev = kb > 0, has_cur = kb < KB;
        W8 ua, va, ub, vb;
        float ra = 0.0f, rb = 0.0f;
#define DS_LOAD(J_, R_, U, V)                                              \
        do {                                                               \
            const long long i_ = pidx[ro + (J_)];                          \
            R_ = rho[ro + (J_)];                                           \
            if (has_prev) U = load_w8(qprev + i_ * kAtomBlock);            \
            if (has_cur) V = load_w8(qcur + i_ * kAtomBlock);              \
        } while (0)
#define DS_APPLY(J_, R_, U, V)                                             \
        do {                                                               \
            if (has_prev) {                                                \
                _Pragma("unroll") for (int k = 0; k < kAtomBlock; ++k)     \
                    R_ = fmaf(-dq[k], U.v[k], R_);                         \
                rho[ro + (J_)] = R_;                                       \
            }                                                              \
            if (has_cur) {                                                 \
                _Pragma("unroll") for (int k = 0; k < kAtomBlock; ++k) {   \
                    acc[k] = fmaf(V.v[k], R_, acc[k]);                     \
                    _Pragma("unroll") for (int l = 0; l <= k; ++l)         \
                        acc[kAtomBlock + k * (k + 1) / 2 + l] =            \
                            fmaf(V.v[k], V.v[l], acc[kAtomBlock + k * (k + 1) / 2 + l]); \
                }                                                          \
            }                                                              \
        } while (0)
        if (np > 0) DS_LOAD(0, ra, ua, va);
        for (int jp = 0; jp < np; jp += 2) {
            if (jp + 1 < np) DS_LOAD(jp + 1, rb, ub, vb);
            DS_APPLY(jp, ra, ua, va);
            if (jp + 1 >= np) break;
            if (jp + 2 < np) DS_LOAD(jp + 2, ra, ua, va);
            DS_APPLY(jp + 1, rb, ub, vb);
        }
#undef DS_LOAD
#undef DS_APPLY
        if (kb == KB) break;

        // per chain: sum the groups in order, publish the CTA partial [c][v][q]
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
#pragma unroll
            for (int v = 0; v < kDSRed; ++v) a.part[((size_t)c * kDSRed + v) * P + q] = acc[v];
        }
        __threadfence();
        if (!grid_barrier(a.bar, a.bar + 1, (unsigned int)ncta, &a.sc->status)) return;

        // chains c, c + grid, ...: fixed-order FP64 sums of the CTA partials,
        // the block's 8 normals in parallel, then the 8 sequential draws
        for (int ch = c; ch < P; ch += ncta) {
            // 11 groups of CTAs per value; each thread's loads are issued
            // together (independent), then summed in order
            const int per = (ncta + 10) / 11;
            if (t < kDSRed * 11) {
                const int v = t % kDSRed, h = t / kDSRed;
                const int c0 = h * per, c1 = min(ncta, (h + 1) * per);
                double sum = 0.0;
                for (int cb = c0; cb < c1; cb += 16) {
                    float x[16];
#pragma unroll
                    for (int u = 0; u < 16; ++u)
                        x[u] = (cb + u < c1) ? __ldcg(&a.part[((size_t)(cb + u) * kDSRed + v) * P + ch]) : 0.0f;
#pragma unroll
                    for (int u = 0; u < 16; ++u) sum += (double)x[u];
                }
                tmp[v][h] = sum;
            }
            if (t < kAtomBlock && kb * kAtomBlock + t < K) dold8[t] = a.D[(long long)(kb * kAtomBlock + t) * P + ch];
            __syncthreads();
            if (t < kDSRed) {
                double sum = 0.0;
                for (int h = 0; h < 11; ++h) sum += tmp[t][h];
                fin[t] = sum;
            }
            __syncthreads();
            if (t == 0) {
                // the 8 sequential draws in FP32 on the FP64-reduced sums
                const float* xo = xis + (size_t)((ch - c) / ncta) * K;
                float dl[kAtomBlock];
                for (int kk = 0; kk < kAtomBlock; ++kk) {
                    const int k = kb * kAtomBlock + kk;
                    dl[kk] = 0.0f;
                    if (k >= K) continue;
                    const float d_old = dold8[kk];
                    const float ckk = (float)fin[kAtomBlock + kk * (kk + 1) / 2 + kk];
                    float num = (float)fin[kk] + d_old * ckk;             // sum w_k r^{-k}
                    for (int l = 0; l < kk; ++l) num = fmaf(-dl[l], (float)fin[kAtomBlock + kk * (kk + 1) / 2 + l], num);
                    const float prec = (float)P + gef * ckk;
                    const float dnew = gef * num / prec + xo[k] * rsqrtf(prec);
                    a.D[(long long)k * P + ch] = dnew;
                    dl[kk] = dnew - d_old;
                }
                for (int kk = 0; kk < kAtomBlock; ++kk) a.delta[ch * kAtomBlock + kk] = dl[kk];
            }
            __syncthreads();
        }
        __threadfence();
        if (!grid_barrier(a.bar, a.bar + 1, (unsigned int)ncta, &a.sc->status)) return;
        if (active) {
#pragma unroll
            for (int k = 0; k < kAtomBlock; ++k) dq[k] = __ldcg(&a.delta[q * kAtomBlock + k]);
        }
    }

    // write the residual back; this CTA's share of sum ||r||^2
    float r2 = 0.0f;
    for (int j = 0; j < np; ++j) {
        const float v = rho[ro + j];
        a.R[slot0 + j] = v;
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

size_t dict_space_smem_bytes(const Geom& g, int max_tile, int max_pairs, int own_max)
{
    const int G = kDSThreads / g.P;
    return sizeof(int) * (size_t)max_tile * g.ndim + sizeof(float) * (size_t)(G > 0 ? G - 1 : 0) * g.P * kDSRedPad +
           (sizeof(float) + sizeof(int)) * (size_t)max_pairs + sizeof(float) * (size_t)own_max * g.K;
}

// Grid for the cooperative launch (one CTA per SM) or 0 if it cannot run.
int dict_space_grid(const Geom& g, size_t smem, int device)
{
    if (g.P > kDSThreads) return 0;
    int optin = 0, sms = 0, coop = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device) != cudaSuccess || !coop) return 0;
    const size_t fixed = sizeof(double) * (kDSRed + kDSRed * 11) + 4 * kAtomBlock + 2 * 4 * (kDSThreads / 32) + 256;
    if (smem + fixed > (size_t)optin) return 0;
    if (cudaFuncSetAttribute((void*)dict_space_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (void*)dict_space_kernel, kDSThreads, smem) !=
            cudaSuccess ||
        per_sm < 1)
        return 0;
    return sms;   // one CTA per SM
}

cudaError_t launch_dict_space(const DictSpaceArgs& a, int grid, size_t smem, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute((void*)dict_space_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void* args[] = {(void*)&a};
    return cudaLaunchCooperativeKernel((void*)dict_space_kernel, dim3(grid), dim3(kDSThreads), args, smem, s);
}

}  // namespace sensai
