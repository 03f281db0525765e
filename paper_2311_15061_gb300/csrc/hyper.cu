// hyper.cu -- conjugate draws of pi_k, gamma_s and gamma_eps, the initial
// state, and the statistics passes behind them.
//
// From the model the BPFA section cites (Beta-Bernoulli and Gamma-Gaussian
// conjugacy), given the current codes, weights and residual:
//   pi_k      ~ Beta(a/K + m_k, b(K-1)/K + N - m_k),    m_k = sum_i z_ik
//   gamma_s   ~ Gamma(c + 1/2 sum_ik z_ik, d + 1/2 sum_{z_ik=1} s_ik^2)
//               (with SENSAI_FLAG_GAMMA_S_FULL: Gamma(c + N K / 2, d + 1/2 sum_ik s_ik^2),
//               the inactive s_ik being the sweep's prior draws)
//   gamma_eps ~ Gamma(e + 1/2 sum_i |Omega_i|, f + 1/2 sum_i ||r_i||^2)
// (shape, rate).  The global sums are FP64 and reduced in a fixed order from
// per-chunk (or per-pixel) partials, so the draws are deterministic.
#include "internal.cuh"

namespace sensai {

constexpr int kHyperThreads = 1024;

// Fixed-order sum of n partials: thread t adds a contiguous range, then a
// block tree.  Result in thread 0.
__device__ double sum_partials(const double* v, int n, double* red)
{
    const int per = (n + (int)blockDim.x - 1) / (int)blockDim.x;
    const int lo = threadIdx.x * per;
    const int hi = min(n, lo + per);
    double acc = 0.0;
    for (int j = lo; j < hi; ++j) acc += v[j];
    return block_sum(acc, red);
}

// pi_k ~ Beta(a/K + m_k, b(K-1)/K + N - m_k), one CTA per atom: m_k is the
// popcount of atom k's activity words (fixed-order sum), and the Beta draw's
// two Gamma draws run on two warps (the value is beta_draw's).  Spreading the
// atoms over the SMs matters: FP64 throughput per SM is low on this part.
__device__ __forceinline__ void pi_body(const HyperArgs& a, const int k)
{
    __shared__ int red[8];
    __shared__ double g2_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t t_it = launch_t(a.t, a.t_dev, a.sc);
    const uint32_t* z = a.Zb + (long long)k * a.g.NW;
    int c = 0;
    for (int w = threadIdx.x; w < a.g.NW; w += blockDim.x) c += __popc(z[w]);
    c = __reduce_add_sync(0xffffffffu, c);
    if (lane == 0) red[warp] = c;
    __syncthreads();
    int mk = 0;
    for (int w = 0; w < 8; ++w) mk += red[w];
    const double alpha = a.a_over_K + (double)mk;
    const double beta = a.b_scaled + (double)a.g.N - (double)mk;
    if (threadIdx.x == 32) g2_s = gamma_draw(beta, a.seed, (uint32_t)k, 0, t_it, kTagPiB);
    double g1 = 0.0;
    if (threadIdx.x == 0) g1 = gamma_draw(alpha, a.seed, (uint32_t)k, 0, t_it, kTagPiA);
    __syncthreads();
    if (threadIdx.x == 0) {
        const double pi = g1 / (g1 + g2_s);
        a.pi[k] = pi;
        a.lpi[k] = (float)(log(pi) - log1p(-pi));
        a.m[k] = mk;
    }
}

// gamma_s and gamma_eps from fixed-order FP64 sums of the per-unit partials;
// the two Gamma draws on two warps.  Last kernel of a batched iteration:
// advances the replay iteration index.
__device__ __forceinline__ void gamma_body(const HyperArgs& a)
{
    __shared__ double red[kHyperThreads / 32];
    __shared__ double ge_s;
    const int K = a.g.K;
    const uint32_t t_it = launch_t(a.t, a.t_dev, a.sc);
    const double s2 = sum_partials(a.part_s2, a.n_s2, red);
    const double r2 = sum_partials(a.part_r2, a.n_r2, red);
    double mk = 0.0;
    for (int k = threadIdx.x; k < K; k += blockDim.x) mk += (double)a.m[k];
    const double mtot = block_sum(mk, red);
    __shared__ double bc[3];
    if (threadIdx.x == 0) {
        bc[0] = s2;
        bc[1] = r2;
        bc[2] = mtot;
    }
    __syncthreads();
    if (threadIdx.x == 32)
        ge_s = gamma_draw(a.e + 0.5 * (double)a.n_observed, a.seed, 0, 0, t_it, kTagGe) / (a.f + 0.5 * bc[1]);
    double gs = 0.0;
    const double s_count = a.full_s ? (double)a.g.N * K : bc[2];   // entries whose s enters the s^2 sum
    if (threadIdx.x == 0) gs = gamma_draw(a.c + 0.5 * s_count, a.seed, 0, 0, t_it, kTagGs) / (a.d + 0.5 * bc[0]);
    __syncthreads();
    if (threadIdx.x == 0) {
        a.sc->gamma_s = gs;
        a.sc->gamma_eps = ge_s;
        a.sc->sum_s2 = bc[0];
        a.sc->sum_r2 = bc[1];
        a.sc->n_active = (long long)bc[2];
        if (a.t_dev) a.sc->t_iter = t_it + 1u;   // the next replay's iteration
    }
}

// Batched instances: pi draws with one CTA per (instance, atom), then the
// gamma draws with one CTA per instance.
__global__ void __launch_bounds__(256) pi_multi_kernel(const HyperArgs* __restrict__ args,
                                                       const int* __restrict__ cta_start, int n)
{
    int k = 0;
    const HyperArgs& a = *stage_instance_args(args, cta_start, n, &k);
    pi_body(a, k);
}

__global__ void __launch_bounds__(kHyperThreads) gamma_multi_kernel(const HyperArgs* __restrict__ args,
                                                                    const int* __restrict__ cta_start, int n)
{
    const HyperArgs& a = *stage_instance_args(args, cta_start, n);
    gamma_body(a);
}

cudaError_t launch_hyper_multi(const HyperArgs* args, const int* pi_start, const int* gamma_start, int n,
                               int pi_grid, cudaStream_t s)
{
    pi_multi_kernel<<<pi_grid, 256, 0, s>>>(args, pi_start, n);
    gamma_multi_kernel<<<n, kHyperThreads, 0, s>>>(args, gamma_start, n);
    return cudaGetLastError();
}

// Reading A of the gamma_s update: every entry the last code sweep left
// inactive (z_ik = 0, patch i < N) has its weight drawn from the prior,
// s_ik ~ N(0, 1/gamma_s), from the Philox words an active entry uses for its
// normal (counter (i, k, t, codes), words 1 and 2, the same Box-Muller
// normal); the weight z s stays 0, so only s_ik^2 is kept, added to the
// sweep's s^2 partial of the patch's work unit.  One warp per 32-slot
// activity word over all atoms (slot s holds patch perm[s]); lane 0 is the
// one writer of its unit.
__global__ void __launch_bounds__(256) prior_s2_kernel(Geom g, const uint32_t* Zb, const int* perm,
                                                       const DevScalars* sc, uint32_t t, bool t_dev,
                                                       unsigned long long seed, int lanes, double* part_s2)
{
    const long long w = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (w >= g.NW) return;
    const uint32_t t_it = launch_t(t, t_dev, sc);
    const float sd = rsqrtf((float)sc->gamma_s);
    const uint2 key = seed_key(seed);
    const long long slot = w * 32 + lane;
    const long long i = perm ? (long long)perm[slot] : slot;
    float s2 = 0.0f;
    if (i < g.N) {
        for (int k = 0; k < g.K; ++k) {
            if ((Zb[(long long)k * g.NW + w] >> lane) & 1u) continue;
            // the normal the code draw of atom k takes from its pair's block
            const uint4 blk = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)(k >> 1), t_it, kTagCodes), key);
            float nc, ns;
            normal32_pair(blk.z, blk.w, nc, ns);
            const float sp = ((k & 1) ? ns : nc) * sd;
            s2 = fmaf(sp, sp, s2);
        }
    }
    const double sum = warp_sum((double)s2);
    if (lane == 0) part_s2[lanes == 2 ? 2 * w : w] += sum;
}

cudaError_t launch_prior_s2(const Geom& g, const uint32_t* Zb, const int* perm, const DevScalars* sc, uint32_t t,
                            bool t_dev, unsigned long long seed, int lanes, double* part_s2, cudaStream_t s)
{
    if (lanes != 1 && lanes != 2) return cudaErrorInvalidValue;
    prior_s2_kernel<<<(unsigned int)((g.NW + 7) / 8), 256, 0, s>>>(g, Zb, perm, sc, t, t_dev, seed, lanes, part_s2);
    return cudaGetLastError();
}

// All of an iteration's draws in one launch of K + 1 CTAs.  CTA k < K
// counts m_k and draws pi_k (as pi_body); CTA K sums the s^2 and r^2
// partials and draws gamma_eps (as gamma_body).  gamma_s needs sum_k m_k and
// the s^2 sum, so the last CTA to publish its part (arrival counter, no
// waiting) sums the counts in index order and draws it on a warp of its own,
// then resets the counter.  Same sums in the same order and the same draw
// counters as the batched pi_multi_kernel + gamma_multi_kernel, so the values
// are identical; the Gamma chains of the K + 2 draws run concurrently instead
// of in two rounds.
__global__ void __launch_bounds__(kHyperThreads) hyper_kernel(const HyperArgs a)
{
    __shared__ int redi[kHyperThreads / 32];
    __shared__ double red[kHyperThreads / 32];
    __shared__ double g2_s, r2_s;
    __shared__ int last_s;
    const int K = a.g.K, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool is_pi = (int)blockIdx.x < K;
    const uint32_t t_it = launch_t(a.t, a.t_dev, a.sc);
    int mk = 0;
    if (is_pi) {
        const int k = blockIdx.x;
        const uint32_t* z = a.Zb + (long long)k * a.g.NW;
        int c = 0;
        for (int w = threadIdx.x; w < a.g.NW; w += blockDim.x) c += __popc(z[w]);
        c = __reduce_add_sync(0xffffffffu, c);
        if (lane == 0) redi[warp] = c;
        __syncthreads();
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mk += redi[w];
        if (threadIdx.x == 0) a.m[k] = mk;
    } else {
        const double s2 = sum_partials(a.part_s2, a.n_s2, red);   // valid in thread 0
        const double r2 = sum_partials(a.part_r2, a.n_r2, red);
        if (threadIdx.x == 0) {
            a.sc->sum_s2 = s2;
            a.sc->sum_r2 = r2;
            r2_s = r2;
        }
    }
    // publish this CTA's part; the last to arrive sees every part
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last_s = atomicAdd(a.arrive, 1u) == (unsigned int)K;
    }
    __syncthreads();
    double g1 = 0.0;
    if (is_pi) {
        const int k = blockIdx.x;
        const double alpha = a.a_over_K + (double)mk;
        const double beta = a.b_scaled + (double)a.g.N - (double)mk;
        if (threadIdx.x == 32) g2_s = gamma_draw(beta, a.seed, (uint32_t)k, 0, t_it, kTagPiB);
        if (threadIdx.x == 0) g1 = gamma_draw(alpha, a.seed, (uint32_t)k, 0, t_it, kTagPiA);
    } else if (threadIdx.x == 32) {
        a.sc->gamma_eps =
            gamma_draw(a.e + 0.5 * (double)a.n_observed, a.seed, 0, 0, t_it, kTagGe) / (a.f + 0.5 * r2_s);
    }
    if (last_s && threadIdx.x == 64) {
        __threadfence();
        double mtot = 0.0;
        for (int k = 0; k < K; ++k) mtot += (double)__ldcg(a.m + k);
        const double s2 = __ldcg(&a.sc->sum_s2);
        const double s_count = a.full_s ? (double)a.g.N * K : mtot;   // entries whose s enters the s^2 sum
        a.sc->gamma_s = gamma_draw(a.c + 0.5 * s_count, a.seed, 0, 0, t_it, kTagGs) / (a.d + 0.5 * s2);
        a.sc->n_active = (long long)mtot;
        atomicExch(a.arrive, 0u);
        if (a.t_dev) a.sc->t_iter = t_it + 1u;   // every CTA has read this replay's index
    }
    __syncthreads();
    if (is_pi && threadIdx.x == 0) {
        const int k = blockIdx.x;
        const double pi = g1 / (g1 + g2_s);
        a.pi[k] = pi;
        a.lpi[k] = (float)(log(pi) - log1p(-pi));
    }
}

cudaError_t launch_hyper(const HyperArgs& a, cudaStream_t s)
{
    if (!a.arrive) return cudaErrorInvalidValue;
    hyper_kernel<<<a.g.K + 1, kHyperThreads, 0, s>>>(a);
    return cudaGetLastError();
}

__global__ void set_iteration_kernel(DevScalars* sc, uint32_t t) { sc->t_iter = t; }

cudaError_t launch_set_iteration(DevScalars* sc, uint32_t t, cudaStream_t s)
{
    set_iteration_kernel<<<1, 1, 0, s>>>(sc, t);
    return cudaGetLastError();
}


// d_kp ~ N(0, 1/P) from counter (p, k, 0, INIT).
__global__ void init_dictionary_kernel(Geom g, float* D, unsigned long long seed)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)g.K * g.P) return;
    const int k = (int)(idx / g.P), p = (int)(idx % g.P);
    const uint4 blk = philox4x32_10(make_uint4((uint32_t)p, (uint32_t)k, 0u, kTagInit), seed_key(seed));
    D[idx] = (float)(normal64(blk.x, blk.y) / sqrt((double)g.P));
}

__global__ void init_scalars_kernel(int K, double* pi, float* lpi, DevScalars* sc)
{
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        pi[k] = 0.5;
        lpi[k] = 0.0f;
    }
    if (threadIdx.x == 0) {
        sc->gamma_s = 1.0;
        sc->gamma_eps = 0.0;
        sc->sum_s2 = 0.0;
        sc->sum_r2 = 0.0;
        sc->n_active = 0;
        sc->chg_n = 0;
        sc->chg_obs = 0;
        sc->act_n = 0;
        sc->rb_obs = 0;
        sc->ge_set = 0;
        sc->status = 0;
    }
}

// gamma_eps = 1 / max(var(frame over sampled pixels), 1e-12), two passes.
// Initial noise precision 1 / var(observed pixels), in two kernels: per CTA
// (a range of mask words, visiting only the observed bits) the count, the sum
// and the sum of squared deviations from the CTA's own mean, in FP64; then
// one CTA merges the partials pairwise in a fixed binary tree with the
// parallel variance update (n, mean, M2) + (n', mean', M2') -> (n + n',
// mean + d n' / (n + n'), M2 + M2' + d^2 n n' / (n + n')), d = mean' - mean,
// so the result does not depend on scheduling.
constexpr int kGeParts = kInitGammaEpsScratch / 3;

__global__ void __launch_bounds__(256) gamma_eps_parts_kernel(long long nframe, const float* x,
                                                              const uint32_t* mbits, double* part)
{
    __shared__ double red[8];
    __shared__ double s_mean;
    const long long nmw = (nframe + 31) / 32;
    const long long w0 = nmw * blockIdx.x / gridDim.x, w1 = nmw * (blockIdx.x + 1) / gridDim.x;
    const uint32_t tail = (nframe & 31) ? (1u << (nframe & 31)) - 1u : 0xffffffffu;
    double sum = 0.0, cnt = 0.0;
    for (long long w = w0 + threadIdx.x; w < w1; w += blockDim.x) {
        uint32_t bits = mbits[w] & (w == nmw - 1 ? tail : 0xffffffffu);
        cnt += (double)__popc(bits);
        while (bits) {
            const int b = __ffs(bits) - 1;
            sum += (double)x[w * 32 + b];
            bits &= bits - 1u;
        }
    }
    sum = block_sum(sum, red);
    cnt = block_sum(cnt, red);
    if (threadIdx.x == 0) s_mean = cnt > 0.0 ? sum / cnt : 0.0;
    __syncthreads();
    const double mean = s_mean;
    double ss = 0.0;
    for (long long w = w0 + threadIdx.x; w < w1; w += blockDim.x) {
        uint32_t bits = mbits[w] & (w == nmw - 1 ? tail : 0xffffffffu);
        while (bits) {
            const int b = __ffs(bits) - 1;
            const double dv = (double)x[w * 32 + b] - mean;
            ss += dv * dv;
            bits &= bits - 1u;
        }
    }
    ss = block_sum(ss, red);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x + 0] = cnt;
        part[3 * blockIdx.x + 1] = sum;
        part[3 * blockIdx.x + 2] = ss;
    }
}

__global__ void __launch_bounds__(kGeParts) gamma_eps_merge_kernel(const double* part, int nparts, DevScalars* sc)
{
    __shared__ double sn[kGeParts], smu[kGeParts], sm2[kGeParts];
    const int t = threadIdx.x;
    double n = 0.0, mu = 0.0, m2 = 0.0;
    if (t < nparts) {
        n = part[3 * t];
        if (n > 0.0) {
            mu = part[3 * t + 1] / n;
            m2 = part[3 * t + 2];
        }
    }
    sn[t] = n;
    smu[t] = mu;
    sm2[t] = m2;
    __syncthreads();
    for (int h = 1; h < kGeParts; h <<= 1) {
        if ((t & (2 * h - 1)) == 0) {
            const double na = sn[t], nb = sn[t + h];
            if (nb > 0.0) {
                if (na > 0.0) {
                    const double nn = na + nb, d = smu[t + h] - smu[t];
                    smu[t] += d * (nb / nn);
                    sm2[t] += sm2[t + h] + d * d * (na * nb / nn);
                    sn[t] = nn;
                } else {
                    sn[t] = nb;
                    smu[t] = smu[t + h];
                    sm2[t] = sm2[t + h];
                }
            }
        }
        __syncthreads();
    }
    if (t == 0) {
        double var = sn[0] > 0.0 ? sm2[0] / sn[0] : 1.0;
        if (var < 1e-12) var = 1e-12;
        sc->gamma_eps = 1.0 / var;
        sc->ge_set = 1;
    }
}

// Statistics of an arbitrary state (after set_state / set_dictionary): active
// counts per atom and per-chunk sum of s^2.
__global__ void code_stats_kernel(Geom g, const float* W, const uint32_t* Zb, const int* perm, int* m,
                                  double* part_s2)
{
    const long long chunk = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (chunk >= g.NW) return;
    const long long slot = chunk * 32 + lane;
    const long long i = perm ? (long long)perm[slot] : slot;
    double s2 = 0.0;
    for (int k = 0; k < g.K; ++k) {
        const uint32_t zw = Zb[(long long)k * g.NW + chunk];
        if (lane == 0 && zw) atomicAdd(&m[k], __popc(zw));
        if ((zw >> lane) & 1u) {
            const double w = W[wblock(g, k / kAtomBlock, i) + k % kAtomBlock];
            s2 += w * w;
        }
    }
    s2 = warp_sum(s2);
    if (lane == 0) part_s2[chunk] = s2;
}

// The residual of the current state, r = x - D w on every observed pixel,
// written to the per-pixel slots, with the per-chunk squared norm.  It is the
// residual a code sweep starts from: per pixel, the stored weights' products
// are subtracted in atom order, zero weights skipped, each as one fused
// multiply-add -- the arithmetic of the sweep's own rebuild, so both give the
// same bits.  One thread per sweep slot, pixels in chunks of 16; the next
// weight record is loaded behind the current one.
constexpr int kResidChunk = 16;

__global__ void __launch_bounds__(256) residual_kernel(Geom g, const float* x, const uint16_t* obs,
                                                       const uint16_t* nobs, const int* perm, const int* imgoff,
                                                       const float* __restrict__ D, const float* W, const int* pos,
                                                       float* R, double* part_r2)
{
    const long long chunk = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (chunk >= g.NW) return;
    const long long slot = chunk * 32 + lane;   // tables by sweep slot, weights by patch
    double r2 = 0.0;
    if (slot < g.N) {
        const long long i = perm ? (long long)perm[slot] : slot;
        const long long org = patch_origin(g, i);
        const int no = nobs[slot];
        for (int j0 = 0; j0 < no; j0 += kResidChunk) {
            const int nj = no - j0 < kResidChunk ? no - j0 : kResidChunk;
            int pj[kResidChunk];
            float r[kResidChunk];
#pragma unroll
            for (int u = 0; u < kResidChunk; ++u) {
                pj[u] = 0;
                r[u] = 0.0f;
                if (u < nj) {
                    pj[u] = obs[(long long)(j0 + u) * g.N + slot];
                    r[u] = x[org + imgoff[pj[u]]];
                }
            }
            W8 nb = load_w8(W + wblock(g, 0, i));
            for (int kb = 0; kb < g.KB; ++kb) {
                const W8 wb = nb;
                if (kb + 1 < g.KB) nb = load_w8(W + wblock(g, kb + 1, i));
#pragma unroll
                for (int kk = 0; kk < kAtomBlock; ++kk) {
                    const float w = wb.v[kk];
                    if (w != 0.0f) {
                        const float* dk = D + (long long)(kb * kAtomBlock + kk) * g.P;
#pragma unroll
                        for (int u = 0; u < kResidChunk; ++u)
                            if (u < nj) r[u] = fmaf(__ldg(dk + pj[u]), -w, r[u]);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < kResidChunk; ++u) {
                if (u < nj) {
                    R[pos[(long long)(j0 + u) * g.N + slot]] = r[u];
                    r2 += (double)r[u] * r[u];
                }
            }
        }
    }
    r2 = warp_sum(r2);
    if (lane == 0) part_r2[chunk] = r2;
}

}  // namespace sensai

namespace sensai {

static inline unsigned int blocks_for(long long n, int threads)
{
    return (unsigned int)((n + threads - 1) / threads);
}

cudaError_t launch_init_state(const Geom& g, float* D, double* pi, float* lpi, DevScalars* sc,
                              unsigned long long seed, cudaStream_t s)
{
    init_dictionary_kernel<<<blocks_for((long long)g.K * g.P, 256), 256, 0, s>>>(g, D, seed);
    init_scalars_kernel<<<1, 256, 0, s>>>(g.K, pi, lpi, sc);
    return cudaGetLastError();
}

cudaError_t launch_init_gamma_eps(const Geom& g, const float* x, const uint32_t* mbits, DevScalars* sc,
                                  double* scratch, cudaStream_t s)
{
    gamma_eps_parts_kernel<<<kGeParts, 256, 0, s>>>(g.nframe, x, mbits, scratch);
    gamma_eps_merge_kernel<<<1, kGeParts, 0, s>>>(scratch, kGeParts, sc);
    return cudaGetLastError();
}

cudaError_t launch_code_stats(const Geom& g, const float* W, const uint32_t* Zb, const int* perm, int* m,
                              double* part_s2, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(m, 0, sizeof(int) * g.K, s);
    if (e != cudaSuccess) return e;
    code_stats_kernel<<<blocks_for(g.NW, 8), 256, 0, s>>>(g, W, Zb, perm, m, part_s2);
    return cudaGetLastError();
}

cudaError_t launch_residual(const Geom& g, const float* x, const uint16_t* obs, const uint16_t* nobs,
                            const int* perm, const int* imgoff, const float* D, const float* W, const int* pos,
                            float* R, double* part_r2, cudaStream_t s)
{
    residual_kernel<<<blocks_for(g.NW, 8), 256, 0, s>>>(g, x, obs, nobs, perm, imgoff, D, W, pos, R, part_r2);
    return cudaGetLastError();
}

// Patch-major (Z bytes, S floats) <-> device layout (Zb bits [K][NW] by sweep
// slot, slot s holding patch perm[s]; W [KB][Npad][8] by patch).
__global__ void export_codes_kernel(Geom g, const float* W, const uint32_t* Zb, const int* perm, uint8_t* Z,
                                    float* S)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= g.N * g.K) return;
    const long long slot = idx / g.K;
    const int k = (int)(idx % g.K);
    const long long i = perm ? (long long)perm[slot] : slot;
    const bool z = (Zb[(long long)k * g.NW + (slot >> 5)] >> (slot & 31)) & 1u;
    Z[i * g.K + k] = z ? 1 : 0;
    S[i * g.K + k] = z ? W[wblock(g, k / kAtomBlock, i) + k % kAtomBlock] : 0.0f;
}

// One thread per (atom, 32-slot word).
__global__ void import_codes_kernel(Geom g, const uint8_t* Z, const float* S, const int* perm, float* W,
                                    uint32_t* Zb)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)g.K * g.NW) return;
    const int k = (int)(idx / g.NW);
    const long long w = idx % g.NW;
    uint32_t bits = 0;
    for (int b = 0; b < 32; ++b) {
        const long long slot = w * 32 + b;
        if (slot >= g.N) break;
        const long long i = perm ? (long long)perm[slot] : slot;
        const bool z = Z[i * g.K + k] != 0;
        if (z) bits |= 1u << b;
        W[wblock(g, k / kAtomBlock, i) + k % kAtomBlock] = z ? S[i * g.K + k] : 0.0f;
    }
    Zb[idx] = bits;
}

__global__ void logit_kernel(int K, const double* pi, float* lpi)
{
    for (int k = threadIdx.x; k < K; k += blockDim.x) lpi[k] = (float)(log(pi[k]) - log1p(-pi[k]));
}

cudaError_t launch_export_codes(const Geom& g, const float* W, const uint32_t* Zb, const int* perm, uint8_t* Z,
                                float* S, cudaStream_t s)
{
    export_codes_kernel<<<blocks_for(g.N * g.K, 256), 256, 0, s>>>(g, W, Zb, perm, Z, S);
    return cudaGetLastError();
}

cudaError_t launch_import_codes(const Geom& g, const uint8_t* Z, const float* S, const int* perm, float* W,
                                uint32_t* Zb, cudaStream_t s)
{
    import_codes_kernel<<<blocks_for((long long)g.K * g.NW, 256), 256, 0, s>>>(g, Z, S, perm, W, Zb);
    return cudaGetLastError();
}

cudaError_t launch_logit(int K, const double* pi, float* lpi, cudaStream_t s)
{
    logit_kernel<<<1, 256, 0, s>>>(K, pi, lpi);
    return cudaGetLastError();
}

}  // namespace sensai
