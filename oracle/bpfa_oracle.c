/*
 * bpfa_oracle.c -- plain FP64 CPU oracle for BPFA inpainting.
 *
 * TEST INFRASTRUCTURE ONLY (see bpfa_oracle.h).  Written for clarity, not
 * speed: every step follows the model and sampler stated in the header, in
 * the order stated there, with no blocking, fusion or reordering.  The only
 * parallelism is an OpenMP loop over patches in the sparse-code sweep, where
 * patches are conditionally independent given D, pi and the precisions; each
 * patch's draws are keyed by its own Philox counter, so results do not depend
 * on the thread count.
 */
#include "bpfa_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ RNG -- */

/* Philox4x32-10 as defined by Salmon et al. (SC'11): ten rounds of two
 * 32x32->64 multiplies by the round multipliers, the high halves xored with
 * the other counter words and the key, the key bumped by the Weyl constants
 * between rounds. */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t mult0 = 0xD2511F53u, mult1 = 0xCD9E8D57u;
    const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)mult0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)mult1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += weyl0;
        k1 += weyl1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void block_at(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t out[4])
{
    const uint32_t ctr[4] = {c0, c1, c2, c3};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox(ctr, key, out);
}

/* u = (x + 1) / 2^32, in (0, 1]. */
static double unit_uniform(uint32_t x)
{
    return ((double)x + 1.0) * (1.0 / 4294967296.0);
}

/* Box-Muller: sqrt(-2 ln u1) cos(2 pi u2). */
static double box_muller(uint32_t x0, uint32_t x1)
{
    const double two_pi = 6.283185307179586476925286766559;
    double u1 = unit_uniform(x0), u2 = unit_uniform(x1);
    return sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
}

/* The two normals of one Box-Muller transform, sqrt(-2 ln u1) cos(2 pi u2)
 * and sqrt(-2 ln u1) sin(2 pi u2): independent standard normals.  second
 * selects the sine. */
static double box_muller_pair(uint32_t x0, uint32_t x1, int second)
{
    const double two_pi = 6.283185307179586476925286766559;
    double u1 = unit_uniform(x0), u2 = unit_uniform(x1);
    double rad = sqrt(-2.0 * log(u1));
    return second ? rad * sin(two_pi * u2) : rad * cos(two_pi * u2);
}

double orc_normal_pair(uint64_t seed, const uint32_t ctr[4], int second)
{
    uint32_t blk[4];
    block_at(seed, ctr[0], ctr[1], ctr[2], ctr[3], blk);
    return box_muller_pair(blk[2], blk[3], second);
}

double orc_normal(uint64_t seed, const uint32_t ctr[4])
{
    uint32_t blk[4];
    block_at(seed, ctr[0], ctr[1], ctr[2], ctr[3], blk);
    return box_muller(blk[0], blk[1]);
}

#define ORC_GAMMA_MAX_ATTEMPTS 64

/* Marsaglia & Tsang (2000), shape >= 1.  Attempt a uses the block at counter
 * (c0, c1, t, tag | a << 8): words 0-1 give the normal, word 2 the uniform of
 * the acceptance test. */
static double gamma_ge1(double shape, uint64_t seed, uint32_t c0, uint32_t c1, uint32_t t, uint32_t tag)
{
    const double dd = shape - 1.0 / 3.0;
    const double cc = 1.0 / sqrt(9.0 * dd);
    for (uint32_t attempt = 0; attempt < ORC_GAMMA_MAX_ATTEMPTS; ++attempt) {
        uint32_t blk[4];
        block_at(seed, c0, c1, t, tag | (attempt << 8), blk);
        double xn = box_muller(blk[0], blk[1]);
        double v = 1.0 + cc * xn;
        if (v <= 0.0) continue;
        v = v * v * v;
        double u = unit_uniform(blk[2]);
        if (u < 1.0 - 0.0331 * xn * xn * xn * xn) return dd * v;
        if (log(u) < 0.5 * xn * xn + dd * (1.0 - v + log(v))) return dd * v;
    }
    return dd; /* not reached in practice: each attempt accepts with p > 0.95 */
}

/* Gamma(shape, 1); shape < 1 uses Gamma(shape + 1) * U^(1/shape), with U from
 * word 3 of the attempt-0 block. */
double orc_gamma(double shape, uint64_t seed, uint32_t c0, uint32_t c1, uint32_t t, uint32_t tag)
{
    if (shape >= 1.0) return gamma_ge1(shape, seed, c0, c1, t, tag);
    double g = gamma_ge1(shape + 1.0, seed, c0, c1, t, tag);
    uint32_t blk[4];
    block_at(seed, c0, c1, t, tag, blk);
    double u = unit_uniform(blk[3]);
    return g * pow(u, 1.0 / shape);
}

double orc_beta(double alpha, double beta, uint64_t seed, uint32_t c0, uint32_t t)
{
    double g1 = orc_gamma(alpha, seed, c0, 0, t, ORC_TAG_PI_A);
    double g2 = orc_gamma(beta, seed, c0, 0, t, ORC_TAG_PI_B);
    return g1 / (g1 + g2);
}

/* ------------------------------------------------------------- geometry -- */

int orc_check(const orc_params* prm)
{
    if (prm->ndim < 1 || prm->ndim > 4) return -1;
    if (prm->K < 1) return -2;
    for (int dd = 0; dd < prm->ndim; ++dd) {
        if (prm->B[dd] < 1 || prm->B[dd] > prm->M[dd]) return -3;
        if (prm->S[dd] < 1) return -4;
        if ((prm->M[dd] - prm->B[dd]) % prm->S[dd] != 0) return -5;
    }
    return 0;
}

static int64_t grid_extent(const orc_params* prm, int dd)
{
    return (prm->M[dd] - prm->B[dd]) / prm->S[dd] + 1;
}

int64_t orc_num_patches(const orc_params* prm)
{
    int64_t n = 1;
    for (int dd = 0; dd < prm->ndim; ++dd) n *= grid_extent(prm, dd);
    return n;
}

int64_t orc_patch_size(const orc_params* prm)
{
    int64_t n = 1;
    for (int dd = 0; dd < prm->ndim; ++dd) n *= prm->B[dd];
    return n;
}

int64_t orc_frame_size(const orc_params* prm)
{
    int64_t n = 1;
    for (int dd = 0; dd < prm->ndim; ++dd) n *= prm->M[dd];
    return n;
}

/* Row-major strides of the frame. */
static void frame_strides(const orc_params* prm, int64_t stride[4])
{
    int64_t s = 1;
    for (int dd = prm->ndim - 1; dd >= 0; --dd) {
        stride[dd] = s;
        s *= prm->M[dd];
    }
}

void orc_patch_origins(const orc_params* prm, int64_t* origin)
{
    int64_t fs[4];
    frame_strides(prm, fs);
    const int64_t n = orc_num_patches(prm);
    for (int64_t i = 0; i < n; ++i) {
        int64_t rem = i, off = 0;
        for (int dd = prm->ndim - 1; dd >= 0; --dd) {
            int64_t g = grid_extent(prm, dd);
            int64_t id = rem % g;
            rem /= g;
            off += id * prm->S[dd] * fs[dd];
        }
        origin[i] = off;
    }
}

void orc_pixel_offsets(const orc_params* prm, int64_t* offset)
{
    int64_t fs[4];
    frame_strides(prm, fs);
    const int64_t P = orc_patch_size(prm);
    for (int64_t p = 0; p < P; ++p) {
        int64_t rem = p, off = 0;
        for (int dd = prm->ndim - 1; dd >= 0; --dd) {
            int64_t q = rem % prm->B[dd];
            rem /= prm->B[dd];
            off += q * fs[dd];
        }
        offset[p] = off;
    }
}

/* Per dimension, the patch starts covering coordinate y are the multiples of
 * S in [max(0, y - B + 1), min(y, (G - 1) S)]; the count is the product over
 * dimensions of floor(hi / S) - ceil(lo / S) + 1. */
void orc_overlap_counts(const orc_params* prm, int32_t* counts)
{
    int64_t fs[4];
    frame_strides(prm, fs);
    const int64_t nf = orc_frame_size(prm);
    for (int64_t u = 0; u < nf; ++u) {
        int64_t rem = u, c = 1;
        for (int dd = prm->ndim - 1; dd >= 0; --dd) {
            int64_t y = rem % prm->M[dd];
            rem /= prm->M[dd];
            int64_t last = (grid_extent(prm, dd) - 1) * prm->S[dd];
            int64_t lo = y - prm->B[dd] + 1;
            if (lo < 0) lo = 0;
            int64_t hi = y < last ? y : last;
            int64_t first_idx = (lo + prm->S[dd] - 1) / prm->S[dd];
            int64_t last_idx = hi / prm->S[dd];
            int64_t nd = last_idx - first_idx + 1;
            c *= nd > 0 ? nd : 0;
        }
        counts[u] = (int32_t)c;
    }
}

/* ----------------------------------------------------------- model steps -- */

void orc_init_dictionary(const orc_params* prm, double* D)
{
    const int64_t P = orc_patch_size(prm);
    const double sd = 1.0 / sqrt((double)P);
    for (int k = 0; k < prm->K; ++k)
        for (int64_t p = 0; p < P; ++p) {
            uint32_t ctr[4] = {(uint32_t)p, (uint32_t)k, 0u, ORC_TAG_INIT};
            D[(int64_t)k * P + p] = sd * orc_normal(prm->seed, ctr);
        }
}

double orc_init_gamma_eps(const orc_params* prm, const float* x, const uint8_t* mask)
{
    const int64_t nf = orc_frame_size(prm);
    double sum = 0.0, sum2 = 0.0;
    int64_t n = 0;
    for (int64_t u = 0; u < nf; ++u)
        if (mask[u]) {
            sum += x[u];
            ++n;
        }
    if (n == 0) return 1.0;
    double mean = sum / (double)n;
    for (int64_t u = 0; u < nf; ++u)
        if (mask[u]) sum2 += ((double)x[u] - mean) * ((double)x[u] - mean);
    double var = sum2 / (double)n;
    if (var < 1e-12) var = 1e-12;
    return 1.0 / var;
}

/* Observed within-patch pixels of patch i: their indices p and frame values. */
static int64_t observed_list(const int64_t* origin, const int64_t* offset, int64_t P,
                             int64_t i, const float* x, const uint8_t* mask,
                             int64_t* plist, double* xlist)
{
    int64_t nobs = 0;
    for (int64_t p = 0; p < P; ++p) {
        int64_t u = origin[i] + offset[p];
        if (mask[u]) {
            plist[nobs] = p;
            xlist[nobs] = x[u];
            ++nobs;
        }
    }
    return nobs;
}

void orc_zs_sweep(const orc_params* prm, const float* x, const uint8_t* mask,
                  const double* D, uint8_t* Z, double* S, const double* pi,
                  double gamma_s, double gamma_eps, int64_t t, double* stats)
{
    orc_zs_sweep_subset(prm, x, mask, D, Z, S, pi, gamma_s, gamma_eps, t, NULL, -1, NULL, stats);
}

void orc_zs_sweep_subset(const orc_params* prm, const float* x, const uint8_t* mask,
                         const double* D, uint8_t* Z, double* S, const double* pi,
                         double gamma_s, double gamma_eps, int64_t t,
                         const int64_t* patches, int64_t npatches, double* logodds, double* stats)
{
    const int64_t N = orc_num_patches(prm), P = orc_patch_size(prm);
    const int K = prm->K;
    int64_t* origin = malloc(sizeof(int64_t) * N);
    int64_t* offset = malloc(sizeof(int64_t) * P);
    double* patch_z = calloc(N, sizeof(double));
    double* patch_s2 = calloc(N, sizeof(double));
    double* patch_r2 = calloc(N, sizeof(double));
    double* logit_pi = malloc(sizeof(double) * K);
    orc_patch_origins(prm, origin);
    orc_pixel_offsets(prm, offset);
    for (int k = 0; k < K; ++k) logit_pi[k] = log(pi[k]) - log1p(-pi[k]);
    const double half_log_gs = 0.5 * log(gamma_s);

#pragma omp parallel
    {
        int64_t* plist = malloc(sizeof(int64_t) * P);
        double* xlist = malloc(sizeof(double) * P);
        double* r = malloc(sizeof(double) * P);
const int64_t nvisit = patches ? npatches : N;
#pragma omp for schedule(static)
        for (int64_t v = 0; v < nvisit; ++v) {
            const int64_t i = patches ? patches[v] : v;
            int64_t nobs = observed_list(origin, offset, P, i, x, mask, plist, xlist);
            /* residual on the observed pixels: r = x - D w_i */
            for (int64_t j = 0; j < nobs; ++j) {
                double acc = xlist[j];
                for (int k = 0; k < K; ++k)
                    if (Z[i * K + k]) acc -= D[(int64_t)k * P + plist[j]] * S[i * K + k];
                r[j] = acc;
            }
            double zc = 0.0, s2 = 0.0;
            for (int k = 0; k < K; ++k) {
                const double* dk = D + (int64_t)k * P;
                double n = 0.0, h = 0.0;
                for (int64_t j = 0; j < nobs; ++j) {
                    n += dk[plist[j]] * dk[plist[j]];
                    h += dk[plist[j]] * r[j];
                }
                double w_old = Z[i * K + k] ? S[i * K + k] : 0.0;
                /* correlation of atom k with the residual that excludes it */
                double g = h + w_old * n;
                double lam = gamma_s + gamma_eps * n;
                /* log odds of z = 1 with s integrated out */
                double L = logit_pi[k] + half_log_gs - 0.5 * log(lam)
                         + gamma_eps * gamma_eps * g * g / (2.0 * lam);
                if (logodds) logodds[i * K + k] = L;
                double sig = 1.0 / (1.0 + exp(-L));
                uint64_t thr = (uint64_t)floor(sig * 4294967296.0);
                /* atoms 2m and 2m + 1 share the block at counter (i, m, t):
                 * word k % 2 decides z, words 2-3 give the Box-Muller pair
                 * (the cosine for the even atom, the sine for the odd one) */
                uint32_t blk[4];
                block_at(prm->seed, (uint32_t)i, (uint32_t)(k >> 1), (uint32_t)t, ORC_TAG_ZS, blk);
                int z = (uint64_t)blk[k & 1] < thr;
                const double nrm = box_muller_pair(blk[2], blk[3], k & 1);
                double w_new = 0.0, s_new = 0.0;
                if (z) {
                    w_new = gamma_eps * g / lam + nrm / sqrt(lam);
                    s_new = w_new;
                    zc += 1.0;
                    s2 += w_new * w_new;
                } else if (prm->flags & ORC_FLAG_GAMMA_S_FULL) {
                    /* inactive: s from its prior; the weight z s stays 0 */
                    s_new = nrm / sqrt(gamma_s);
                    s2 += s_new * s_new;
                }
                double dw = w_new - w_old;
                if (dw != 0.0)
                    for (int64_t j = 0; j < nobs; ++j) r[j] -= dk[plist[j]] * dw;
                Z[i * K + k] = (uint8_t)z;
                S[i * K + k] = s_new;
            }
            double r2 = 0.0;
            for (int64_t j = 0; j < nobs; ++j) r2 += r[j] * r[j];
            patch_z[i] = zc;
            patch_s2[i] = s2;
            patch_r2[i] = r2;
        }
        free(plist);
        free(xlist);
        free(r);
    }
    if (stats) {
        double a = 0.0, b = 0.0, c = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            a += patch_z[i];
            b += patch_s2[i];
            c += patch_r2[i];
        }
        stats[0] = a;
        stats[1] = b;
        stats[2] = c;
    }
    free(origin);
    free(offset);
    free(patch_z);
    free(patch_s2);
    free(patch_r2);
    free(logit_pi);
}

void orc_d_sweep(const orc_params* prm, const float* x, const uint8_t* mask,
                 double* D, const uint8_t* Z, const double* S, double gamma_eps, int64_t t)
{
    const int64_t N = orc_num_patches(prm), P = orc_patch_size(prm);
    const int K = prm->K;
    int64_t* origin = malloc(sizeof(int64_t) * N);
    int64_t* offset = malloc(sizeof(int64_t) * P);
    double* r = malloc(sizeof(double) * N * P);   /* residual, 0 where unobserved */
    double* num = malloc(sizeof(double) * P);
    double* den = malloc(sizeof(double) * P);
    double* delta = malloc(sizeof(double) * P);
    orc_patch_origins(prm, origin);
    orc_pixel_offsets(prm, offset);
    for (int64_t i = 0; i < N; ++i)
        for (int64_t p = 0; p < P; ++p) {
            int64_t u = origin[i] + offset[p];
            double acc = 0.0;
            if (mask[u]) {
                acc = x[u];
                for (int k = 0; k < K; ++k)
                    if (Z[i * K + k]) acc -= D[(int64_t)k * P + p] * S[i * K + k];
            }
            r[i * P + p] = acc;
        }
    for (int k = 0; k < K; ++k) {
        double* dk = D + (int64_t)k * P;
        for (int64_t p = 0; p < P; ++p) num[p] = den[p] = 0.0;
        /* posterior sums over the patches that use atom k, on observed pixels,
         * with the residual that excludes atom k */
        for (int64_t i = 0; i < N; ++i) {
            if (!Z[i * K + k]) continue;
            double w = S[i * K + k];
            for (int64_t p = 0; p < P; ++p) {
                if (!mask[origin[i] + offset[p]]) continue;
                num[p] += w * (r[i * P + p] + dk[p] * w);
                den[p] += w * w;
            }
        }
        for (int64_t p = 0; p < P; ++p) {
            double prec = (double)P + gamma_eps * den[p];
            double mean = gamma_eps * num[p] / prec;
            uint32_t ctr[4] = {(uint32_t)p, (uint32_t)k, (uint32_t)t, ORC_TAG_D};
            double dnew = mean + orc_normal(prm->seed, ctr) / sqrt(prec);
            delta[p] = dnew - dk[p];
            dk[p] = dnew;
        }
        for (int64_t i = 0; i < N; ++i) {
            if (!Z[i * K + k]) continue;
            double w = S[i * K + k];
            for (int64_t p = 0; p < P; ++p)
                if (mask[origin[i] + offset[p]]) r[i * P + p] -= delta[p] * w;
        }
    }
    free(origin);
    free(offset);
    free(r);
    free(num);
    free(den);
    free(delta);
}

void orc_hyper(const orc_params* prm, const float* x, const uint8_t* mask,
               const double* D, const uint8_t* Z, const double* S,
               double* pi, double* gamma_s, double* gamma_eps, int64_t t, double* stats)
{
    const int64_t N = orc_num_patches(prm), P = orc_patch_size(prm);
    const int K = prm->K;
    int64_t* origin = malloc(sizeof(int64_t) * N);
    int64_t* offset = malloc(sizeof(int64_t) * P);
    orc_patch_origins(prm, origin);
    orc_pixel_offsets(prm, offset);

    const int full_s = (prm->flags & ORC_FLAG_GAMMA_S_FULL) != 0;
    double z_total = 0.0, s2_total = 0.0;
    for (int k = 0; k < K; ++k) {
        double m = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            if (Z[i * K + k]) m += 1.0;
            if (Z[i * K + k] || full_s) s2_total += S[i * K + k] * S[i * K + k];
        }
        z_total += m;
        double alpha = prm->a / K + m;
        double beta = prm->b * (K - 1) / K + (double)N - m;
        pi[k] = orc_beta(alpha, beta, prm->seed, (uint32_t)k, (uint32_t)t);
    }

    double r2_total = 0.0, obs_total = 0.0;
    for (int64_t i = 0; i < N; ++i)
        for (int64_t p = 0; p < P; ++p) {
            int64_t u = origin[i] + offset[p];
            if (!mask[u]) continue;
            double acc = x[u];
            for (int k = 0; k < K; ++k)
                if (Z[i * K + k]) acc -= D[(int64_t)k * P + p] * S[i * K + k];
            r2_total += acc * acc;
            obs_total += 1.0;
        }

    const double s_count = full_s ? (double)N * K : z_total;   /* entries whose s enters the sum */
    *gamma_s = orc_gamma(prm->c + 0.5 * s_count, prm->seed, 0, 0, (uint32_t)t, ORC_TAG_GS)
             / (prm->d + 0.5 * s2_total);
    *gamma_eps = orc_gamma(prm->e + 0.5 * obs_total, prm->seed, 0, 0, (uint32_t)t, ORC_TAG_GE)
               / (prm->f + 0.5 * r2_total);
    if (stats) {
        stats[0] = z_total;
        stats[1] = s2_total;
        stats[2] = r2_total;
        stats[3] = obs_total;
    }
    free(origin);
    free(offset);
}

void orc_reconstruct(const orc_params* prm, const double* D, const uint8_t* Z,
                     const double* S, double* out)
{
    const int64_t N = orc_num_patches(prm), P = orc_patch_size(prm);
    const int64_t nf = orc_frame_size(prm);
    const int K = prm->K;
    int64_t* origin = malloc(sizeof(int64_t) * N);
    int64_t* offset = malloc(sizeof(int64_t) * P);
    int32_t* counts = malloc(sizeof(int32_t) * nf);
    orc_patch_origins(prm, origin);
    orc_pixel_offsets(prm, offset);
    orc_overlap_counts(prm, counts);
    for (int64_t u = 0; u < nf; ++u) out[u] = 0.0;
    for (int64_t i = 0; i < N; ++i)
        for (int64_t p = 0; p < P; ++p) {
            double v = 0.0;
            for (int k = 0; k < K; ++k)
                if (Z[i * K + k]) v += D[(int64_t)k * P + p] * S[i * K + k];
            out[origin[i] + offset[p]] += v;
        }
    for (int64_t u = 0; u < nf; ++u) out[u] = counts[u] > 0 ? out[u] / counts[u] : 0.0;
    free(origin);
    free(offset);
    free(counts);
}

/* Posterior-mean reconstruction over T samples of the chain: the mean of the
 * T overlap-add reconstructions, sample t given by D + t K P, Z + t N K and
 * S + t N K. */
void orc_reconstruct_mean(const orc_params* prm, int T, const double* D, const uint8_t* Z, const double* S,
                          double* out)
{
    const int64_t N = orc_num_patches(prm), P = orc_patch_size(prm);
    const int64_t nf = orc_frame_size(prm);
    const int64_t K = prm->K;
    double* one = malloc(sizeof(double) * nf);
    for (int64_t u = 0; u < nf; ++u) out[u] = 0.0;
    for (int t = 0; t < T; ++t) {
        orc_reconstruct(prm, D + (int64_t)t * K * P, Z + (int64_t)t * N * K, S + (int64_t)t * N * K, one);
        for (int64_t u = 0; u < nf; ++u) out[u] += one[u];
    }
    for (int64_t u = 0; u < nf; ++u) out[u] = T > 0 ? out[u] / T : 0.0;
    free(one);
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
