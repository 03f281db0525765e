/*
 * bpfa_oracle.h -- plain FP64 CPU oracle for Beta-Process Factor Analysis
 * (BPFA) inpainting.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path; the two agree only
 * through the published definitions they both implement.
 *
 * What it computes.  The paper ("Beta-Process Factor Analysis (BPFA)"
 * section) uses BPFA as its inpainting model and defers its definition to the
 * cited nonparametric factor-analysis / dictionary-learning papers (Paisley &
 * Carin 2009; Zhou et al. 2009).  Each iteration performs a sparse-coding
 * step and a dictionary-learning step on all overlapping N-D patches of a
 * subsampled frame ("N-Dimensional Inpainting" section).  The model, written
 * out from those references, is
 *
 *   x_i  = D (z_i o s_i) + eps_i        observed on the patch mask Omega_i
 *   d_k  ~ N(0, I_P / P)                s_ik ~ N(0, 1/gamma_s)
 *   z_ik ~ Bernoulli(pi_k)              pi_k ~ Beta(a/K, b(K-1)/K)
 *   gamma_s ~ Gamma(c, d)               gamma_eps ~ Gamma(e, f)   (shape, rate)
 *   eps_i ~ N(0, I / gamma_eps)
 *
 * and the Gibbs sampler visits, per iteration t:
 *   1. the sparse codes, patch by patch (independent given D), atoms in
 *      order k = 0..K-1, drawing z_ik with s_ik integrated out and then
 *      s_ik | z_ik = 1 (inactive weights are never stored);
 *   2. the dictionary, atom by atom in order, each d_kp from its conjugate
 *      Gaussian given every other atom's current value;
 *   3. pi_k, gamma_s, gamma_eps from their conjugate Beta / Gamma posteriors.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) keyed by
 * the 64-bit seed, with counter (c0, c1, c2, c3) = (index0, index1,
 * iteration, tag | attempt << 8).  Uniforms u = (x + 1) 2^-32 in (0, 1];
 * normals by Box-Muller (1958) from the first two words of a block; Gamma by
 * Marsaglia & Tsang (2000) with the U^(1/alpha) boost for shape < 1; Beta as
 * G1 / (G1 + G2).
 *
 * Layouts: frames and masks are row-major over M (last dimension fastest);
 * patches are numbered row-major over the patch-start grid, pixels within a
 * patch row-major over B.  D is K x P, Z (uint8) and S are N x K, pi has K
 * entries.  All arrays are caller-owned.
 */
#ifndef BPFA_ORACLE_H
#define BPFA_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t ndim;      /* 1..4 */
    int64_t M[4];      /* frame shape */
    int32_t B[4];      /* patch shape */
    int32_t S[4];      /* patch stride */
    int32_t K;         /* number of atoms */
    double a, b;       /* pi_k ~ Beta(a/K, b(K-1)/K) */
    double c, d;       /* gamma_s ~ Gamma(c, d), shape / rate */
    double e, f;       /* gamma_eps ~ Gamma(e, f), shape / rate */
    uint64_t seed;     /* Philox key */
    int32_t flags;     /* ORC_FLAG_* */
} orc_params;

/* Reading of the gamma_s update.  Default: the weights of inactive atoms are
 * integrated out, and gamma_s ~ Ga(c + sum z / 2, d + sum_{z=1} s^2 / 2).
 * ORC_FLAG_GAMMA_S_FULL: the sweep also draws s_ik ~ N(0, 1/gamma_s) for
 * every inactive entry (from the same Philox words a z = 1 entry uses for its
 * normal) and stores it in S; then gamma_s ~ Ga(c + N K / 2,
 * d + sum_all s^2 / 2).  Both are valid samplers of the same posterior; z
 * and the active s are the same under both for the same counters. */
enum { ORC_FLAG_GAMMA_S_FULL = 4 };

enum {
    ORC_TAG_INIT = 1,  /* dictionary initialisation, counter (p, k, 0) */
    ORC_TAG_ZS = 2,    /* sparse-code draws of atoms 2m, 2m + 1, counter (i, m, t): word k % 2 -> z_ik,
                          words 2-3 -> one Box-Muller pair (cosine: even atom, sine: odd atom) */
    ORC_TAG_D = 3,     /* dictionary draw, counter (p, k, t) */
    ORC_TAG_PI_A = 4,  /* first Gamma of the Beta draw of pi_k, counter (k, 0, t) */
    ORC_TAG_PI_B = 5,  /* second Gamma of the Beta draw of pi_k */
    ORC_TAG_GS = 6,    /* gamma_s draw, counter (0, 0, t) */
    ORC_TAG_GE = 7     /* gamma_eps draw, counter (0, 0, t) */
};

/* 0 when the geometry is valid (1 <= ndim <= 4, 1 <= B_d <= M_d, S_d >= 1,
 * (M_d - B_d) divisible by S_d, K >= 1), else a negative code. */
int orc_check(const orc_params* prm);
int64_t orc_num_patches(const orc_params* prm);
int64_t orc_patch_size(const orc_params* prm);
int64_t orc_frame_size(const orc_params* prm);

/* One Philox4x32-10 block. */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* Standard normal from the block at counter ctr (words 0 and 1). */
double orc_normal(uint64_t seed, const uint32_t ctr[4]);
/* One of the two normals of the Box-Muller transform of words 2 and 3 of the
 * block at counter ctr: the cosine one (second = 0) or the sine one; the pair
 * the code draws of atoms 2m and 2m + 1 use. */
double orc_normal_pair(uint64_t seed, const uint32_t ctr[4], int second);
/* Gamma(shape, 1) and Beta(alpha, beta) with the counter conventions above;
 * c0 is the index word, tag the stream tag (attempts go in tag's high bits). */
double orc_gamma(double shape, uint64_t seed, uint32_t c0, uint32_t c1, uint32_t t, uint32_t tag);
double orc_beta(double alpha, double beta, uint64_t seed, uint32_t c0, uint32_t t);

/* Number of patches covering each frame pixel (closed form per dimension). */
void orc_overlap_counts(const orc_params* prm, int32_t* counts);
/* Frame index of every patch's first pixel (N entries) and the frame offset
 * of every within-patch pixel (P entries). */
void orc_patch_origins(const orc_params* prm, int64_t* origin);
void orc_pixel_offsets(const orc_params* prm, int64_t* offset);

/* Initial dictionary: d_kp ~ N(0, 1/P) from counter (p, k, 0, INIT). */
void orc_init_dictionary(const orc_params* prm, double* D);
/* Initial noise precision: 1 / max(var(x over observed pixels), 1e-12). */
double orc_init_gamma_eps(const orc_params* prm, const float* x, const uint8_t* mask);

/* Sparse-code sweep at iteration t.  Updates Z and S in place.  stats (may be
 * NULL) receives {sum z, sum of s^2 over active entries (over all entries
 * with ORC_FLAG_GAMMA_S_FULL), sum over patches of the squared residual on
 * observed pixels after the sweep}. */
void orc_zs_sweep(const orc_params* prm, const float* x, const uint8_t* mask,
                  const double* D, uint8_t* Z, double* S, const double* pi,
                  double gamma_s, double gamma_eps, int64_t t, double* stats);

/* The same sweep restricted to the listed patches (patches are independent
 * given D, pi and the precisions, and each keeps its own Philox counters), and
 * optionally recording the log odds L of every visited draw in logodds
 * (N x K, may be NULL).  patches == NULL visits all of them.  Test
 * instrumentation: the arithmetic is that of orc_zs_sweep. */
void orc_zs_sweep_subset(const orc_params* prm, const float* x, const uint8_t* mask,
                         const double* D, uint8_t* Z, double* S, const double* pi,
                         double gamma_s, double gamma_eps, int64_t t,
                         const int64_t* patches, int64_t npatches, double* logodds, double* stats);

/* Dictionary sweep at iteration t, atoms in order.  Updates D in place. */
void orc_d_sweep(const orc_params* prm, const float* x, const uint8_t* mask,
                 double* D, const uint8_t* Z, const double* S, double gamma_eps, int64_t t);

/* pi, gamma_s and gamma_eps draws at iteration t from the current state.
 * stats (may be NULL) receives {sum z, sum s^2 (active entries; all entries
 * with ORC_FLAG_GAMMA_S_FULL), sum r^2, sum |Omega_i|}. */
void orc_hyper(const orc_params* prm, const float* x, const uint8_t* mask,
               const double* D, const uint8_t* Z, const double* S,
               double* pi, double* gamma_s, double* gamma_eps, int64_t t, double* stats);

/* Overlap-add reconstruction: mean over covering patches of (D w_i). */
void orc_reconstruct(const orc_params* prm, const double* D, const uint8_t* Z,
                     const double* S, double* out);

/* Posterior-mean reconstruction over the last T samples of a chain: the mean
 * of the T overlap-add reconstructions (samples stacked: D is T x K x P, Z and
 * S are T x N x K). */
void orc_reconstruct_mean(const orc_params* prm, int T, const double* D, const uint8_t* Z, const double* S,
                          double* out);

/* Number of OpenMP threads the sweeps use. */
int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
