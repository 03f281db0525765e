/*
 * sensai.h -- C ABI of the GB300 (sm_103a) BPFA inpainting library.
 *
 * The library runs the Gibbs sampler of Beta-Process Factor Analysis (BPFA),
 * the model the paper's "Beta-Process Factor Analysis (BPFA)" section uses for
 * joint dictionary learning and sparse coding, over every overlapping N-D
 * patch of a subsampled frame ("N-Dimensional Inpainting" section), with all
 * arithmetic in hand-written CUDA kernels on one GPU.
 *
 * Model (from the nonparametric factor-analysis papers the BPFA section
 * cites): patch i of P pixels, observed on its mask Omega_i,
 *   x_i = D (z_i o s_i) + eps_i,  d_k ~ N(0, I/P),  s_ik ~ N(0, 1/gamma_s),
 *   z_ik ~ Bernoulli(pi_k),  pi_k ~ Beta(a/K, b(K-1)/K),
 *   gamma_s ~ Gamma(c, d),  gamma_eps ~ Gamma(e, f)  (shape, rate),
 *   eps_i ~ N(0, I/gamma_eps).
 * One iteration t: (1) sparse-code sweep, patches in parallel, atoms
 * k = 0..K-1 in order, z_ik drawn with s_ik integrated out, then s_ik | z=1;
 * (2) dictionary sweep, atoms in order, d_kp from its conjugate Gaussian;
 * (3) pi_k, gamma_s, gamma_eps from their conjugate Beta / Gamma laws.
 * Inactive weights are not stored (w_ik = z_ik s_ik, zero when z_ik = 0).
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11) keyed by `seed`,
 * counter (index0, index1, t, tag | attempt << 8); uniforms (x + 1) 2^-32;
 * Box-Muller normals; Marsaglia-Tsang Gamma.  The code draws of atoms 2m and
 * 2m + 1 of patch i share the block at (i, m, t, 2): word k % 2 decides
 * z_ik, words 2-3 give one Box-Muller pair (cosine: even atom, sine: odd).  Results depend only on the
 * parameters, seed, frame, mask and iteration index.
 *
 * Conventions for every entry point:
 *  - Frames, masks and outputs are row-major over M (last dimension fastest).
 *    Patches are numbered row-major over the grid of patch starts; pixels in
 *    a patch row-major over B.  D is K x P row-major.
 *  - Pointers documented "host or device" are classified with
 *    cudaPointerGetAttributes; device pointers must be on the context's GPU.
 *    The caller owns every buffer it passes and keeps it valid until the call
 *    returns; calls that read or write host memory synchronise `stream`
 *    before returning.  Calls that only touch device memory are asynchronous
 *    on `stream` (a cudaStream_t; NULL is the legacy default stream).
 *  - Errors are returned, never raised: SENSAI_EINVAL for bad arguments
 *    (nothing is changed), SENSAI_ENOMEM when device memory runs out,
 *    SENSAI_ECUDA for a CUDA error, SENSAI_ESTATE when the context is unusable
 *    (after a sticky CUDA error, or a frame is needed and none was given).
 *    sensai_last_error() returns a message for the calling thread.
 *  - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef SENSAI_H
#define SENSAI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sensai_ctx sensai_ctx;

typedef enum {
    SENSAI_OK = 0,
    SENSAI_EINVAL = 1,
    SENSAI_ENOMEM = 2,
    SENSAI_ECUDA = 3,
    SENSAI_ETIMEOUT = 4,
    SENSAI_EBUSY = 5,
    SENSAI_ESTATE = 6
} sensai_status;

/* Problem definition.  Requirements: 1 <= ndim <= 4; 1 <= B[d] <= M[d];
 * stride[d] >= 1 with (M[d] - B[d]) divisible by stride[d]; 1 <= K <= 1024;
 * P = prod(B) <= 1024; number of patches < 2^31; at most 256 observed pixels
 * in any patch (above 96 a patch's pixels are split over a lane pair).  a <= 0 selects a = K and
 * b <= 0 selects b = N / 8 (N = number of patches).  c..f > 0.  flags:
 * SENSAI_FLAG_CHAIN_DICTIONARY, SENSAI_FLAG_STREAM_DICTIONARY, and with the
 * latter SENSAI_SLICE_ATOMS(n), SENSAI_FLAG_GAMMA_S_FULL,
 * SENSAI_FLAG_DENSE_STATISTICS, SENSAI_FLAG_TF32_STATISTICS; other bits
 * are EINVAL.
 *
 * The dictionary draw (BPFA section, the dictionary-learning step) takes one
 * of three forms, all the same atom-ordered conditionals: by default the
 * residual form, atoms in blocks of 8 over the residual of every observed
 * pixel (the space-organised cooperative kernel); SENSAI_FLAG_CHAIN_DICTIONARY
 * the residual form with one CTA per pixel; SENSAI_FLAG_DENSE_STATISTICS
 * (K <= 128) the dense-statistics form -- per within-patch pixel p the Gram
 * C_p = sum w_i w_i^T and the correlations Y_p = sum w_i x_ip over the
 * patches observing p, contracted on the tensor cores, then the draws in
 * FP64 from C_p, Y_p and the current dictionary.
 *
 * The code sweep keeps the whole dictionary in shared memory when
 * (P + 1) * (K rounded up to 8, odd) floats fit (K = 128, P = 100: 52 KB);
 * otherwise it streams the dictionary through shared memory in slices of
 * atoms.  SENSAI_FLAG_STREAM_DICTIONARY streams it always;
 * SENSAI_SLICE_ATOMS(n) fixes the slice at n atoms (n a multiple of 8, no
 * larger than what fits).  Results do not depend on either. */
#define SENSAI_FLAG_STREAM_DICTIONARY 0x1
/* The dictionary draw runs one CTA per within-patch pixel chain instead of
 * the cooperative space-organised kernel, so that the context can share the
 * GPU with others (required for sensai_batch_create).  Results are the same
 * draws up to FP32 summation order. */
#define SENSAI_FLAG_CHAIN_DICTIONARY 0x2
/* Reading of the gamma_s update (BPFA section: the weights' precision has a
 * Gamma prior).  Default: the weights of inactive atoms are integrated out;
 * gamma_s ~ Ga(c + sum z / 2, d + sum_{z=1} s^2 / 2).  With this flag every
 * code sweep is followed by a draw of s_ik ~ N(0, 1/gamma_s) for each entry
 * it left inactive (from the Philox words an active entry uses for its
 * normal; the weight z s stays 0 and the draw is not stored), whose square
 * is added to the s^2 sum; then
 * gamma_s ~ Ga(c + N K / 2, d + sum_all s^2 / 2).  z and the active weights
 * are the same draws under both readings.  The inactive draws exist only
 * within the sweep that made them: a gamma_s draw from a state set by
 * sensai_set_state with no sweep since sums the stored (active) weights.
 * One extra kernel per code sweep; not accepted by sensai_batch_create. */
#define SENSAI_FLAG_GAMMA_S_FULL 0x4
/* The dense-statistics form of the dictionary draw (tensor-core Grams, FP32
 * level: head/tail TF32 split).  Requires K <= 128 (else EINVAL); not with
 * SENSAI_FLAG_CHAIN_DICTIONARY. */
#define SENSAI_FLAG_DENSE_STATISTICS 0x8
/* The dense-statistics form at reduced precision: the Grams C_p from the
 * TF32 heads of the weights alone (one tensor-core product instead of the
 * head/tail split that gives FP32-level sums); relative error of C_p about
 * 2^-11, of the drawn atoms about 1e-3.  Everything else is unchanged
 * (correlations Y_p in FP32, sums and draws in FP64). */
#define SENSAI_FLAG_TF32_STATISTICS 0x10
#define SENSAI_SLICE_ATOMS(n) ((((n) / 8) & 0xff) << 8)
typedef struct {
    int32_t ndim;
    int64_t M[4];
    int32_t B[4];
    int32_t stride[4];
    int32_t K;
    double a, b;
    double c, d;
    double e, f;
    uint64_t seed;
    int32_t flags;
} sensai_params;

/* Sampler state as host arrays (get/set).  Any pointer may be NULL to skip
 * that part.  D: K*P floats.  Z: N*K bytes, patch-major (Z[i*K + k]).  S:
 * N*K floats, patch-major; S is 0 where Z is 0.  pi: K doubles. */
typedef struct {
    float* D;
    uint8_t* Z;
    float* S;
    double* pi;
    double gamma_s;
    double gamma_eps;   /* <= 0 on get: not yet initialised; on set: leave unset */
    int64_t iter;       /* iteration index t used by the next draws */
} sensai_state;

/* Summary of the last completed phase, read back from the device. */
typedef struct {
    int64_t iter;          /* current iteration index t */
    int64_t n_patches;     /* N */
    int64_t patch_size;    /* P */
    int64_t n_observed;    /* sum_i |Omega_i| */
    int64_t n_active;      /* sum_ik z_ik */
    int32_t max_observed;  /* max_i |Omega_i| */
    int32_t K;
    double sum_s2;         /* sum of s_ik^2 over active entries */
    double sum_r2;         /* sum_i ||r_i||^2 on observed pixels (last residual pass) */
    double gamma_s;
    double gamma_eps;
    int64_t kernel_launches;   /* kernels this context has launched so far */
    int64_t changed_updates;   /* code updates whose weight changed, since the last profile start */
    int64_t changed_observed;  /* sum of |Omega_i| over those updates */
    int64_t active_draws;      /* code draws with z = 1, since the last profile start */
    int32_t slice_atoms;       /* code sweep: 0 = dictionary resident in shared memory, else atoms per streamed slice */
    int32_t slices;            /* code sweep: streamed slices per pass (0 when resident) */
    int64_t rebuild_observed;  /* residual rebuilds inside code sweeps (patch extraction): sum of
                                  |Omega_i| x non-zero stored weights, since the last profile start */
    int32_t dictionary_form;   /* kernel of the dictionary draw: 0 one CTA per chain, 1 space-organised
                                  (weight records read through L1), 2 space-organised with each atom
                                  block's weight records staged in shared memory, 3 dense statistics */
    int32_t dictionary_smem_kb;  /* dynamic shared memory of the dictionary kernel, KB (forms 1 and 2) */
} sensai_stats;

/* Create a context on the current CUDA device.  `mask` is prod(M) host bytes
 * (nonzero = sampled pixel), copied.  Geometry (observed-pixel lists, per-
 * pixel patch bitmaps) is built on the device; the dictionary is drawn from
 * its prior (counter (p, k, 0, INIT)), all codes are 0, pi_k = 0.5,
 * gamma_s = 1 and gamma_eps is set from the first frame as
 * 1 / max(var(observed pixels), 1e-12).  Device memory is allocated here
 * and released by sensai_destroy.  Sec. "N-Dimensional Inpainting" (patch
 * shape B in any dimension), Sec. "SenseAI: Feature Summary" (modular
 * library, programmatic signal selection = the caller's mask).  Any failure
 * frees everything allocated so far; out of device memory is ENOMEM.  For
 * tests of that path the environment variable SENSAI_FAULT=alloc:N makes the
 * N-th device allocation of the call (1-based) fail as out of memory. */
sensai_status sensai_create(const sensai_params* params, const uint8_t* mask, sensai_ctx** out);
void sensai_destroy(sensai_ctx* ctx);

/* Copy a frame (prod(M) floats, host or device) into the context. */
sensai_status sensai_set_frame(sensai_ctx* ctx, const float* frame, void* stream);

/* Return the state to its initial draw (dictionary from the prior, codes 0,
 * pi = 0.5, gamma_s = 1, gamma_eps unset, t = 0).  Asynchronous. */
sensai_status sensai_reset(sensai_ctx* ctx, void* stream);

/* Joint dictionary learning and sparse coding (Sec. "Beta-Process Factor
 * Analysis (BPFA)": each iteration performs a dictionary-learning step and a
 * sparse-coding step).  `frame` (host or device, may be NULL to keep the
 * current frame) is copied first.  Runs `iters` iterations, each: code
 * sweep, dictionary sweep, pi / gamma draws, then t += 1. */
sensai_status sensai_learn(sensai_ctx* ctx, const float* frame, int32_t iters, void* stream);

/* Sparse coding with the dictionary held fixed (dictionary transfer, Sec.
 * "SenseAI: Feature Summary"): copies `frame` (host or device, not NULL),
 * clears the codes, runs `sweeps` iterations of code sweep + pi / gamma
 * draws (t += 1 each), then writes the overlap-add reconstruction to `out`
 * (prod(M) floats, host or device; may be NULL to skip). */
sensai_status sensai_inpaint(sensai_ctx* ctx, const float* frame, int32_t sweeps, float* out, void* stream);

/* Single phases at the current t (t is not advanced):
 *  - sensai_sweep_codes: one sparse-code sweep (patch extraction fused);
 *  - sensai_draw_dictionary: one dictionary sweep, atoms in order;
 *  - sensai_draw_hyper: pi_k, gamma_s, gamma_eps (gamma_eps uses the current
 *    residual).
 * These exist so each step can be checked on its own. */
sensai_status sensai_sweep_codes(sensai_ctx* ctx, void* stream);
sensai_status sensai_draw_dictionary(sensai_ctx* ctx, void* stream);
sensai_status sensai_draw_hyper(sensai_ctx* ctx, void* stream);

/* Overlap-add reconstruction: every pixel's mean over the patches covering
 * it of (D w_i) at that pixel, observed pixels included (the reconstruction
 * of Sec. "Time-To-Solution").  `out`: prod(M) floats, host or device. */
sensai_status sensai_reconstruct(sensai_ctx* ctx, float* out, void* stream);

/* Posterior-mean reconstruction over several samples of the chain (the
 * reconstructions of Sec. "Time-To-Solution" are built from the sampler's
 * draws; averaging the last T samples estimates the posterior mean of the
 * image instead of showing one draw).
 *  - sensai_mean_reset: empties the running sum (asynchronous on `stream`);
 *  - sensai_mean_add: adds the overlap-add reconstruction of the current
 *    state (as sensai_reconstruct would return it), in FP64, and counts it;
 *    typically called after each of the last T iterations of sensai_learn
 *    (iters = 1 per call) or sweeps of sensai_inpaint;
 *  - sensai_mean_read: writes the running sum / count to `out` (prod(M)
 *    floats, host or device).  SENSAI_ESTATE when nothing was added since
 *    the last reset.
 * The running sum (8 bytes per pixel) is allocated with the context. */
sensai_status sensai_mean_reset(sensai_ctx* ctx, void* stream);
sensai_status sensai_mean_add(sensai_ctx* ctx, void* stream);
sensai_status sensai_mean_read(sensai_ctx* ctx, float* out, void* stream);

/* Number of patches covering each pixel (int32, prod(M), host or device):
 * per dimension floor(min(y, last) / S) - ceil(max(0, y - B + 1) / S) + 1
 * with last = (G - 1) S the final patch start, multiplied over dimensions. */
sensai_status sensai_overlap_counts(sensai_ctx* ctx, int32_t* out, void* stream);

/* Dictionary transfer: K*P host floats. */
sensai_status sensai_get_dictionary(sensai_ctx* ctx, float* D);
sensai_status sensai_set_dictionary(sensai_ctx* ctx, const float* D);

/* Read or replace the sampler state (host arrays, synchronous). */
sensai_status sensai_get_state(sensai_ctx* ctx, sensai_state* state);
sensai_status sensai_set_state(sensai_ctx* ctx, const sensai_state* state);

/* Synchronise the last stream used and report the statistics. */
sensai_status sensai_get_stats(sensai_ctx* ctx, sensai_stats* stats);

/* ---- Live serving (reconstruction of a continuous feed, Sec. "Introduction"
 * and Sec. "Visitors Experience"; dictionary transfer, Sec. "SenseAI: Feature
 * Summary").  sensai_serve_start snapshots the context's dictionary, pi,
 * gamma_s, gamma_eps and iteration index; submitted frames are then inpainted
 * with that fixed dictionary (codes cleared, `sweeps` iterations of code sweep
 * + pi / gamma draws, then overlap-add), exactly like sensai_inpaint.
 *
 * Each frame has its own shape M (same ndim, patch shape and stride as the
 * context; (M[d] - B[d]) divisible by the stride) and its own mask.  Its
 * random numbers are keyed by seed_f = h(h(h(seed) ^ stream_id) ^ frame_id),
 * h = SplitMix64's finaliser (Steele, Lea & Flood 2014), so a frame's result
 * does not depend on what else is in flight.
 *
 * Admission: `slots` frames may be on the GPU at once, each with its own CUDA
 * stream and worker thread; a queued frame is admitted in arrival order when
 * a slot is free and the device bytes of the frames in flight plus its own
 * stay within `memory_budget`.  Work of different frames overlaps on the
 * device. */
typedef void (*sensai_done_fn)(void* user, uint64_t frame_id, int32_t status);

typedef struct {
    int32_t slots;           /* frames in flight, 1..64 */
    int64_t max_pixels;      /* largest frame accepted, in pixels */
    int64_t memory_budget;   /* device bytes for frames in flight; <= 0: slots x largest frame */
    int32_t max_observed;    /* cap on observed pixels per patch (<= 256); frames above it fail */
} sensai_serve_params;

/* Start the serving engine on a context (allocates the slots' device memory).
 * EBUSY if it is already serving. */
sensai_status sensai_serve_start(sensai_ctx* ctx, const sensai_serve_params* sp);

/* Queue one frame.  `frame` (prod(M) floats), `mask` (prod(M) bytes) and
 * `out` (prod(M) floats) are host buffers read and written after admission,
 * so the caller keeps them valid until `done(user, frame_id, status)` runs
 * (on a worker thread; status is a sensai_status).
 * Returns EINVAL (nothing queued) for a bad shape or a frame above
 * max_pixels; ESTATE when the engine is not running. */
sensai_status sensai_submit_frame(sensai_ctx* ctx, int32_t stream_id, uint64_t frame_id, const float* frame,
                                  const uint8_t* mask, const int64_t* M, int32_t sweeps, float* out,
                                  sensai_done_fn done, void* user);

/* Block until every submitted frame has completed; returns the first
 * failure of a frame since the previous drain (with its message), else OK. */
sensai_status sensai_serve_drain(sensai_ctx* ctx);

/* Drain, stop the workers and release the slots. */
sensai_status sensai_serve_stop(sensai_ctx* ctx);

/* ---- Batches: many independent problems learned together -------------------
 *
 * The paper processes frames one after another; a batch runs the Gibbs
 * iterations (the BPFA section's sampler) of n independent contexts together
 * so that small problems share the GPU.  One iteration of all instances is a
 * few launches that each cover every instance (code sweeps per kernel
 * variant, dictionary draws per storage mode, pi and gamma draws), captured
 * once into a CUDA graph and replayed per iteration.  Each context ends
 * exactly where sensai_learn(iters) on it alone would: the same per-instance
 * arithmetic, the same draws.
 *
 * Contexts must have a frame set (sensai_set_frame or an earlier call with a
 * frame), share one device, be created with SENSAI_FLAG_CHAIN_DICTIONARY (the
 * cooperative dictionary kernel cannot share the GPU) and not be serving;
 * a context may belong to one batch at a time.  The batch does not own the
 * contexts; destroy it before them.  Errors: EINVAL for bad arguments, the
 * first instance's error otherwise. */
typedef struct sensai_batch sensai_batch;
sensai_status sensai_batch_create(sensai_ctx* const* ctxs, int32_t n, sensai_batch** out);

/* iters Gibbs iterations of every instance, asynchronous on cuda_stream
 * (ordered after the work already on it, and work enqueued on it afterwards
 * waits for the batch). */
sensai_status sensai_batch_learn(sensai_batch* b, int32_t iters, void* cuda_stream);

/* Autotuner: times the batch with the batched code sweeps' grids at 4 / d
 * waves of the GPU for d = 1, 2, 4, 8, 16 (the CTAs are divided among the
 * instances in proportion to their work), iters_per_trial iterations per
 * candidate, and keeps the fastest; *divisor (may be NULL) receives d.  The trials are real
 * Gibbs iterations: each candidate runs one warm-up and iters_per_trial timed
 * iterations, so every instance advances by 5 * (1 + iters_per_trial)
 * iterations.  Results do not depend on the choice. */
sensai_status sensai_batch_tune(sensai_batch* b, int32_t iters_per_trial, void* cuda_stream, int32_t* divisor);

void sensai_batch_destroy(sensai_batch* b);

/* Failure detection self-test.  Every device-side wait of the library (the
 * dictionary kernel's grid barrier, the streamed sweep's mbarrier waits) gives
 * up after about one second, sets SENSAI_ETIMEOUT in the context's status
 * word and returns, instead of hanging the GPU.  This runs one such wait on a
 * condition that nothing satisfies (which = 0: grid barrier, 1: mbarrier) on
 * the current device.  It returns SENSAI_ETIMEOUT when the wait gave up as
 * designed (the expected result; the device stays usable), SENSAI_OK if it
 * did not give up, SENSAI_EINVAL for another `which`.  Takes ~1 s. */
sensai_status sensai_selftest_wait(int32_t which);

/* Per-iteration metrics trace: the live statistics, parameters and
 * image-quality metrics that the paper's display window plots (abstract;
 * Sec. "SenseAI: Feature Summary"), as text lines instead of plots.  path: a
 * file opened for appending; NULL stops
 * tracing (and closes the file).  clean: NULL, or the ground-truth frame
 * (prod(M) floats, host or device; copied).  After every Gibbs iteration of
 * sensai_learn and sensai_inpaint the context appends one JSON line:
 * {"t": the iteration's counter, "mode": "learn" | "inpaint", "gamma_s",
 * "gamma_eps": the iteration's draws, "active": sum z, "active_per_patch",
 * "sum_s2", "sum_r2": the sums behind the gamma draws, "psnr_db": 10 log10(1 /
 * MSE) of the current overlap-add reconstruction against clean over all
 * pixels (null without clean), "wall_ms": host time since the previous
 * line}.  Each line synchronises the stream; with clean it adds one
 * reconstruction and a frame-sized device-to-host copy.  The sampler's
 * results do not depend on tracing.  EINVAL if the file cannot be opened. */
sensai_status sensai_trace(sensai_ctx* ctx, const char* path, const float* clean);

/* Per-phase device timing.  enable = 1 clears the record and starts timing:
 * every later phase records a CUDA event pair on its launching stream;
 * enable = 0 stops.  sensai_profile_read synchronises and returns, for the
 * phases {code sweep, dictionary sweep, pi/gamma draws, reconstruction}, the
 * summed milliseconds ms[4] and the number of timed launches counts[4].
 * Tracing support; the paper has no counterpart. */
sensai_status sensai_profile(sensai_ctx* ctx, int32_t enable);
sensai_status sensai_profile_read(sensai_ctx* ctx, double* ms, int64_t* counts);

/* Overlap-add reconstruction that allocates nothing, for callers that cannot
 * allocate GPU memory themselves: a plugin inside a host application whose
 * memory pool owns the device, or a live-acquisition callback with a hard
 * time budget in which cudaMalloc (which may block and synchronise the
 * device) is not allowed.  The paper has no counterpart; it computes the same
 * frame as sensai_reconstruct without a context.
 *  - params: frame / patch / stride geometry and K (the other fields are
 *    ignored); the same validity rules as sensai_create (P <= 1024, N and
 *    prod(M) below 2^31), checked before anything touches the device.
 *  - D: K*P floats, S: N*K floats patch-major (S[i*K + k], 0 where atom k
 *    is inactive in patch i), out: prod(M) floats -- all device (or
 *    managed) pointers on the current device, owned by the caller; host
 *    memory and another GPU's memory are refused with SENSAI_EINVAL.  The
 *    element counts cannot be checked from bare pointers: the caller
 *    guarantees them.
 *  - Scratch is a fixed 16 MiB static device array (4,194,304 floats) that
 *    every GPU loading the library holds until exit; P * N above that is
 *    rejected with SENSAI_EINVAL.  No cudaMalloc / cudaFree is called.
 *  - The first call on a device looks up the array's device address; make
 *    that first call before any stream capture.  All calls share the array:
 *    calls that overlap on the GPU race and must be serialised by the caller.
 *  - Asynchronous on `stream`; errors as for the other entry points. */
sensai_status sensai_reconstruct_static(const sensai_params* params, const float* D, const float* S,
                                        float* out, void* stream);

/* Message describing the last error on the calling thread ("" if none). */
const char* sensai_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
