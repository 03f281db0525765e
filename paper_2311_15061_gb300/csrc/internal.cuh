// internal.cuh -- device-side building blocks shared by the sensai kernels.
//
// Random numbers follow the library's published counter convention (see
// include/sensai.h): Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) keyed by
// the 64-bit seed, counter (index0, index1, t, tag | attempt << 8), uniforms
// (x + 1) 2^-32, Box-Muller normals, Marsaglia-Tsang Gamma (ACM TOMS 2000)
// with the U^(1/alpha) boost below shape 1, Beta as a ratio of Gammas.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "sensai.h"

namespace sensai {

enum : uint32_t {
    kTagInit = 1,   // dictionary initialisation, counter (p, k, 0)
    kTagCodes = 2,  // sparse-code draws of atoms 2m, 2m + 1, counter (i, m, t)
    kTagDict = 3,   // dictionary draw, counter (p, k, t)
    kTagPiA = 4,    // Beta draw of pi_k: numerator Gamma, counter (k, 0, t)
    kTagPiB = 5,    // Beta draw of pi_k: denominator Gamma
    kTagGs = 6,     // gamma_s, counter (0, 0, t)
    kTagGe = 7      // gamma_eps, counter (0, 0, t)
};

constexpr int kMaxDim = 4;
constexpr int kGammaAttempts = 64;

// Patch geometry, passed by value to kernels.
struct Geom {
    int ndim;
    int P;                 // pixels per patch
    int K;                 // atoms
    int KB;                // 8-atom blocks: ceil(K / 8)
    int NW;                // 32-patch words: ceil(N / 32)
    long long Npad;        // NW * 32
    long long N;           // patches
    long long nframe;      // pixels per frame
    long long M[kMaxDim];  // frame shape
    long long G[kMaxDim];  // patch-start grid shape
    long long fs[kMaxDim]; // frame strides (row-major)
    int B[kMaxDim];
    int S[kMaxDim];
};

// Scalars that live on the device between phases.
struct DevScalars {
    double gamma_s;
    double gamma_eps;
    double sum_s2;     // last code sweep: sum of s^2 over active entries
    double sum_r2;     // last residual pass: sum of squared residuals
    long long n_active;
    unsigned long long chg_n;    // code updates whose weight changed
    unsigned long long chg_obs;  // sum of |Omega_i| over those updates
    unsigned long long act_n;    // code draws with z = 1
    unsigned long long rb_obs;   // in-sweep residual rebuilds: sum over patches of |Omega_i| x non-zero weights
    int ge_set;        // gamma_eps initialised from a frame
    int status;        // sticky error word written by kernels (0 = ok)
    uint32_t t_iter;   // iteration index for kernels replayed from a CUDA graph
};

// Nanoseconds since an arbitrary origin (the GPU's global timer); bounds the
// device-side waits by time as well as by poll count.
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
constexpr unsigned long long kWaitLimitNs = 1000000000ull;   // 1 s: every device wait gives up after this

// Iteration index of a launch: the argument, or the device copy when the
// launch is replayed from a captured graph (t_dev set).
__device__ __forceinline__ uint32_t launch_t(uint32_t t, bool t_dev, const DevScalars* sc)
{
    return t_dev ? sc->t_iter : t;
}

// Weights are stored in 8-atom blocks per patch, [KB][Npad][8]: the eight
// weights of patch i for atoms 8 kb .. 8 kb + 7 are one 32-byte sector, and a
// warp's 32 patches of one block are 1 KB contiguous.  Inactive weights and
// padding atoms (k >= K) are 0.
constexpr int kAtomBlock = 8;

__host__ __device__ __forceinline__ long long wblock(const Geom& g, int kb, long long i)
{
    return ((long long)kb * g.Npad + i) * kAtomBlock;
}

// One 32-byte weight record as a single 256-bit access (address 32-byte
// aligned): one L1 wavefront per lane instead of two.
struct W8 {
    float v[kAtomBlock];
};

// Not volatile: the compiler may schedule these loads early (stores of the
// same array carry a memory clobber, so no load moves across them).
__device__ __forceinline__ W8 load_w8(const float* p)
{
    W8 r;
    asm("ld.global.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3]),
                   "=f"(r.v[4]), "=f"(r.v[5]), "=f"(r.v[6]), "=f"(r.v[7])
                 : "l"(p));
    return r;
}

__device__ __forceinline__ void store_w8(float* p, float a0, float a1, float a2, float a3, float a4, float a5,
                                         float a6, float a7)
{
    asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
                 :: "l"(p), "f"(a0), "f"(a1), "f"(a2), "f"(a3), "f"(a4), "f"(a5), "f"(a6), "f"(a7)
                 : "memory");
}

// Frame offset of patch i's first pixel.
__host__ __device__ inline long long patch_origin(const Geom& g, long long i)
{
    long long off = 0;
    for (int d = g.ndim - 1; d >= 0; --d) {
        long long id = i % g.G[d];
        i /= g.G[d];
        off += id * g.S[d] * g.fs[d];
    }
    return off;
}

// ------------------------------------------------------------------- RNG --

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k.x, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k.y, (uint32_t)p0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// Philox4x32-10 key schedule (k0 + r W0, k1 + r W1 for rounds r = 0..9),
// computed once on the host so the kernels read it from the constant bank.
struct PhiloxKeys {
    uint32_t k0[10];
    uint32_t k1[10];
};

inline PhiloxKeys philox_round_keys(unsigned long long seed)
{
    PhiloxKeys r;
    uint32_t a = (uint32_t)seed, b = (uint32_t)(seed >> 32);
    for (int i = 0; i < 10; ++i) {
        r.k0[i] = a;
        r.k1[i] = b;
        a += 0x9E3779B9u;
        b += 0xBB67AE85u;
    }
    return r;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxKeys& ks)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ ks.k0[round], (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ ks.k1[round], (uint32_t)p0);
    }
    return c;
}

__device__ __forceinline__ uint2 seed_key(unsigned long long seed)
{
    return make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
}

__device__ __forceinline__ double uniform64(uint32_t x)
{
    return ((double)x + 1.0) * (1.0 / 4294967296.0);
}

// Box-Muller in FP64: sqrt(-2 ln u1) cos(2 pi u2).
__device__ __forceinline__ double normal64(uint32_t x0, uint32_t x1)
{
    return sqrt(-2.0 * log(uniform64(x0))) * cospi(2.0 * uniform64(x1));
}

// Box-Muller in FP32 (used for the code draws): the pair
// sqrt(-2 ln u1) (cos, sin)(2 pi u2) with u = (x + 1) 2^-32, evaluated so
// that no FP32 rounding of the 32-bit words is amplified:
//  * ln u1: for u1 <= 1/2 the hardware log2 (relative error ~2^-22 there);
//    for u1 > 1/2, with v = 1 - u1 = (2^32-1 - x0) 2^-32 formed in integers,
//    ln(1 - v) = -(v + v^2/2 + ... + v^8/8) when v < 1/8 (relative
//    truncation error below 1e-8) and the hardware log2 of 1 - v otherwise
//    (there |ln(1 - v)| >= 0.13);
//  * the angle 2 pi (x1 + 1) / 2^32 is split in integers into the nearest
//    multiple of pi/2 (quarter q) and a remainder d in [-2^29, 2^29), so the
//    cosine and sine are +-cos or +-sin of t = pi d / 2^31 with
//    |t| <= pi/4, evaluated by their Taylor series (to t^10 and t^9;
//    remainders below 2e-9).
__device__ __forceinline__ void normal32_pair(uint32_t x0, uint32_t x1, float& n_cos, float& n_sin)
{
    const float two_m32 = 2.3283064365386963e-10f;  // 2^-32
    const float ln2 = 0.69314718055994531f;
    float ln_u1;
    if (x0 < 0x80000000u) {
        ln_u1 = ln2 * __log2f(fmaf((float)x0, two_m32, two_m32));
    } else {
        const float v = (float)(0xFFFFFFFFu - x0) * two_m32;
        if (v < 0.125f) {
            // -(v + v^2/2 + ... + v^8/8), Horner form
            float t = fmaf(v, 0.125f, 1.0f / 7.0f);
            t = fmaf(v, t, 1.0f / 6.0f);
            t = fmaf(v, t, 0.2f);
            t = fmaf(v, t, 0.25f);
            t = fmaf(v, t, 1.0f / 3.0f);
            t = fmaf(v, t, 0.5f);
            t = fmaf(v, t, 1.0f);
            ln_u1 = -v * t;
        } else {
            ln_u1 = ln2 * __log2f(1.0f - v);
        }
    }
    const uint64_t y = (uint64_t)x1 + 1u;                               // angle = 2 pi y / 2^32
    const uint32_t quarter = (uint32_t)((y + (1u << 29)) >> 30);        // nearest multiple of pi/2
    const int32_t d = (int32_t)((int64_t)y - ((int64_t)quarter << 30));
    const float t = (float)d * 1.4629180792671596e-09f;                 // pi d / 2^31, |t| <= pi/4
    const float t2 = t * t;
    // sin t = t (1 - t^2/6 (1 - t^2/20 (1 - t^2/42 (1 - t^2/72))))
    float sn = fmaf(-t2, 1.0f / 72.0f, 1.0f);
    sn = fmaf(-t2 * (1.0f / 42.0f), sn, 1.0f);
    sn = fmaf(-t2 * (1.0f / 20.0f), sn, 1.0f);
    sn = fmaf(-t2 * (1.0f / 6.0f), sn, 1.0f);
    sn *= t;
    // cos t = 1 - t^2/2 (1 - t^2/12 (1 - t^2/30 (1 - t^2/56 (1 - t^2/90))))
    float cs = fmaf(-t2, 1.0f / 90.0f, 1.0f);
    cs = fmaf(-t2 * (1.0f / 56.0f), cs, 1.0f);
    cs = fmaf(-t2 * (1.0f / 30.0f), cs, 1.0f);
    cs = fmaf(-t2 * (1.0f / 12.0f), cs, 1.0f);
    cs = fmaf(-t2 * 0.5f, cs, 1.0f);
    // cos(q pi/2 + t): cos t, -sin t, -cos t, sin t; sin(q pi/2 + t): sin t,
    // cos t, -sin t, -cos t (q mod 4)
    const bool odd = (quarter & 1u) != 0;
    const float c = odd ? sn : cs;
    const float sv = odd ? cs : sn;
    const float sign_c = ((quarter + 1u) & 2u) ? -1.0f : 1.0f;   // quarters 1, 2 negative
    const float sign_s = (quarter & 2u) ? -1.0f : 1.0f;          // quarters 2, 3 negative
    const float m = -2.0f * ln_u1;
    const float rad = m * rsqrtf(fmaxf(m, 1e-30f));
    n_cos = sign_c * c * rad;
    n_sin = sign_s * sv * rad;
}

// Marsaglia-Tsang for shape >= 1; attempt a uses block (c0, c1, t, tag | a << 8):
// words 0-1 -> the normal, word 2 -> the acceptance uniform.
__device__ inline double gamma_shape_ge1(double shape, unsigned long long seed, uint32_t c0,
                                         uint32_t c1, uint32_t t, uint32_t tag)
{
    const double dd = shape - 1.0 / 3.0;
    const double cc = 1.0 / sqrt(9.0 * dd);
    const uint2 key = seed_key(seed);
    for (uint32_t a = 0; a < (uint32_t)kGammaAttempts; ++a) {
        const uint4 blk = philox4x32_10(make_uint4(c0, c1, t, tag | (a << 8)), key);
        const double xn = normal64(blk.x, blk.y);
        double v = 1.0 + cc * xn;
        if (v <= 0.0) continue;
        v = v * v * v;
        const double u = uniform64(blk.z);
        const double x2 = xn * xn;
        if (u < 1.0 - 0.0331 * x2 * x2) return dd * v;
        if (log(u) < 0.5 * x2 + dd * (1.0 - v + log(v))) return dd * v;
    }
    return dd;
}

// Gamma(shape, 1); below shape 1: Gamma(shape + 1) U^(1/shape), U = word 3 of
// the attempt-0 block.
__device__ inline double gamma_draw(double shape, unsigned long long seed, uint32_t c0, uint32_t c1,
                                    uint32_t t, uint32_t tag)
{
    if (shape >= 1.0) return gamma_shape_ge1(shape, seed, c0, c1, t, tag);
    const double g = gamma_shape_ge1(shape + 1.0, seed, c0, c1, t, tag);
    const uint4 blk = philox4x32_10(make_uint4(c0, c1, t, tag), seed_key(seed));
    return g * pow(uniform64(blk.w), 1.0 / shape);
}

__device__ inline double beta_draw(double alpha, double beta, unsigned long long seed, uint32_t k, uint32_t t)
{
    const double g1 = gamma_draw(alpha, seed, k, 0, t, kTagPiA);
    const double g2 = gamma_draw(beta, seed, k, 0, t, kTagPiB);
    return g1 / (g1 + g2);
}

// ------------------------------------------------------------ reductions --

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Fixed-order block sum (deterministic); result valid in thread 0.
// `scratch` must hold blockDim.x / 32 doubles.
__device__ inline double block_sum(double v, double* scratch)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (warp == 0) {
        r = (lane < (int)(blockDim.x >> 5)) ? scratch[lane] : 0.0;
        r = warp_sum(r);
    }
    return r;
}

// ------------------------------------------------------ kernel arguments --

// Per-patch tables of the code sweep are in sweep order: position (slot) s
// of the sweep holds patch perm[s] (perm null: the identity).  A warp sweeps
// 32 consecutive slots, so its activity word Zb[k][w] holds the bits of the
// patches at slots 32 w .. 32 w + 31.  Weights W stay in patch order.
struct SweepArgs {
    Geom g;
    const float* x;            // frame
    const uint16_t* obs;       // [maxobs][N] within-patch index of each observed pixel, by slot
    const uint16_t* nobs;      // [N] observed pixels per patch, by slot
    const int* perm = nullptr; // [Npad] slot -> patch (slots >= N: themselves); null: identity
    const int* imgoff;         // [P] frame offset of within-patch pixel p
    const float* D;            // [K][P]
    float* W;                  // [KB][Npad][8] weights (0 where inactive), by patch
    uint32_t* Zb;              // [K][NW] activity bits by slot (written)
    const float* lpi;          // [K] logit(pi_k)
    const DevScalars* sc;
    const int* pos;            // [maxobs][N] residual position of observed pixel j of the patch at a slot
    float* R;                  // residual in the dictionary step's layout, R[pos[j][slot]]
                               // (null: serving, the residual is not kept)
    const float* R_in = nullptr;   // non-null: R holds the current residual at launch (the
                                   // sweep starts from it instead of rebuilding x - D w)
    double* part_s2;           // [NW] per 32-patch chunk
    double* part_r2;           // [NW] per 32-patch chunk
    unsigned int* chunk_counter;  // work counter, zeroed before each launch
    unsigned int unit_lo = 0;     // the launch's work units: unit_lo + counter values below unit_hi
    unsigned int unit_hi = 0;     // (0: every unit)
    DevScalars* sc_out;           // change counters (same object as sc)
    PhiloxKeys keys;              // round keys of the seed
    uint32_t t;
    bool t_dev = false;           // take t from sc->t_iter (graph replay)
    // streamed dictionary (sweep_tiled.cu); Dsl null: the whole dictionary
    // is resident in shared memory (sweep.cu)
    const float* Dsl = nullptr;   // [slices][slice_stride] slices in shared-memory layout
    int slice_atoms = 0;          // KS, a multiple of 8
    int slices = 0;               // ceil(8 KB / KS)
    long long slice_stride = 0;   // floats per slice, ((P + 1) (KS + 1)) rounded up to 4
};

struct DictArgs {
    Geom g;
    float* D;                  // [K][P]
    const float* W;            // [KB][Npad][8]
    const int* Ilist;          // per pixel p: the patches observing p, in slot order
    const int* Rbase;          // [P + 1]
    float* R;
    const DevScalars* sc;
    double* part_r2;           // [P]
    unsigned long long seed;
    uint32_t t;
    bool t_dev = false;        // take t from sc->t_iter (graph replay)
};

// The space-organised dictionary sweep (dict_space.cu), planned per context:
// pair jp of thread t in CTA c is element base[c] + jp * 512 + t of R and pidx.
struct DictSpacePlan {
    int grid = 0;              // CTAs of the cooperative launch; 0: use dict.cu
    size_t smem = 0;           // dynamic shared memory
    bool rho_smem = false;     // residual pairs staged in shared memory
    bool staged = false;       // weight records staged in shared memory per block
    int* nb = nullptr;         // [grid][2 * kMaxDim] neighbourhood origin and extents (staged)
    int half_floats = 0;       // floats of one half-record array of a staging buffer
    int buf_floats = 0;        // floats of one staging buffer (0 when not staged)
    int red_sep_floats = 0;    // group-sum scratch outside the staging buffers
    int rows_max = 0;          // largest neighbourhood row count (staged)
    int own_max = 0;           // chains per CTA: ceil(P / grid)
    int max_np = 0;            // largest pair count of a thread
    long long pairs = 0;       // length of R and pidx (padded)
    int* order = nullptr;      // observed pixels, box by box, tile by tile
    int* start = nullptr;      // [grid + 1] each CTA's range of order
    int* np = nullptr;         // [grid][512] pairs per thread
    long long* base = nullptr; // [grid] first pair of each CTA
    int* pidx = nullptr;       // patch of every pair (staged: its neighbourhood position)
    float* part = nullptr;     // [P][grid][44] per-CTA block sums, chain-major
    float* delta = nullptr;    // [P][8] the block's updates
    unsigned int* bar = nullptr;   // grid barrier arrival counter, zeroed per launch
};

struct DictSpaceArgs {
    Geom g;
    float* D;                  // [K][P]
    const float* W;            // [KB][Npad][8]
    float* R;                  // residual pairs (plan layout)
    const int* pidx;
    const int* np;
    const long long* base;
    DevScalars* sc;            // gamma_eps in, status out
    double* part_r2;           // [gridDim.x]
    float* part;
    float* delta;
    unsigned int* bar;
    int own_max;
    const int* nb;             // staged: [grid][2 * kMaxDim]
    int half_floats, buf_floats, red_sep_floats, rows_max;
    unsigned long long seed;
    uint32_t t;
};

// The dictionary step in its dense-statistics form (gram.cu).
struct GramArgs {
    Geom g;
    const float* W;            // [KB][Npad][8]
    const int* Ilist;          // per pixel p: the patches observing p (Rbase layout)
    const float* Xlist;        // the frame value of each (p, patch) entry of Ilist
    const int4* items;         // (p, first entry, entries, -): segments of the per-pixel lists
    long long n_items;
    float* Cpart;              // [items][128][128] per-item partials T^T, C = (T + T^T) / 2 (FP32)
    float* Ypart;              // [items][2][128] per-item correlation partials (FP32), one per patch half
    double* C64;               // [P][128][128] FP64 sums of the partials (symmetrised by the draws)
    double* Y64;               // [P][128] Y_p
    const int* pitem_start;    // [P + 1] pixel p's items: pitem_idx[pitem_start[p] ..]
    const int* pitem_idx;
    float* D;                  // [K][P], redrawn in place
    const DevScalars* sc;      // gamma_eps, t_iter
    unsigned long long seed;
    uint32_t t;
    bool t_dev = false;
    bool tf32 = false;         // TF32-level statistics (one pass) instead of FP32-level (split)
    int* status;               // SENSAI_ETIMEOUT on a device-side wait that gives up
};

struct HyperArgs {
    Geom g;
    const uint32_t* Zb;        // [K][NW] activity words (the counts m_k come from them)
    int* m;                    // [K] active counts, written by the pi draws
    unsigned int* arrive = nullptr;   // arrival counter of the fused draw kernel (0 between launches)
    const double* part_s2;
    int n_s2;
    const double* part_r2;
    int n_r2;
    long long n_observed;
    double a_over_K, b_scaled, c, d, e, f;
    double* pi;                // [K]
    float* lpi;                // [K]
    DevScalars* sc;
    unsigned long long seed;
    uint32_t t;
    bool t_dev = false;        // take t from sc->t_iter (graph replay)
    bool full_s = false;       // SENSAI_FLAG_GAMMA_S_FULL: gamma_s shape c + N K / 2
};

// Live serving engine (serve.cu).
struct ServeEngine;
struct ServeInit {
    int device;
    Geom base;                 // ndim, B, S, K, KB, P of the context (M unused)
    const float* D;            // device [K][P], copied
    const double* pi;          // device [K], copied
    double gamma_s, gamma_eps;
    double a_over_K, b_param;  // b_param <= 0: b = N / 8 per frame
    double c, d, e, f;
    uint64_t seed;
    uint32_t t0;
    int slots;
    long long max_pixels;
    long long memory_budget;
    int max_observed;
    bool stream_dictionary;    // the context's SENSAI_FLAG_STREAM_DICTIONARY
    int slice_atoms;           // the context's SENSAI_SLICE_ATOMS (0: largest that fits)
    bool full_s = false;       // the context's SENSAI_FLAG_GAMMA_S_FULL
};
ServeEngine* serve_create(const ServeInit& in, sensai_status* status);
sensai_status serve_submit(ServeEngine* e, int32_t stream_id, uint64_t frame_id, const float* frame,
                           const uint8_t* mask, const int64_t* M, int32_t sweeps, float* out, sensai_done_fn done,
                           void* user);
sensai_status serve_drain(ServeEngine* e, std::string* message);   // first failure since the last drain
void serve_destroy(ServeEngine* e);
uint64_t serve_frame_seed(uint64_t seed, int32_t stream_id, uint64_t frame_id);

// Sets the calling thread's message returned by sensai_last_error().
void record_error(const char* msg);

// Batched launches: CTA b belongs to instance i with cta_start[i] <= b <
// cta_start[i + 1].  Copies that instance's arguments into shared memory and
// returns the copy (valid for the CTA's lifetime); *local (if not null)
// receives b - cta_start[i].  CTA-uniform; all threads must call it.
template <class Args>
__device__ __forceinline__ const Args* stage_instance_args(const Args* args, const int* cta_start, int n,
                                                           int* local = nullptr)
{
    __shared__ __align__(16) unsigned char buf[sizeof(Args)];
    __shared__ int inst_s, local_s;
    if (threadIdx.x == 0) {
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (cta_start[mid] <= (int)blockIdx.x) lo = mid;
            else hi = mid - 1;
        }
        inst_s = lo;
        local_s = (int)blockIdx.x - cta_start[lo];
    }
    __syncthreads();
    const int* src = reinterpret_cast<const int*>(args + inst_s);
    int* dst = reinterpret_cast<int*>(buf);
    for (int w = threadIdx.x; w < (int)(sizeof(Args) / sizeof(int)); w += blockDim.x) dst[w] = src[w];
    if (local) *local = local_s;
    __syncthreads();
    return reinterpret_cast<const Args*>(buf);
}

// Launchers (defined in the .cu files).
cudaError_t launch_sweep(const SweepArgs& a, int maxobs, int grid, cudaStream_t s);
int sweep_block_size();
int sweep_smem_bytes(const Geom& g);
int sweep_grid_size(const Geom& g, int maxobs, int device);
cudaError_t preload_sweep_variants();   // load every code-sweep kernel variant now
int sweep_lanes(int maxobs);            // lanes per patch for a largest |Omega_i|: 1, or 2 above 96
int sweep_variant(int maxobs);          // the template capacity serving maxobs (equal: same kernel)
// Batched code sweeps of instances sharing one variant (resident dictionary).
cudaError_t launch_sweep_multi(const SweepArgs* args, const int* cta_start, int n, int maxobs, int grid,
                               size_t smem, cudaStream_t s);
int sweep_multi_ctas_per_sm(int maxobs, size_t smem);
cudaError_t launch_sweep_tiled_multi(const SweepArgs* args, const int* cta_start, int n, int maxobs, int grid,
                                     size_t smem, cudaStream_t s);
int sweep_tiled_multi_ctas_per_sm(int maxobs, size_t smem);
cudaError_t preload_tiled_variants();

// How a code sweep runs: the whole dictionary resident in shared memory
// (slice_atoms = 0) or streamed in slices of slice_atoms atoms.
struct SweepPlan {
    int grid = 0;
    int lanes = 1;             // lanes per patch (2 above 96 observed pixels)
    int slice_atoms = 0;
    int slices = 0;
    long long slice_stride = 0;
    // Split by observed-pixel count (resident dictionary, one lane per
    // patch): the first split_units work units (slots in decreasing |Omega_i|
    // order) run the kernel for the largest count on split_grid CTAs, the
    // rest the kernel for kSplitObs pixels on light_grid CTAs, concurrently
    // (the latter on `side`, forked and joined by events); 0: no split.
    unsigned int split_units = 0;
    int split_grid = 0, light_grid = 0;
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    unsigned int* counter2 = nullptr;
};
constexpr int kSplitObs = 16;   // the light kernel's pixel capacity
// Resident when it fits (unless force_stream); else the largest slice that
// fits, or force_slice_atoms (a multiple of 8 no larger than that) if > 0.
bool plan_sweep(const Geom& g, int maxobs, int device, bool force_stream, int force_slice_atoms, SweepPlan* out);
long long slice_capacity_floats(const Geom& g);
// One code sweep by plan.  Dsl (slice_capacity_floats floats) is needed when
// streamed and is refilled from a.D on the stream first.  *nlaunch (if not
// null) receives the number of kernels launched.
cudaError_t launch_code_sweep(SweepArgs a, const SweepPlan& plan, int maxobs, float* Dsl, cudaStream_t s,
                              int* nlaunch);
cudaError_t launch_sweep_split(const SweepArgs& a, const SweepPlan& plan, int maxobs, cudaStream_t s);
// The residual x - D W rebuilt by the sweep's rebuild into a.R (through
// a.pos) and its squares' sums per work unit into a.part_r2 (resident
// dictionary only).
cudaError_t launch_rebuild(const SweepArgs& a, int maxobs, int grid, cudaStream_t s);
long long slice_stride_floats(const Geom& g, int KS);
size_t tiled_smem_bytes(const Geom& g, int KS);
int tiled_slice_atoms(const Geom& g, int maxobs, int device);
int tiled_grid_size(const Geom& g, int maxobs, int KS, int device);
cudaError_t launch_slice_dictionary(const Geom& g, const float* D, float* Dsl, int KS, cudaStream_t s);
cudaError_t launch_sweep_tiled(const SweepArgs& a, int maxobs, int grid, cudaStream_t s);
cudaError_t launch_dict(const DictArgs& a, int max_slots, cudaStream_t s);
// Reading A of the gamma_s update (SENSAI_FLAG_GAMMA_S_FULL): after a code
// sweep with the same (t, t_dev, seed), adds to part_s2 the squares of the
// prior draws of the entries that sweep left inactive.  lanes: the sweep's
// lanes per patch (its partials are per 32 / lanes patches).
cudaError_t launch_prior_s2(const Geom& g, const uint32_t* Zb, const int* perm, const DevScalars* sc, uint32_t t,
                            bool t_dev, unsigned long long seed, int lanes, double* part_s2, cudaStream_t s);
cudaError_t launch_hyper(const HyperArgs& a, cudaStream_t s);   // one kernel: K pi draws + gamma_s, gamma_eps
// Batched: pi_start is the prefix of K_i (one CTA per atom), gamma_start = 0..n.
cudaError_t launch_hyper_multi(const HyperArgs* args, const int* pi_start, const int* gamma_start, int n,
                               int pi_grid, cudaStream_t s);
// Per-chain dictionary kernels, batched: mode / smem from dict_mode(max slots).
int dict_mode(int max_slots, size_t* smem);
cudaError_t launch_dict_multi(const DictArgs* args, const int* cta_start, int n, int mode, size_t smem, int grid,
                              cudaStream_t s);
cudaError_t launch_set_iteration(DevScalars* sc, uint32_t t, cudaStream_t s);   // sc->t_iter = t
// Self-tests of the bounded device waits (each gives up after ~1 s).
cudaError_t launch_barrier_timeout_selftest(unsigned int* count, int* status, cudaStream_t s);
cudaError_t launch_mbar_timeout_selftest(int* status, cudaStream_t s);
// Builds the plan and its residual array R, filling pos[j][i] for the
// sweep; plan->grid = 0 (and no allocation) when the kernel cannot run.
cudaError_t ds_build(const Geom& g, const uint8_t* host_mask, const uint16_t* obs, const uint16_t* nobs, int device,
                     int* pos, float** R, DictSpacePlan* plan, cudaStream_t s);
void ds_free(DictSpacePlan* plan);
// pos[j][i] for the per-chain slot layout of dict.cu.
// Posterior-mean reconstruction: acc[u] += frame[u] (FP64); out = acc / count.
cudaError_t launch_mean_accumulate(long long n, const float* frame, double* acc, cudaStream_t s);
cudaError_t launch_mean_finish(long long n, const double* acc, long long count, float* out, cudaStream_t s);
// Rewrites obs, pos ([maxobs][N]) and nobs ([N]) into sweep order (slot s
// holds patch perm[s]).
cudaError_t launch_sweep_order(const Geom& g, int maxobs, const int* perm, const uint16_t* obs_in,
                               const uint16_t* nobs_in, const int* pos_in, uint16_t* obs_out, uint16_t* nobs_out,
                               int* pos_out, cudaStream_t s);
// Stable order of the patches by decreasing count (counting sort on the
// host): perm[s] for s < N, then perm[s] = s up to Npad.
void sweep_order_host(const uint16_t* nobs, long long N, long long Npad, int* perm);
cudaError_t launch_pos_slots(const Geom& g, const uint16_t* obs, const uint16_t* nobs, const uint32_t* Ibits,
                             const uint32_t* Ipre, const int* Rbase, int* pos, cudaStream_t s);
cudaError_t launch_dict_space(const DictSpaceArgs& a, const DictSpacePlan& plan, cudaStream_t s);
// The dense-statistics dictionary step (gram.cu): K <= 128.
bool gram_available(const Geom& g);
void gram_plan_items(const std::vector<int>& Rbase, int P, int seg, std::vector<int4>* items,
                     std::vector<int>* pitem_start, std::vector<int>* pitem_idx);
cudaError_t launch_xlist(const Geom& g, const int* Ilist, const int* Rbase, int max_slots, const int* imgoff,
                         const float* x, float* Xlist, cudaStream_t s);
cudaError_t launch_gram(const GramArgs& a, int grid, cudaStream_t s);   // statistics, then the draws
cudaError_t launch_geometry(const Geom& g, const uint8_t* mask_bytes, uint32_t* mask_bits, int* imgoff,
                            uint16_t* nobs, int* maxobs, unsigned long long* total, cudaStream_t s);
cudaError_t launch_fill_obs(const Geom& g, const uint32_t* mask_bits, const int* imgoff, uint16_t* obs, cudaStream_t s);
cudaError_t launch_slots(const Geom& g, const uint32_t* mask_bits, const int* imgoff, uint16_t* obs,
                         uint32_t* Ibits, uint32_t* Ipre, int* Icnt, int* Rbase, int* max_slots, cudaStream_t s);
cudaError_t launch_ilist(const Geom& g, const uint32_t* Ibits, const uint32_t* Ipre, const int* Rbase, int* Ilist,
                         cudaStream_t s);
cudaError_t launch_overlap_counts(const Geom& g, int* counts, cudaStream_t s);
// Per-patch reconstructions Y = W D (tensor cores for P <= 256, with Dc the
// recon_tc_operand_floats(g) scratch for their dictionary operands; else the
// FP32 ALU kernel) and the overlap-add gather into out; a device-side wait
// that gives up sets SENSAI_ETIMEOUT in *status.  reconstruct_launches(g)
// kernels.
cudaError_t launch_reconstruct(const Geom& g, const float* D, float* Dc, const float* W, float* Y, float* out,
                               int* status, cudaStream_t s);
int reconstruct_launches(const Geom& g);
bool recon_tc_available(const Geom& g);
size_t recon_tc_operand_floats(const Geom& g);   // 0 if the tensor-core form does not apply
cudaError_t launch_recon_tc(const Geom& g, const float* D, float* Dc, const float* W, float* Y, int* status,
                            cudaStream_t s);
cudaError_t launch_recon_alu(const Geom& g, const float* D, const float* W, float* Y, cudaStream_t s);
cudaError_t launch_init_state(const Geom& g, float* D, double* pi, float* lpi, DevScalars* sc,
                              unsigned long long seed, cudaStream_t s);
// scratch: kInitGammaEpsScratch doubles.
constexpr int kInitGammaEpsScratch = 3 * 256;
cudaError_t launch_init_gamma_eps(const Geom& g, const float* x, const uint32_t* mbits, DevScalars* sc,
                                  double* scratch, cudaStream_t s);
cudaError_t launch_code_stats(const Geom& g, const float* W, const uint32_t* Zb, const int* perm, int* m,
                              double* part_s2, cudaStream_t s);
cudaError_t launch_residual(const Geom& g, const float* x, const uint16_t* obs, const uint16_t* nobs,
                            const int* perm, const int* imgoff, const float* D, const float* W, const int* pos,
                            float* R, double* part_r2, cudaStream_t s);
cudaError_t launch_export_codes(const Geom& g, const float* W, const uint32_t* Zb, const int* perm, uint8_t* Z,
                                float* S, cudaStream_t s);
cudaError_t launch_import_codes(const Geom& g, const uint8_t* Z, const float* S, const int* perm, float* W,
                                uint32_t* Zb, cudaStream_t s);
cudaError_t launch_logit(int K, const double* pi, float* lpi, cudaStream_t s);

}  // namespace sensai
