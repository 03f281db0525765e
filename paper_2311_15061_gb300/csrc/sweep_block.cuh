// sweep_block.cuh -- one 8-atom block of the sparse-code sweep for one patch
// (the sparse-coding step of the BPFA section), shared by the kernel that
// holds the whole dictionary in shared memory (sweep.cu) and the kernel that
// streams it through in atom slices (sweep_tiled.cu).
//
// Per atom k of the block, with r the residual of patch i on its observed
// pixels (registers) and Dcol[p * ld] = d_kp (shared memory):
//   n = sum d_kp^2, h = sum d_kp r_p, g = h + w_old n, lam = gamma_s + gamma_eps n,
//   L = logit pi_k + 1/2 ln(gamma_s / lam) + gamma_eps^2 g^2 / (2 lam),
//   z = [x0 < floor(sigmoid(L) 2^32)], s | z=1 ~ N(gamma_eps g / lam, 1 / lam),
//   r -= d_k (w_new - w_old).
#pragma once
#include "internal.cuh"

namespace sensai {

// Per-thread constants of one sweep launch.
struct CodeConst {
    float gs, ge, half_log_gs, half_ge2;
};

__device__ __forceinline__ CodeConst code_const(const DevScalars* sc)
{
    CodeConst c;
    c.gs = (float)sc->gamma_s;
    c.ge = (float)sc->gamma_eps;
    c.half_log_gs = 0.5f * logf(c.gs);
    c.half_ge2 = 0.5f * c.ge * c.ge;
    return c;
}

// Work tallies of one thread (changed updates, their |Omega_i|, z = 1 draws).
struct CodeTally {
    unsigned int chg_n = 0, chg_obs = 0, act_n = 0;
};

// r -= sum_k d_k w_k over the block's non-zero stored weights.
template <int MAXOBS>
__device__ __forceinline__ void rebuild_block(const float* Dcol, const int (&offK)[MAXOBS], float (&r)[MAXOBS],
                                              int wmax, const W8& wb)
{
    const float* wv = wb.v;
#pragma unroll
    for (int kk = 0; kk < kAtomBlock; ++kk) {
        if (wv[kk] != 0.0f) {
            const float* dk = Dcol + kk;
#pragma unroll
            for (int g4 = 0; g4 < MAXOBS / 4; ++g4) {
                if (4 * g4 >= wmax) break;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = 4 * g4 + u;
                    r[j] = fmaf(-dk[offK[j]], wv[kk], r[j]);
                }
            }
        }
    }
}

// The block's atoms kbase .. kbase + kend - 1 in order; w0..w7 hold the
// block's stored weights on entry and its new weights on return (padding
// atoms keep their zero).  Dcol points at the block's first atom column.
template <int MAXOBS>
__device__ __forceinline__ void code_block(const float* Dcol, const float* lpi_blk, const int (&offK)[MAXOBS],
                                           float (&r)[MAXOBS], int wmax, int nobs, long long i, bool valid,
                                           int kbase, int kend, const CodeConst& c, const PhiloxKeys& keys,
                                           uint32_t t, uint32_t* Zb, int NW, unsigned int chunk, int lane,
                                           float& w0, float& w1, float& w2, float& w3,
                                           float& w4, float& w5, float& w6, float& w7, float& s2,
                                           CodeTally& tl)
{
#pragma unroll 1
    for (int kk = 0; kk < kAtomBlock; ++kk) {
        const int k = kbase + kk;
        float w_new = w0;
        if (kk < kend) {
            const float* dk = Dcol + kk;
            float n = 0.0f, h = 0.0f;
#pragma unroll
            for (int g4 = 0; g4 < MAXOBS / 4; ++g4) {
                if (4 * g4 >= wmax) break;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = 4 * g4 + u;
                    const float d = dk[offK[j]];
                    n = fmaf(d, d, n);
                    h = fmaf(d, r[j], h);
                }
            }
            const float w_old = w0;
            const float g = fmaf(w_old, n, h);
            const float lam = fmaf(c.ge, n, c.gs);
            const float rlam = __fdividef(1.0f, lam);
            const float L = lpi_blk[kk] + c.half_log_gs - 0.5f * __logf(lam) + c.half_ge2 * g * g * rlam;
            const float sig = __fdividef(1.0f, 1.0f + __expf(-L));
            // z = [x0 < floor(sig 2^32)] in 32-bit integers: the saturating
            // conversion gives the floor below 2^32, and sig = 1 (threshold
            // 2^32) accepts every word (a 64-bit conversion would run on the
            // FP64 pipe)
            const uint32_t thr = __float2uint_rz(sig * 4294967296.0f);
            const uint4 blk = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)k, t, kTagCodes), keys);
            const bool z = valid && (blk.x < thr || sig >= 1.0f);
            w_new = 0.0f;
            if (z) {
                w_new = fmaf(normal32(blk.y, blk.z), sqrtf(rlam), c.ge * g * rlam);
                s2 = fmaf(w_new, w_new, s2);
                tl.act_n += 1;
            }
            const float dw = w_new - w_old;
            if (dw != 0.0f) {
                tl.chg_n += 1;
                tl.chg_obs += (unsigned int)nobs;
#pragma unroll
                for (int g4 = 0; g4 < MAXOBS / 4; ++g4) {
                    if (4 * g4 >= wmax) break;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int j = 4 * g4 + u;
                        r[j] = fmaf(-dk[offK[j]], dw, r[j]);
                    }
                }
            }
            // the activity word; per-atom counts are summed from these words
            // after the sweep (a per-atom shared-memory count here would
            // serialise the next atom's dictionary loads behind its store)
            const uint32_t bal = __ballot_sync(0xffffffffu, z);
            if (lane == 0) Zb[(long long)k * NW + chunk] = bal;
        }
        w0 = w1; w1 = w2; w2 = w3; w3 = w4; w4 = w5; w5 = w6; w6 = w7; w7 = w_new;
    }
}

// End of a patch's sweep: scatter the residual to the dictionary step's
// layout (when kept) and publish the chunk's sum of s^2 and ||r||^2 (fixed-order warp sums).
template <int MAXOBS>
__device__ __forceinline__ void finish_patch(const SweepArgs& a, const float (&r)[MAXOBS], int wmax, int nobs,
                                             long long i, unsigned int chunk, int lane, float s2)
{
    const long long N = a.g.N;
    float r2 = 0.0f;
#pragma unroll
    for (int g4 = 0; g4 < MAXOBS / 4; ++g4) {
        if (4 * g4 >= wmax) break;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = 4 * g4 + u;
            if (j < nobs) {
                if (a.R) a.R[a.pos[(long long)j * N + i]] = r[j];
                r2 = fmaf(r[j], r[j], r2);
            }
        }
    }
    double s2d = warp_sum((double)s2);
    double r2d = warp_sum((double)r2);
    if (lane == 0) {
        a.part_s2[chunk] = s2d;
        a.part_r2[chunk] = r2d;
    }
}

// Observed pixels of patch i: within-patch offsets into a [p][ld] shared
// dictionary (padding slots point at the zero row p = P) and the frame values.
template <int MAXOBS>
__device__ __forceinline__ void gather_patch(const SweepArgs& a, long long i, int nobs, long long org, int ld,
                                             int (&offK)[MAXOBS], float (&r)[MAXOBS])
{
    const long long N = a.g.N;
    const int P = a.g.P;
#pragma unroll
    for (int j = 0; j < MAXOBS; ++j) {
        int p = P;
        float v = 0.0f;
        if (j < nobs) {
            p = a.obs[(long long)j * N + i];
            v = a.x[org + a.imgoff[p]];
        }
        offK[j] = p * ld;
        r[j] = v;
    }
}

// A warp's work counters, once per launch.
__device__ __forceinline__ void flush_counts(const SweepArgs& a, int lane, const CodeTally& tl)
{
    unsigned long long cn = tl.chg_n, co = tl.chg_obs, ca = tl.act_n;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cn += __shfl_down_sync(0xffffffffu, cn, o);
        co += __shfl_down_sync(0xffffffffu, co, o);
        ca += __shfl_down_sync(0xffffffffu, ca, o);
    }
    if (lane == 0 && (cn | ca)) {
        atomicAdd(&a.sc_out->chg_n, cn);
        atomicAdd(&a.sc_out->chg_obs, co);
        atomicAdd(&a.sc_out->act_n, ca);
    }
}

}  // namespace sensai
