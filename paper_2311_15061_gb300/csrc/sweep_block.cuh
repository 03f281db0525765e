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

// Lanes per patch.  Above 96 observed pixels a patch's pixels are split over
// a lane pair (pixel j on lane j % 2) so that each lane's residual still fits
// in registers.  The pair's partial sums are combined by one shuffle; both
// lanes then make the same draw, and only the even lane stores and counts.
// A warp then owns 16 patches, half of a 32-patch activity word.
template <int LANES>
struct PatchLanes {
    static_assert(LANES == 1 || LANES == 2, "1 or 2 lanes per patch");
    static constexpr int kPatchesPerWarp = 32 / LANES;
};

// Shared-memory offsets (in floats) of a lane's observed pixels.  At a
// per-lane capacity above 96 two 16-bit offsets share a register, which keeps
// the residual in registers up to 112; every offset is below 58,112 (a dictionary
// buffer fits in 227 KB), so 16 bits hold it.
template <int MAXOBS>
struct PixelOffsets {
    static constexpr bool kPacked = MAXOBS > 96;
    uint32_t v[kPacked ? MAXOBS / 2 : MAXOBS];
    __device__ __forceinline__ int operator[](int j) const
    {
        if (kPacked) return (int)((j & 1) ? (v[j >> 1] >> 16) : (v[j >> 1] & 0xffffu));
        return (int)v[j];
    }
    __device__ __forceinline__ void set(int j, int off)
    {
        if (kPacked) {
            if (j & 1) v[j >> 1] |= (uint32_t)off << 16;
            else v[j >> 1] = (uint32_t)off;
        } else {
            v[j] = (uint32_t)off;
        }
    }
};

// The 16 even-lane bits of a ballot, in order (lane 2m -> bit m).
__device__ __forceinline__ uint32_t even_lane_bits(uint32_t b)
{
    b &= 0x55555555u;
    b = (b | (b >> 1)) & 0x33333333u;
    b = (b | (b >> 2)) & 0x0F0F0F0Fu;
    b = (b | (b >> 4)) & 0x00FF00FFu;
    b = (b | (b >> 8)) & 0x0000FFFFu;
    return b;
}

// Work tallies of one thread (changed updates, their |Omega_i|, z = 1 draws).
struct CodeTally {
    unsigned int chg_n = 0, chg_obs = 0, act_n = 0;
};

// r -= sum_k d_k w_k over the block's non-zero stored weights.
template <int MAXOBS>
__device__ __forceinline__ void rebuild_block(const float* Dcol, const PixelOffsets<MAXOBS>& offK, float (&r)[MAXOBS],
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
// MAXOBS is per lane; unit is the warp's work unit (a 32-patch chunk, or with
// two lanes per patch a 16-patch half chunk).
template <int MAXOBS, int LANES = 1>
__device__ __forceinline__ void code_block(const float* Dcol, const float* lpi_blk, const PixelOffsets<MAXOBS>& offK,
                                           float (&r)[MAXOBS], int wmax, int nobs, long long i, bool valid,
                                           int kbase, int kend, const CodeConst& c, const PhiloxKeys& keys,
                                           uint32_t t, uint32_t* Zb, int NW, unsigned int unit, int lane,
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
            if (LANES == 2) {   // a + b on one lane, b + a on the other: identical sums
                n += __shfl_xor_sync(0xffffffffu, n, 1);
                h += __shfl_xor_sync(0xffffffffu, h, 1);
            }
            const bool owner = LANES == 1 || (lane & 1) == 0;
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
                if (owner) {
                    s2 = fmaf(w_new, w_new, s2);
                    tl.act_n += 1;
                }
            }
            const float dw = w_new - w_old;
            if (dw != 0.0f) {
                if (owner) {
                    tl.chg_n += 1;
                    tl.chg_obs += (unsigned int)nobs;
                }
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
            // the activity word; the pi draws sum the per-atom counts from
            // these words
            const uint32_t bal = __ballot_sync(0xffffffffu, z);
            if (LANES == 1) {
                if (lane == 0) Zb[(long long)k * NW + unit] = bal;
            } else if (lane == 0) {   // this half of the chunk's word (little-endian: patches 0-15 low)
                reinterpret_cast<uint16_t*>(Zb)[((long long)k * NW + (unit >> 1)) * 2 + (unit & 1)] =
                    (uint16_t)even_lane_bits(bal);
            }
        }
        w0 = w1; w1 = w2; w2 = w3; w3 = w4; w4 = w5; w5 = w6; w6 = w7; w7 = w_new;
    }
}

// End of a patch's sweep: scatter the residual to the dictionary step's
// layout (when kept) and publish the chunk's sum of s^2 and ||r||^2 (fixed-order warp sums).
// nobs is this lane's count of observed pixels (its pixel jj is the patch's
// pixel jj * LANES + half); the partials are per work unit.
template <int MAXOBS, int LANES = 1>
__device__ __forceinline__ void finish_patch(const SweepArgs& a, const float (&r)[MAXOBS], int wmax, int nobs,
                                             long long i, unsigned int unit, int lane, float s2)
{
    const long long N = a.g.N;
    const int half = LANES == 1 ? 0 : (lane & 1);
    float r2 = 0.0f;
#pragma unroll
    for (int g4 = 0; g4 < MAXOBS / 4; ++g4) {
        if (4 * g4 >= wmax) break;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int jj = 4 * g4 + u;
            if (jj < nobs) {
                if (a.R) a.R[a.pos[(long long)(jj * LANES + half) * N + i]] = r[jj];
                r2 = fmaf(r[jj], r[jj], r2);
            }
        }
    }
    double s2d = warp_sum((double)s2);
    double r2d = warp_sum((double)r2);
    if (lane == 0) {
        a.part_s2[unit] = s2d;
        a.part_r2[unit] = r2d;
    }
}

// Observed pixels of patch i: within-patch offsets into a [p][ld] shared
// dictionary (padding slots point at the zero row p = P) and the frame values.
// nobs: this lane's count; its pixel jj is the patch's pixel jj * LANES + half.
template <int MAXOBS, int LANES = 1>
__device__ __forceinline__ void gather_patch(const SweepArgs& a, long long i, int nobs, long long org, int ld,
                                             PixelOffsets<MAXOBS>& offK, float (&r)[MAXOBS], int half)
{
    const long long N = a.g.N;
    const int P = a.g.P;
#pragma unroll
    for (int jj = 0; jj < MAXOBS; ++jj) {
        int p = P;
        float v = 0.0f;
        if (jj < nobs) {
            p = a.obs[(long long)(jj * LANES + half) * N + i];
            v = a.x[org + a.imgoff[p]];
        }
        offK.set(jj, p * ld);
        r[jj] = v;
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
