// sweep_block.cuh -- one 8-atom block of the sparse-code sweep for one patch
// (the sparse-coding step of the BPFA section), shared by the kernel that
// holds the whole dictionary in shared memory (sweep.cu) and the kernel that
// streams it through in atom slices (sweep_tiled.cu).
//
// Per atom k of the block, with r the residual of patch i on its observed
// pixels (registers) and d_k the atom's column in shared memory:
//   n = sum d_kp^2, h = sum d_kp r_p, g = h + w_old n, lam = gamma_s + gamma_eps n,
//   L = logit pi_k + 1/2 ln(gamma_s / lam) + gamma_eps^2 g^2 / (2 lam),
//   z = [x0 < floor(sigmoid(L) 2^32)], s | z=1 ~ N(gamma_eps g / lam, 1 / lam),
//   r -= d_k (w_new - w_old).
//
// Instruction economy (the sweep is bound by instruction issue):
//  * a lane's pixels are processed in pairs with packed FP32x2 FMAs: one
//    instruction updates (n, h) partial sums or two residual entries;
//  * one pass over the pixels applies atom k-1's rank-1 update and forms
//    atom k's n and h, so the dictionary columns are read once per atom and
//    pixel for both;
//  * the block's 8 atoms are unrolled at compile time, so each dictionary
//    read is one shared load at a register address plus an immediate column
//    offset (the per-pixel row addresses are rebased once per block);
//  * one Philox block and one Box-Muller pair serve two atoms (2m, 2m + 1);
//    the next pair's are computed inside atom 2m's scalar chain, on which
//    they do not depend.
#pragma once
#include <type_traits>

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

// The dictionary in shared memory, in either kernel: rows p = 0..P (row P is
// all zero: padded pixel slots point at it), columns 0..: column 0 is all
// zero, atom kk of a buffer is column 1 + kk.  A block's atoms 0..7 are
// columns c0 .. c0 + 7 and column c0 - 1 is the previous atom (or the zero
// column).  Byte pitch = 4 x (odd number of columns).
constexpr int kDictColumnOffset = 1;

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// A shared-memory load at a byte address of the shared window.  volatile
// keeps the compiler front end from merging or moving it across barriers and
// the bulk copies that refill a buffer; the assembler still schedules it.
__device__ __forceinline__ float lds_f32(uint32_t addr)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
    return v;
}

// Shared-memory addresses of a lane's observed pixels (padding slots point
// at the zero row).  Up to 96 per lane: one register per pixel holding the
// byte address of (row p_j, the current block's first atom column), rebased
// when the block moves.  Above 96 (two lanes per patch, 112 or 128 per lane)
// two 16-bit row indices share a register and the address is formed per load.
template <int MAXOBS>
struct PixelAddr {
    static constexpr bool kPacked = MAXOBS > 96;
    uint32_t v[kPacked ? MAXOBS / 2 : MAXOBS];
    uint32_t base;    // byte address of (row 0, the current block's first atom column)
    uint32_t pitch;   // bytes per dictionary row

    __device__ __forceinline__ void set(int j, int p)
    {
        if (kPacked) {
            if (j & 1) v[j >> 1] |= (uint32_t)p << 16;
            else v[j >> 1] = (uint32_t)p;
        } else {
            v[j] = base + (uint32_t)p * pitch;
        }
    }
    // Atom column offset col (-1 .. 7, a compile-time constant after
    // unrolling) of the current block, pixel j.
    __device__ __forceinline__ float load(int j, int col) const
    {
        if (kPacked) {
            const uint32_t p = (j & 1) ? (v[j >> 1] >> 16) : (v[j >> 1] & 0xffffu);
            return lds_f32(base + p * pitch + 4 * col);
        }
        return lds_f32(v[j] + 4 * col);
    }
    // Move to a block whose first atom column is at nb (pixels below wmax).
    __device__ __forceinline__ void rebase(uint32_t nb, int wmax)
    {
        if (!kPacked) {
            const uint32_t dlt = nb - base;
#pragma unroll
            for (int g4 = 0; g4 < MAXOBS / 4; ++g4) {
                if (4 * g4 >= wmax) break;
#pragma unroll
                for (int u = 0; u < 4; ++u) v[4 * g4 + u] += dlt;
            }
        }
        base = nb;
    }
};

// A lane's residual on its observed pixels, in pixel pairs (2q, 2q + 1).
template <int MAXOBS>
struct Resid {
    static_assert(MAXOBS % 4 == 0, "pixel capacity in groups of 4");
    float2 v[MAXOBS / 2];
    __device__ __forceinline__ float get(int j) const { return (j & 1) ? v[j >> 1].y : v[j >> 1].x; }
    __device__ __forceinline__ void put(int j, float x)
    {
        if (j & 1) v[j >> 1].y = x;
        else v[j >> 1].x = x;
    }
};

// One pass over a lane's pixels (groups of 4 up to the warp's largest count):
//   UPD: r -= d_PREV (dw)              (an atom's rank-1 update)
//   NH:  n = sum d_CUR^2, h = sum d_CUR r  (after the update)
// PREV and CUR are column offsets from the block's first atom column.
// Two accumulator pairs (the group's first and second pixel pair) halve the
// dependent chains.
template <int MAXOBS, int PREV, int CUR, bool UPD, bool NH>
__device__ __forceinline__ void pixel_pass(const PixelAddr<MAXOBS>& ad, Resid<MAXOBS>& r, int wmax, float dw,
                                           float& n, float& h)
{
    float2 nn[2] = {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};
    float2 hh[2] = {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};
    const float2 mdw = make_float2(-dw, -dw);
#pragma unroll
    for (int g4 = 0; g4 < MAXOBS / 4; ++g4) {
        if (4 * g4 >= wmax) break;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int q = 2 * g4 + u;
            if (UPD) {
                const float2 dp = make_float2(ad.load(2 * q, PREV), ad.load(2 * q + 1, PREV));
                r.v[q] = __ffma2_rn(dp, mdw, r.v[q]);
            }
            if (NH) {
                const float2 dc = make_float2(ad.load(2 * q, CUR), ad.load(2 * q + 1, CUR));
                nn[u] = __ffma2_rn(dc, dc, nn[u]);
                hh[u] = __ffma2_rn(dc, r.v[q], hh[u]);
            }
        }
    }
    n = (nn[0].x + nn[0].y) + (nn[1].x + nn[1].y);
    h = (hh[0].x + hh[0].y) + (hh[1].x + hh[1].y);
}

// r -= sum_k d_k w_k over the block's non-zero stored weights (the residual
// rebuild at the start of a sweep); ad is at the block.
template <int MAXOBS>
__device__ __forceinline__ void rebuild_block(const PixelAddr<MAXOBS>& ad, Resid<MAXOBS>& r, int wmax, const W8& wb)
{
#pragma unroll
    for (int kk = 0; kk < kAtomBlock; ++kk) {
        const float w = wb.v[kk];
        if (w != 0.0f) {
            const float2 mw = make_float2(-w, -w);
#pragma unroll
            for (int g4 = 0; g4 < MAXOBS / 4; ++g4) {
                if (4 * g4 >= wmax) break;
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int q = 2 * g4 + u;
                    const float2 d = make_float2(ad.load(2 * q, kk), ad.load(2 * q + 1, kk));
                    r.v[q] = __ffma2_rn(d, mw, r.v[q]);
                }
            }
        }
    }
}

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
    unsigned int chg_n_patch0 = 0;   // chg_n when the current patch began
    unsigned int rb_obs = 0;   // in-sweep residual rebuild: this lane's pixels x non-zero stored weights
};

// At a patch's start and end: chg_obs gains |Omega_i| per changed update of
// the patch (counted in chg_n during its atoms).
__device__ __forceinline__ void begin_patch_counts(CodeTally& tl) { tl.chg_n_patch0 = tl.chg_n; }
__device__ __forceinline__ void end_patch_counts(CodeTally& tl, int nobs)
{
    tl.chg_obs += (tl.chg_n - tl.chg_n_patch0) * (unsigned int)nobs;
}

// Non-zero weights of a stored 8-atom block.
__device__ __forceinline__ unsigned int w8_nonzero(const W8& wb)
{
    unsigned int c = 0;
#pragma unroll
    for (int kk = 0; kk < kAtomBlock; ++kk) c += wb.v[kk] != 0.0f ? 1u : 0u;
    return c;
}

// The random numbers of the code draws of atoms 2m and 2m + 1: one Philox
// block at counter (i, m, t, codes); word k % 2 decides z_ik, words 2-3 give
// one Box-Muller pair (the cosine normal for the even atom, the sine one for
// the odd atom).
struct CodePair {
    uint32_t x0[2];
    float nrm[2];
};

__device__ __forceinline__ CodePair code_pair(long long i, int m, uint32_t t, const PhiloxKeys& keys)
{
    const uint4 blk = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)m, t, kTagCodes), keys);
    CodePair cp;
    cp.x0[0] = blk.x;
    cp.x0[1] = blk.y;
    normal32_pair(blk.z, blk.w, cp.nrm[0], cp.nrm[1]);
    return cp;
}

// Per-lane facts of the patch being swept.
struct LanePatch {
    long long i;        // patch index (the Philox counter)
    bool valid;         // i < N
    int nobs;           // |Omega_i| (counts of changed updates)
    unsigned int unit;  // the warp's work unit (activity word, or its 16-bit half)
    int lane;
    int wmax;           // the warp's largest per-lane pixel count
};

// Carried from one atom to the next: the pending rank-1 update of the
// previous atom, the random numbers of the current atom pair and, from the
// pair's even atom on, those of the next pair.
struct AtomCarry {
    float dw;
    CodePair cur, nxt;
};

// The block's atoms kbase .. kbase + 7 in order (atoms >= K are padding: their
// columns are zero and their z is 0).  ad is at the block.  On entry
// carry.dw is the previous atom's update, still to be applied (FUSE: its
// column is the one before the block; otherwise it must be 0), and
// carry.cur the random numbers of atoms kbase, kbase + 1.  wb holds the stored weights;
// on return, the new ones, and carry.dw atom kbase + 7's update, applied to r
// unless FUSE (then the next block's first pass applies it).  Returns whether
// a weight of the block changed.
template <int MAXOBS, int LANES, bool FUSE>
__device__ __forceinline__ bool code_block(const PixelAddr<MAXOBS>& ad, Resid<MAXOBS>& r, const float* lpi_blk,
                                           const LanePatch& lp, int kbase, int K, const CodeConst& c,
                                           const PhiloxKeys& keys, uint32_t t, uint32_t* Zb, int NW, W8& wb,
                                           AtomCarry& carry, float& s2, CodeTally& tl)
{
    bool changed = false;
    auto atom = [&](auto KKc) {
        constexpr int KK = decltype(KKc)::value;
        const int k = kbase + KK;
        float n, h;
        if constexpr (KK == 0 && !FUSE) pixel_pass<MAXOBS, -1, KK, false, true>(ad, r, lp.wmax, 0.0f, n, h);
        else pixel_pass<MAXOBS, KK - 1, KK, true, true>(ad, r, lp.wmax, carry.dw, n, h);
        if (LANES == 2) {   // a + b on one lane, b + a on the other: identical sums
            n += __shfl_xor_sync(0xffffffffu, n, 1);
            h += __shfl_xor_sync(0xffffffffu, h, 1);
        }
        // kbase is a multiple of 8, so k and KK have the same parity
        const uint32_t x0 = carry.cur.x0[KK & 1];
        const float nrm = carry.cur.nrm[KK & 1];
        if constexpr ((KK & 1) == 0)
            carry.nxt = code_pair(lp.i, (k >> 1) + 1, t, keys);   // the next pair's, independent of this chain
        else
            carry.cur = carry.nxt;
        const bool owner = LANES == 1 || (lp.lane & 1) == 0;
        const float w_old = wb.v[KK];
        const float g = fmaf(w_old, n, h);
        const float lam = fmaf(c.ge, n, c.gs);
        const float rlam = __fdividef(1.0f, lam);
        const float grl = g * rlam;
        // lpi_blk holds logit(pi_k) + ln(gamma_s) / 2 (staged per launch)
        const float L = fmaf(c.half_ge2 * g, grl, fmaf(-0.5f, __logf(lam), lpi_blk[KK]));
        const float sig = __fdividef(1.0f, 1.0f + __expf(-L));
        // z = [x0 < floor(sig 2^32)] in 32-bit integers: the saturating
        // conversion gives the floor below 2^32, and sig = 1 (threshold
        // 2^32) accepts every word (a 64-bit conversion would run on the
        // FP64 pipe)
        const uint32_t thr = __float2uint_rz(sig * 4294967296.0f);
        const bool z = lp.valid && k < K && (x0 < thr || sig >= 1.0f);
        // branch-free from here to the ballot: one basic block per atom lets
        // the next atom's random numbers interleave with this chain
        const float w_new = z ? fmaf(nrm, rsqrtf(lam), c.ge * grl) : 0.0f;
        const bool zo = z && owner;
        s2 = zo ? fmaf(w_new, w_new, s2) : s2;
        tl.act_n += zo ? 1u : 0u;
        const float dw = w_new - w_old;
        const bool chg = dw != 0.0f;
        changed = changed || chg;
        const bool co = chg && owner;
        tl.chg_n += co ? 1u : 0u;   // chg_obs: once per patch (the caller's add_changed_obs)
        wb.v[KK] = w_new;
        carry.dw = dw;
        // the activity word; the pi draws sum the per-atom counts from it
        const uint32_t bal = __ballot_sync(0xffffffffu, z);
        if (k < K && lp.lane == 0) {
            if (LANES == 1) Zb[(long long)k * NW + lp.unit] = bal;
            else   // this half of the chunk's word (little-endian: patches 0-15 low)
                reinterpret_cast<uint16_t*>(Zb)[((long long)k * NW + (lp.unit >> 1)) * 2 + (lp.unit & 1)] =
                    (uint16_t)even_lane_bits(bal);
        }
    };
    atom(std::integral_constant<int, 0>{});
    atom(std::integral_constant<int, 1>{});
    atom(std::integral_constant<int, 2>{});
    atom(std::integral_constant<int, 3>{});
    atom(std::integral_constant<int, 4>{});
    atom(std::integral_constant<int, 5>{});
    atom(std::integral_constant<int, 6>{});
    atom(std::integral_constant<int, 7>{});
    if constexpr (!FUSE) {   // atom 7's update now
        float n, h;
        pixel_pass<MAXOBS, 7, 7, true, false>(ad, r, lp.wmax, carry.dw, n, h);
        carry.dw = 0.0f;
    }
    return changed;
}

// Applies the pending update of the current block's last atom (the end of a
// fused sweep).
template <int MAXOBS>
__device__ __forceinline__ void apply_update(const PixelAddr<MAXOBS>& ad, Resid<MAXOBS>& r, int wmax, float dw)
{
    float n, h;
    pixel_pass<MAXOBS, 7, 7, true, false>(ad, r, wmax, dw, n, h);
}

// End of a patch's sweep: scatter the residual to the dictionary step's
// layout (when kept) and publish the unit's sum of s^2 and ||r||^2
// (fixed-order warp sums).  nl is this lane's count of observed pixels (its
// pixel jj is the patch's pixel jj * LANES + half); slot is the patch's
// position in the sweep order (the row of the position table).
template <int MAXOBS, int LANES = 1>
__device__ __forceinline__ void finish_patch(const SweepArgs& a, const Resid<MAXOBS>& r, int wmax, int nl,
                                             long long slot, unsigned int unit, int lane, float s2)
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
            if (jj < nl) {
                const float v = r.get(jj);
                if (a.R) a.R[a.pos[(long long)(jj * LANES + half) * N + slot]] = v;
                r2 = fmaf(v, v, r2);
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

// Observed pixels of the patch at sweep position slot (patch i): the pixel
// addresses (padding slots at the zero row p = P) and either the frame values
// (from_resid false: the caller rebuilds the residual) or the current
// residual kept by the previous phase.
// nl: this lane's count; its pixel jj is the patch's pixel jj * LANES + half.
template <int MAXOBS, int LANES = 1>
__device__ __forceinline__ void gather_patch(const SweepArgs& a, long long slot, int nl, long long org,
                                             PixelAddr<MAXOBS>& ad, Resid<MAXOBS>& r, int half, bool from_resid)
{
    const long long N = a.g.N;
    const int P = a.g.P;
#pragma unroll
    for (int jj = 0; jj < MAXOBS; ++jj) {
        int p = P;
        float v = 0.0f;
        if (jj < nl) {
            const long long e = (long long)(jj * LANES + half) * N + slot;
            p = a.obs[e];
            v = from_resid ? a.R_in[a.pos[e]] : a.x[org + a.imgoff[p]];
        }
        ad.set(jj, p);
        r.put(jj, v);
    }
}

// Sweep position slot -> patch index (identity without a sweep order).
__device__ __forceinline__ long long slot_patch(const SweepArgs& a, long long slot)
{
    return a.perm ? (long long)a.perm[slot] : slot;
}

// A warp's work counters, once per launch.
__device__ __forceinline__ void flush_counts(const SweepArgs& a, int lane, const CodeTally& tl)
{
    unsigned long long cn = tl.chg_n, co = tl.chg_obs, ca = tl.act_n, rb = tl.rb_obs;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cn += __shfl_down_sync(0xffffffffu, cn, o);
        co += __shfl_down_sync(0xffffffffu, co, o);
        ca += __shfl_down_sync(0xffffffffu, ca, o);
        rb += __shfl_down_sync(0xffffffffu, rb, o);
    }
    if (lane == 0 && (cn | ca | rb)) {
        atomicAdd(&a.sc_out->chg_n, cn);
        atomicAdd(&a.sc_out->chg_obs, co);
        atomicAdd(&a.sc_out->act_n, ca);
        atomicAdd(&a.sc_out->rb_obs, rb);
    }
}

}  // namespace sensai
