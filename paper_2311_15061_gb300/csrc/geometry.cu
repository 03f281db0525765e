// geometry.cu -- patch geometry on the device (the N-D patch extraction of
// the "N-Dimensional Inpainting" section: patch shape B and stride S in every
// dimension of a frame of shape M), built once per sampling mask.
//
//  * mask bits: one bit per frame pixel;
//  * imgoff[p]: frame offset of within-patch pixel p (row-major over B);
//  * nobs[i], obs[j][i]: the observed within-patch pixels of patch i, in
//    increasing p, padded layout [maxobs][N] so a warp reads them coalesced;
//  * Ibits[p][w]: bit b of word w says patch 32w+b observes pixel p;
//    Ipre[p][w]: popcount of Ibits[p][0..w) -- the rank of a patch among the
//    patches observing p, i.e. its residual slot for the dictionary chains;
//  * Rbase[p]: start of pixel p's slots (exclusive scan of the counts);
//  * overlap counts c_q: per dimension floor(min(y, last)/S) -
//    ceil(max(0, y - B + 1)/S) + 1, multiplied over dimensions.
#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace sensai {

__global__ void pack_mask_kernel(long long nframe, const uint8_t* bytes, uint32_t* bits)
{
    const long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nw = (nframe + 31) / 32;
    if (w >= nw) return;
    uint32_t v = 0;
    for (int b = 0; b < 32; ++b) {
        const long long u = w * 32 + b;
        if (u < nframe && bytes[u]) v |= 1u << b;
    }
    bits[w] = v;
}

__global__ void pixel_offsets_kernel(Geom g, int* imgoff)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.P) return;
    int rem = p;
    long long off = 0;
    for (int d = g.ndim - 1; d >= 0; --d) {
        off += (long long)(rem % g.B[d]) * g.fs[d];
        rem /= g.B[d];
    }
    imgoff[p] = (int)off;
}

__device__ __forceinline__ bool mask_at(const uint32_t* bits, long long u)
{
    return (bits[u >> 5] >> (u & 31)) & 1u;
}

// misc[0] <- max_i |Omega_i|; *total (if given) += sum_i |Omega_i|.
__global__ void count_obs_kernel(Geom g, const uint32_t* mbits, const int* imgoff, uint16_t* nobs, int* maxobs,
                                 unsigned long long* total)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int c = 0;
    if (i < g.N) {
        const long long org = patch_origin(g, i);
        for (int p = 0; p < g.P; ++p) c += mask_at(mbits, org + imgoff[p]);
        nobs[i] = (uint16_t)c;
        atomicMax(maxobs, c);
    }
    if (total) {
        unsigned long long v = (unsigned long long)c;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(total, v);
    }
}

__global__ void fill_obs_kernel(Geom g, const uint32_t* mbits, const int* imgoff, uint16_t* obs)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    const long long org = patch_origin(g, i);
    int c = 0;
    for (int p = 0; p < g.P; ++p)
        if (mask_at(mbits, org + imgoff[p])) obs[(long long)(c++) * g.N + i] = (uint16_t)p;
}

// Grid: (ceil(NW / blockDim), P).
__global__ void ibits_kernel(Geom g, const uint32_t* mbits, const int* imgoff, uint32_t* Ibits)
{
    const long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int p = blockIdx.y;
    if (w >= g.NW) return;
    uint32_t v = 0;
    for (int b = 0; b < 32; ++b) {
        const long long i = w * 32 + b;
        if (i < g.N && mask_at(mbits, patch_origin(g, i) + imgoff[p])) v |= 1u << b;
    }
    Ibits[(long long)p * g.NW + w] = v;
}

// One CTA per pixel p: exclusive scan of popcounts over the words.
__global__ void __launch_bounds__(1024) iprefix_kernel(Geom g, const uint32_t* Ibits, uint32_t* Ipre, int* Icnt)
{
    __shared__ int warp_tot[32];
    __shared__ int carry;
    const int p = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (long long base = 0; base < g.NW; base += blockDim.x) {
        const long long w = base + threadIdx.x;
        const int v = w < g.NW ? __popc(Ibits[(long long)p * g.NW + w]) : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int n = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += n;
        }
        if (lane == 31) warp_tot[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const int nw = blockDim.x >> 5;
            int t = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int n = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += n;
            }
            if (lane < nw) warp_tot[lane] = t;  // inclusive over warps
        }
        __syncthreads();
        const int before = carry + (warp > 0 ? warp_tot[warp - 1] : 0) + incl - v;
        if (w < g.NW) Ipre[(long long)p * g.NW + w] = (uint32_t)before;
        __syncthreads();
        if (threadIdx.x == 0) carry += warp_tot[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) Icnt[p] = carry;
}

// Single thread: Rbase = exclusive scan of Icnt, Rbase[P] = total; largest count.
__global__ void rbase_kernel(int P, const int* Icnt, int* Rbase, int* max_slots)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    long long acc = 0;
    int mx = 0;
    for (int p = 0; p < P; ++p) {
        Rbase[p] = (int)acc;
        acc += Icnt[p];
        mx = Icnt[p] > mx ? Icnt[p] : mx;
    }
    Rbase[P] = (int)acc;
    *max_slots = mx;
}

__device__ __forceinline__ void cover_range(const Geom& g, int d, long long y, long long* first, long long* last)
{
    const long long lastp = (g.G[d] - 1) * g.S[d];
    long long lo = y - g.B[d] + 1;
    if (lo < 0) lo = 0;
    const long long hi = y < lastp ? y : lastp;
    *first = (lo + g.S[d] - 1) / g.S[d];
    *last = hi / g.S[d];
}

__global__ void overlap_counts_kernel(Geom g, int* counts)
{
    const long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= g.nframe) return;
    long long rem = u, c = 1;
    for (int d = g.ndim - 1; d >= 0; --d) {
        const long long y = rem % g.M[d];
        rem /= g.M[d];
        long long f, l;
        cover_range(g, d, y, &f, &l);
        c *= (l >= f) ? (l - f + 1) : 0;
    }
    counts[u] = (int)c;
}

// Overlap-add, gather form: pixel q averages Y[p][i] over the patches i that
// cover it, with p = q - origin(i).  Y holds every patch's reconstruction.
// The covering patches are visited in row-major order, eight addresses at a
// time, so that eight independent loads are in flight per thread; the sum
// takes them in that order.  NDIM is the frame's dimension count, so that
// the per-dimension state stays in registers.
constexpr int kGatherBatch = 8;

template <int NDIM>
__global__ void ola_gather_kernel(Geom g, const float* Y, float* out)
{
    const long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= g.nframe) return;
    long long y[NDIM], f[NDIM], l[NDIM], cur[NDIM];
    long long rem = u;
    bool empty = false;
#pragma unroll
    for (int d = NDIM - 1; d >= 0; --d) {
        y[d] = rem % g.M[d];
        rem /= g.M[d];
        cover_range(g, d, y[d], &f[d], &l[d]);
        empty = empty || l[d] < f[d];
        cur[d] = f[d];
    }
    if (empty) {
        out[u] = 0.0f;
        return;
    }
    float acc = 0.0f;
    int count = 0;
    bool more = true;
    while (more) {
        long long at[kGatherBatch];
#pragma unroll
        for (int j = 0; j < kGatherBatch; ++j) {
            at[j] = -1;
            if (!more) continue;
            long long i = 0;
            int p = 0;
#pragma unroll
            for (int d = 0; d < NDIM; ++d) {
                i = i * g.G[d] + cur[d];
                p = p * g.B[d] + (int)(y[d] - cur[d] * g.S[d]);
            }
            at[j] = (long long)p * g.N + i;
            ++count;
            bool carry = true;   // odometer step, last dimension fastest
#pragma unroll
            for (int d = NDIM - 1; d >= 0; --d) {
                if (carry) {
                    if (++cur[d] > l[d]) cur[d] = f[d];
                    else carry = false;
                }
            }
            more = !carry;
        }
        float v[kGatherBatch];
#pragma unroll
        for (int j = 0; j < kGatherBatch; ++j) v[j] = at[j] >= 0 ? __ldg(Y + at[j]) : 0.0f;
#pragma unroll
        for (int j = 0; j < kGatherBatch; ++j)
            if (at[j] >= 0) acc += v[j];
    }
    out[u] = acc / (float)count;
}

static cudaError_t launch_ola_gather(const Geom& g, const float* Y, float* out, cudaStream_t s);

// Residual position of observed pixel j of patch i in the per-pixel slot
// layout: slot Rbase[p] + rank of i among the patches observing p.
__global__ void pos_slots_kernel(Geom g, const uint16_t* obs, const uint16_t* nobs, const uint32_t* Ibits,
                                 const uint32_t* Ipre, const int* Rbase, int* pos)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    const long long w = i >> 5;
    const uint32_t below = (1u << (i & 31)) - 1u;
    for (int j = 0; j < (int)nobs[i]; ++j) {
        const int p = obs[(long long)j * g.N + i];
        const long long wd = (long long)p * g.NW + w;
        pos[(long long)j * g.N + i] = Rbase[p] + (int)Ipre[wd] + __popc(Ibits[wd] & below);
    }
}

// Slot -> patch list of every pixel p: Ilist[Rbase[p] + rank] = the patches
// observing p in increasing index (one thread per (word, pixel)).
__global__ void ilist_kernel(Geom g, const uint32_t* Ibits, const uint32_t* Ipre, const int* Rbase, int* Ilist)
{
    const long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int p = blockIdx.y;
    if (w >= g.NW) return;
    uint32_t bits = Ibits[(long long)p * g.NW + w];
    int slot = Rbase[p] + (int)Ipre[(long long)p * g.NW + w];
    while (bits) {
        const int b = __ffs(bits) - 1;
        bits &= bits - 1u;
        Ilist[slot++] = (int)(w * 32 + b);
    }
}

// Per-patch reconstruction Y[p][i] = sum_k z_ik w_ik d_kp on the FP32 ALUs, for
// patches of more than 256 pixels (the tensor-core form covers the rest).  One thread per
// patch, 32 pixels at a time; the dictionary chunk is read with warp-uniform
// (broadcast) shared-memory loads.
__global__ void __launch_bounds__(256) patch_recon_kernel(Geom g, const float* D, const float* W, float* Y)
{
    extern __shared__ float Ds[];  // Kpad x 32: columns p0 .. p0 + 31 of D, zero past P and K
    const int K = g.K, P = g.P, KB = g.KB;
    const int lane = threadIdx.x & 31;
    const long long chunk = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const bool on = chunk < g.NW;
    const long long i = chunk * 32 + lane;
    for (int p0 = 0; p0 < P; p0 += 32) {
        __syncthreads();   // the previous slab is consumed
        for (int idx = threadIdx.x; idx < KB * kAtomBlock * 32; idx += blockDim.x) {
            const int k = idx >> 5, q = idx & 31;
            Ds[idx] = (k < K && p0 + q < P) ? D[(long long)k * P + p0 + q] : 0.0f;
        }
        __syncthreads();
        if (!on) continue;
        float acc[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) acc[q] = 0.0f;
        for (int kb = 0; kb < KB; ++kb) {
            const W8 wb = load_w8(W + wblock(g, kb, i));
#pragma unroll
            for (int kk = 0; kk < kAtomBlock; ++kk) {
                const float w = wb.v[kk];   // zero for padding atoms
                if (w != 0.0f) {
                    const float* dk = Ds + (kb * kAtomBlock + kk) * 32;
#pragma unroll
                    for (int q = 0; q < 32; ++q) acc[q] = fmaf(dk[q], w, acc[q]);
                }
            }
        }
        if (i < g.N) {
#pragma unroll
            for (int q = 0; q < 32; ++q)
                if (p0 + q < P) Y[(long long)(p0 + q) * g.N + i] = acc[q];
        }
    }
}

}  // namespace sensai

namespace sensai {

// Posterior-mean reconstruction: acc += frame (FP64), then out = acc / count.
__global__ void mean_accumulate_kernel(long long n, const float* frame, double* acc)
{
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < n;
         u += (long long)gridDim.x * blockDim.x)
        acc[u] += (double)frame[u];
}

__global__ void mean_finish_kernel(long long n, const double* acc, double count, float* out)
{
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < n;
         u += (long long)gridDim.x * blockDim.x)
        out[u] = (float)(acc[u] / count);
}

// The code sweep's tables in sweep order: slot s holds patch perm[s].
// obs and pos ([maxobs][N]) and nobs ([N]) are gathered row by row.
__global__ void sweep_order_kernel(Geom g, int maxobs, const int* perm, const uint16_t* obs_in,
                                   const uint16_t* nobs_in, const int* pos_in, uint16_t* obs_out,
                                   uint16_t* nobs_out, int* pos_out)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long rows = (long long)maxobs + 1;
    if (idx >= rows * g.N) return;
    const long long j = idx / g.N, slot = idx - j * g.N;
    const long long i = perm[slot];
    if (j == maxobs) {
        nobs_out[slot] = nobs_in[i];
    } else {
        obs_out[j * g.N + slot] = obs_in[j * g.N + i];
        pos_out[j * g.N + slot] = pos_in[j * g.N + i];
    }
}

static inline unsigned int blocks_for(long long n, int threads)
{
    return (unsigned int)((n + threads - 1) / threads);
}

cudaError_t launch_geometry(const Geom& g, const uint8_t* mask_bytes, uint32_t* mask_bits, int* imgoff,
                            uint16_t* nobs, int* maxobs, unsigned long long* total, cudaStream_t s)
{
    const long long nmw = (g.nframe + 31) / 32;
    pack_mask_kernel<<<blocks_for(nmw, 256), 256, 0, s>>>(g.nframe, mask_bytes, mask_bits);
    pixel_offsets_kernel<<<blocks_for(g.P, 256), 256, 0, s>>>(g, imgoff);
    count_obs_kernel<<<blocks_for(g.N, 256), 256, 0, s>>>(g, mask_bits, imgoff, nobs, maxobs, total);
    return cudaGetLastError();
}

cudaError_t launch_fill_obs(const Geom& g, const uint32_t* mask_bits, const int* imgoff, uint16_t* obs, cudaStream_t s)
{
    fill_obs_kernel<<<blocks_for(g.N, 256), 256, 0, s>>>(g, mask_bits, imgoff, obs);
    return cudaGetLastError();
}

cudaError_t launch_slots(const Geom& g, const uint32_t* mask_bits, const int* imgoff, uint16_t* obs,
                         uint32_t* Ibits, uint32_t* Ipre, int* Icnt, int* Rbase, int* max_slots, cudaStream_t s)
{
    fill_obs_kernel<<<blocks_for(g.N, 256), 256, 0, s>>>(g, mask_bits, imgoff, obs);
    ibits_kernel<<<dim3(blocks_for(g.NW, 256), g.P), 256, 0, s>>>(g, mask_bits, imgoff, Ibits);
    iprefix_kernel<<<g.P, 1024, 0, s>>>(g, Ibits, Ipre, Icnt);
    rbase_kernel<<<1, 32, 0, s>>>(g.P, Icnt, Rbase, max_slots);
    return cudaGetLastError();
}

cudaError_t launch_ilist(const Geom& g, const uint32_t* Ibits, const uint32_t* Ipre, const int* Rbase, int* Ilist,
                         cudaStream_t s)
{
    ilist_kernel<<<dim3(blocks_for(g.NW, 256), g.P), 256, 0, s>>>(g, Ibits, Ipre, Rbase, Ilist);
    return cudaGetLastError();
}

cudaError_t launch_pos_slots(const Geom& g, const uint16_t* obs, const uint16_t* nobs, const uint32_t* Ibits,
                             const uint32_t* Ipre, const int* Rbase, int* pos, cudaStream_t s)
{
    pos_slots_kernel<<<blocks_for(g.N, 256), 256, 0, s>>>(g, obs, nobs, Ibits, Ipre, Rbase, pos);
    return cudaGetLastError();
}

cudaError_t launch_overlap_counts(const Geom& g, int* counts, cudaStream_t s)
{
    overlap_counts_kernel<<<blocks_for(g.nframe, 256), 256, 0, s>>>(g, counts);
    return cudaGetLastError();
}

cudaError_t launch_recon_alu(const Geom& g, const float* D, const float* W, float* Y, cudaStream_t s)
{
    const int smem = (int)(sizeof(float) * (size_t)g.KB * kAtomBlock * 32);
    cudaError_t e = cudaFuncSetAttribute((void*)patch_recon_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    patch_recon_kernel<<<blocks_for(g.NW, 8), 256, smem, s>>>(g, D, W, Y);
    return cudaGetLastError();
}

int reconstruct_launches(const Geom& g) { return recon_tc_available(g) ? 3 : 2; }

cudaError_t launch_reconstruct(const Geom& g, const float* D, float* Dc, const float* W, float* Y, float* out,
                               int* status, cudaStream_t s)
{
    cudaError_t e = recon_tc_available(g) ? launch_recon_tc(g, D, Dc, W, Y, status, s)
                                          : launch_recon_alu(g, D, W, Y, s);
    if (e != cudaSuccess) return e;
    return launch_ola_gather(g, Y, out, s);
}

static cudaError_t launch_ola_gather(const Geom& g, const float* Y, float* out, cudaStream_t s)
{
    const unsigned int blocks = blocks_for(g.nframe, 256);
    switch (g.ndim) {
    case 1: ola_gather_kernel<1><<<blocks, 256, 0, s>>>(g, Y, out); break;
    case 2: ola_gather_kernel<2><<<blocks, 256, 0, s>>>(g, Y, out); break;
    case 3: ola_gather_kernel<3><<<blocks, 256, 0, s>>>(g, Y, out); break;
    case 4: ola_gather_kernel<4><<<blocks, 256, 0, s>>>(g, Y, out); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace sensai

namespace sensai {

void sweep_order_host(const uint16_t* nobs, long long N, long long Npad, int* perm)
{
    // counting sort, largest counts first (a warp's work is set by its
    // largest count; the heaviest warps start first, so the tail of a sweep
    // is light); ties keep patch order
    std::vector<long long> start(65537, 0);
    for (long long i = 0; i < N; ++i) ++start[65535 - nobs[i] + 1];
    for (int v = 1; v <= 65536; ++v) start[v] += start[v - 1];
    for (long long i = 0; i < N; ++i) perm[start[65535 - nobs[i]]++] = (int)i;
    for (long long s = N; s < Npad; ++s) perm[s] = (int)s;
}

cudaError_t launch_mean_accumulate(long long n, const float* frame, double* acc, cudaStream_t s)
{
    const long long blocks = std::min<long long>((n + 255) / 256, 4096);
    mean_accumulate_kernel<<<(unsigned int)blocks, 256, 0, s>>>(n, frame, acc);
    return cudaGetLastError();
}

cudaError_t launch_mean_finish(long long n, const double* acc, long long count, float* out, cudaStream_t s)
{
    const long long blocks = std::min<long long>((n + 255) / 256, 4096);
    mean_finish_kernel<<<(unsigned int)blocks, 256, 0, s>>>(n, acc, (double)count, out);
    return cudaGetLastError();
}

cudaError_t launch_sweep_order(const Geom& g, int maxobs, const int* perm, const uint16_t* obs_in,
                               const uint16_t* nobs_in, const int* pos_in, uint16_t* obs_out, uint16_t* nobs_out,
                               int* pos_out, cudaStream_t s)
{
    const long long n = ((long long)maxobs + 1) * g.N;
    sweep_order_kernel<<<(unsigned int)((n + 255) / 256), 256, 0, s>>>(g, maxobs, perm, obs_in, nobs_in, pos_in,
                                                                       obs_out, nobs_out, pos_out);
    return cudaGetLastError();
}

}  // namespace sensai
