// dict.cu -- the dictionary sweep (the dictionary-learning step of the BPFA
// section), atoms in order k = 0..K-1, each d_kp from its conjugate Gaussian
// given every other atom's current value:
//   Lambda_kp = P + gamma_eps sum_{i: z_ik=1, p in Omega_i} w_ik^2
//   mu_kp     = gamma_eps / Lambda_kp * sum_{i: z_ik=1, p in Omega_i} w_ik r^{-k}_ip
//   d_kp      = mu_kp + Lambda_kp^-1/2 BoxMuller(Philox(p, k, t, DICT))
// with r^{-k} = r + d_k w_k the residual that leaves atom k out; afterwards the
// residual takes the new atom: r -= (d_new - d_old) w_k.
//
// Neither sum couples different pixels p, so the sweep splits into P
// independent chains of K sequential draws.  GB300 mapping: one CTA per pixel
// p keeps that pixel's residual slots (one per patch observing p) in shared
// memory for all K atoms.  Each thread owns fixed 32-patch words; per atom it
// ANDs the atom's activity word with the pixel's observation word, applies
// the previous atom's update to its own slots and accumulates the two sums,
// which a fixed-order block reduction (FP32 within warps, FP64 across warps)
// turns into one draw; the K normals are drawn up front.  Two barriers per
// atom, no global synchronisation, no float atomics: results are
// deterministic.
#include "internal.cuh"

namespace sensai {

constexpr int kDictThreads = 1024;
constexpr int kDictMaxK = 1024;

// WPT: 32-patch words per thread (NW <= WPT * kDictThreads), kept in registers.
template <int WPT, bool SMEM_R>
__global__ void __launch_bounds__(kDictThreads, 1) dict_kernel(const DictArgs a)
{
    extern __shared__ float rsm[];
    __shared__ float red_a[kDictThreads / 32], red_b[kDictThreads / 32];
    __shared__ double xi[kDictMaxK];
    __shared__ float s_delta;
    const int p = blockIdx.x;
    const int K = a.g.K, P = a.g.P, NW = a.g.NW;
    const long long N = a.g.N;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int base = a.Rbase[p];
    const int cnt = a.Rbase[p + 1] - base;
    float* Rp = SMEM_R ? rsm : a.R + base;
    if (SMEM_R)
        for (int s = threadIdx.x; s < cnt; s += blockDim.x) rsm[s] = a.R[base + s];
    // the K normals of this pixel's draws, off the sequential path
    const uint2 key = seed_key(a.seed);
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const uint4 blk = philox4x32_10(make_uint4((uint32_t)p, (uint32_t)k, a.t, kTagDict), key);
        xi[k] = normal64(blk.x, blk.y);
    }
    __syncthreads();

    const uint32_t* Ib = a.Ibits + (long long)p * NW;
    const uint32_t* Ip = a.Ipre + (long long)p * NW;
    const double ge = a.sc->gamma_eps;
    uint32_t ib[WPT], zprev[WPT];
    int pre[WPT];
#pragma unroll
    for (int m = 0; m < WPT; ++m) {
        const int j = threadIdx.x + m * kDictThreads;
        ib[m] = j < NW ? Ib[j] : 0u;
        pre[m] = j < NW ? (int)Ip[j] : 0;
        zprev[m] = 0u;
    }
    float delta_prev = 0.0f;

    for (int k = 0; k <= K; ++k) {
        uint32_t zcur[WPT];
#pragma unroll
        for (int m = 0; m < WPT; ++m) {
            const int j = threadIdx.x + m * kDictThreads;
            zcur[m] = (k < K && ib[m]) ? (a.Zb[(long long)k * NW + j] & ib[m]) : 0u;
        }
        float acc_a = 0.0f, acc_b = 0.0f;
#pragma unroll
        for (int m = 0; m < WPT; ++m) {
            const int j = threadIdx.x + m * kDictThreads;
            uint32_t bits = delta_prev != 0.0f ? zprev[m] : 0u;
            if (bits) {
                const float* wrow = a.W + (long long)(k - 1) * N + (long long)j * 32;
                do {
                    const int b = __ffs(bits) - 1;
                    bits &= bits - 1u;
                    const int slot = pre[m] + __popc(ib[m] & ((1u << b) - 1u));
                    Rp[slot] = fmaf(-delta_prev, __ldg(wrow + b), Rp[slot]);
                } while (bits);
            }
            bits = zcur[m];
            if (bits) {
                const float* wrow = a.W + (long long)k * N + (long long)j * 32;
                do {
                    const int b = __ffs(bits) - 1;
                    bits &= bits - 1u;
                    const int slot = pre[m] + __popc(ib[m] & ((1u << b) - 1u));
                    const float w = __ldg(wrow + b);
                    acc_a = fmaf(w, Rp[slot], acc_a);
                    acc_b = fmaf(w, w, acc_b);
                } while (bits);
            }
            zprev[m] = zcur[m];
        }
        if (k == K) break;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc_a += __shfl_down_sync(0xffffffffu, acc_a, o);
            acc_b += __shfl_down_sync(0xffffffffu, acc_b, o);
        }
        if (lane == 0) {
            red_a[warp] = acc_a;
            red_b[warp] = acc_b;
        }
        __syncthreads();
        if (warp == 0) {
            const int nwarp = blockDim.x >> 5;
            double va = lane < nwarp ? (double)red_a[lane] : 0.0;
            double vb = lane < nwarp ? (double)red_b[lane] : 0.0;
            va = warp_sum(va);
            vb = warp_sum(vb);
            if (lane == 0) {
                const float d_old = a.D[(long long)k * P + p];
                const double num = va + (double)d_old * vb;   // sum w r^{-k}
                const double prec = (double)P + ge * vb;
                const double dnew = ge * num / prec + xi[k] / sqrt(prec);
                const float dnew_f = (float)dnew;
                a.D[(long long)k * P + p] = dnew_f;
                s_delta = dnew_f - d_old;
            }
        }
        __syncthreads();
        delta_prev = s_delta;
    }
    __syncthreads();
    float r2 = 0.0f;
    for (int s = threadIdx.x; s < cnt; s += blockDim.x) {
        const float v = Rp[s];
        r2 = fmaf(v, v, r2);
        if (SMEM_R) a.R[base + s] = v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r2 += __shfl_down_sync(0xffffffffu, r2, o);
    if (lane == 0) red_a[warp] = r2;
    __syncthreads();
    if (warp == 0) {
        double v = lane < (int)(blockDim.x >> 5) ? (double)red_a[lane] : 0.0;
        v = warp_sum(v);
        if (lane == 0) a.part_r2[p] = v;
    }
}

template <int WPT>
static cudaError_t launch_wpt(const DictArgs& a, size_t smem, bool smem_r, cudaStream_t s)
{
    void* args[] = {(void*)&a};
    void* fn = smem_r ? (void*)dict_kernel<WPT, true> : (void*)dict_kernel<WPT, false>;
    if (smem_r) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return cudaLaunchKernel(fn, dim3(a.g.P), dim3(kDictThreads), args, smem_r ? smem : 0, s);
}

cudaError_t launch_dict(const DictArgs& a, int max_slots, cudaStream_t s)
{
    if (a.g.K > kDictMaxK) return cudaErrorInvalidValue;
    const size_t smem = sizeof(float) * (size_t)max_slots;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const size_t fixed = sizeof(double) * kDictMaxK + 2 * sizeof(float) * (kDictThreads / 32) + 64;
    const bool smem_r = smem + fixed <= (size_t)optin;
    const int wpt = (a.g.NW + kDictThreads - 1) / kDictThreads;
    if (wpt <= 1) return launch_wpt<1>(a, smem, smem_r, s);
    if (wpt <= 2) return launch_wpt<2>(a, smem, smem_r, s);
    if (wpt <= 4) return launch_wpt<4>(a, smem, smem_r, s);
    if (wpt <= 8) return launch_wpt<8>(a, smem, smem_r, s);
    if (wpt <= 16) return launch_wpt<16>(a, smem, smem_r, s);
    if (wpt <= 32) return launch_wpt<32>(a, smem, smem_r, s);
    return cudaErrorInvalidValue;
}

}  // namespace sensai
