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
// which a fixed-order block reduction (FP64 across threads) turns into one
// draw.  No global synchronisation, no float atomics; results are
// deterministic.
#include "internal.cuh"

namespace sensai {

constexpr int kDictThreads = 1024;

template <bool SMEM_R>
__global__ void __launch_bounds__(kDictThreads, 1) dict_kernel(const DictArgs a)
{
    extern __shared__ float rsm[];
    __shared__ double red[kDictThreads / 32];
    __shared__ float s_delta;
    const int p = blockIdx.x;
    const int K = a.g.K, P = a.g.P, NW = a.g.NW;
    const long long N = a.g.N;
    const int base = a.Rbase[p];
    const int cnt = a.Rbase[p + 1] - base;
    float* Rp = SMEM_R ? rsm : a.R + base;
    if (SMEM_R) {
        for (int s = threadIdx.x; s < cnt; s += blockDim.x) rsm[s] = a.R[base + s];
        __syncthreads();
    }
    const uint32_t* Ib = a.Ibits + (long long)p * NW;
    const uint32_t* Ip = a.Ipre + (long long)p * NW;
    const double ge = a.sc->gamma_eps;
    const uint2 key = seed_key(a.seed);
    float delta_prev = 0.0f;

    for (int k = 0; k <= K; ++k) {
        float acc_a = 0.0f, acc_b = 0.0f;
        for (int j = threadIdx.x; j < NW; j += blockDim.x) {
            const uint32_t ib = Ib[j];
            if (!ib) continue;
            const int pre = (int)Ip[j];
            if (k > 0 && delta_prev != 0.0f) {
                uint32_t bits = a.Zb[(long long)(k - 1) * NW + j] & ib;
                const float* wrow = a.W + (long long)(k - 1) * N + (long long)j * 32;
                while (bits) {
                    const int b = __ffs(bits) - 1;
                    bits &= bits - 1u;
                    const int slot = pre + __popc(ib & ((1u << b) - 1u));
                    Rp[slot] = fmaf(-delta_prev, wrow[b], Rp[slot]);
                }
            }
            if (k < K) {
                uint32_t bits = a.Zb[(long long)k * NW + j] & ib;
                const float* wrow = a.W + (long long)k * N + (long long)j * 32;
                while (bits) {
                    const int b = __ffs(bits) - 1;
                    bits &= bits - 1u;
                    const int slot = pre + __popc(ib & ((1u << b) - 1u));
                    const float w = wrow[b];
                    acc_a = fmaf(w, Rp[slot], acc_a);
                    acc_b = fmaf(w, w, acc_b);
                }
            }
        }
        if (k == K) break;
        const double sum_wr = block_sum((double)acc_a, red);
        const double sum_ww = block_sum((double)acc_b, red);
        if (threadIdx.x == 0) {
            const float d_old = a.D[(long long)k * P + p];
            const double num = sum_wr + (double)d_old * sum_ww;   // sum w r^{-k}
            const double prec = (double)P + ge * sum_ww;
            const uint4 blk = philox4x32_10(make_uint4((uint32_t)p, (uint32_t)k, a.t, kTagDict), key);
            const double dnew = ge * num / prec + normal64(blk.x, blk.y) / sqrt(prec);
            const float dnew_f = (float)dnew;
            a.D[(long long)k * P + p] = dnew_f;
            s_delta = dnew_f - d_old;
        }
        __syncthreads();
        delta_prev = s_delta;
    }
    __syncthreads();
    double r2 = 0.0;
    for (int s = threadIdx.x; s < cnt; s += blockDim.x) {
        const double v = Rp[s];
        r2 += v * v;
        if (SMEM_R) a.R[base + s] = Rp[s];
    }
    r2 = block_sum(r2, red);
    if (threadIdx.x == 0) a.part_r2[p] = r2;
}

cudaError_t launch_dict(const DictArgs& a, int max_slots, cudaStream_t s)
{
    const size_t smem = sizeof(float) * (size_t)max_slots;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const size_t reserve = sizeof(double) * (kDictThreads / 32) + 64;
    void* args[] = {(void*)&a};
    if (smem + reserve <= (size_t)optin) {
        void* fn = (void*)dict_kernel<true>;
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        return cudaLaunchKernel(fn, dim3(a.g.P), dim3(kDictThreads), args, smem, s);
    }
    return cudaLaunchKernel((void*)dict_kernel<false>, dim3(a.g.P), dim3(kDictThreads), args, 0, s);
}

}  // namespace sensai
