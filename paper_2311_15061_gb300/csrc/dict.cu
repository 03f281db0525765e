// dict.cu -- the dictionary sweep (the dictionary-learning step of the BPFA
// section), atoms in order k = 0..K-1, each d_kp from its conjugate Gaussian
// given every other atom's current value:
//   Lambda_kp = P + gamma_eps sum_{i: p in Omega_i} w_ik^2
//   mu_kp     = gamma_eps / Lambda_kp * sum_{i: p in Omega_i} w_ik r^{-k}_ip
//   d_kp      = mu_kp + Lambda_kp^-1/2 BoxMuller(Philox(p, k, t, DICT))
// with r^{-k} the residual that leaves atom k out (atoms before k already
// redrawn); afterwards the residual takes the new atom: r -= (d_new - d_old) w_k.
//
// Neither sum couples different pixels p, so the sweep splits into P
// independent chains of K sequential draws.  GB300 mapping: one CTA per pixel
// p keeps the residual slots of the patches observing p in shared memory.
// Atoms go in blocks of 8: one pass over the slots reads each patch's 8
// weights as one 32-byte sector, applies the previous block's update and
// accumulates G_k = sum w_k r and the in-block Gram C_kl = sum w_k w_l
// (l <= k); a fixed-order block reduction (FP32 within warps, FP64 across
// warps) feeds 8 sequential draws on one thread, exactly the atom-ordered
// conditionals because
//   sum w_k r^{-k} = G_k + d_old,k C_kk - sum_{l<k in block} (d_new,l - d_old,l) C_kl.
// The K normals are drawn up front.  No global synchronisation and no float
// atomics: results are deterministic.
#include "internal.cuh"

namespace sensai {

constexpr int kDictThreads = 512;
constexpr int kDictWarps = kDictThreads / 32;
constexpr int kDictMaxK = 1024;
constexpr int kGram = kAtomBlock * (kAtomBlock + 1) / 2;   // 36
constexpr int kRed = kAtomBlock + kGram;                    // 44 sums per block

// RHO: residual slots in shared memory; LIST: slot -> patch list too.
template <bool RHO, bool LIST>
__device__ __forceinline__ void dict_body(const DictArgs& a, const int p)
{
    extern __shared__ float dsm[];
    __shared__ float red[kDictWarps][kRed];
    __shared__ double fin[kRed];
    __shared__ double xi[kDictMaxK];
    __shared__ float s_delta[kAtomBlock];
    const int K = a.g.K, P = a.g.P, KB = a.g.KB;
    const long long Npad = a.g.Npad;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int base = a.Rbase[p];
    const int cnt = a.Rbase[p + 1] - base;
    float* rho = RHO ? dsm : a.R + base;
    int* list_s = reinterpret_cast<int*>(dsm + (RHO ? cnt : 0));
    const int* ilist = LIST ? list_s : a.Ilist + base;
    for (int s = threadIdx.x; s < cnt; s += blockDim.x) {
        if (RHO) rho[s] = a.R[base + s];
        if (LIST) list_s[s] = a.Ilist[base + s];
    }
    const uint2 key = seed_key(a.seed);
    const uint32_t t_it = launch_t(a.t, a.t_dev, a.sc);
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const uint4 blk = philox4x32_10(make_uint4((uint32_t)p, (uint32_t)k, t_it, kTagDict), key);
        xi[k] = normal64(blk.x, blk.y);
    }
    __syncthreads();

    const double ge = a.sc->gamma_eps;
    float dprev[kAtomBlock];
#pragma unroll
    for (int kk = 0; kk < kAtomBlock; ++kk) dprev[kk] = 0.0f;

    for (int kb = 0; kb <= KB; ++kb) {
        float G[kAtomBlock], C[kGram];
#pragma unroll
        for (int v = 0; v < kAtomBlock; ++v) G[v] = 0.0f;
#pragma unroll
        for (int v = 0; v < kGram; ++v) C[v] = 0.0f;
        // Two register sets (A, B) alternate over this thread's slots: the
        // loads of one slot are issued before the other slot is computed and
        // no pending load is ever copied, so two slots are always in flight.
        const float* qprev = a.W + (long long)(kb > 0 ? kb - 1 : 0) * Npad * kAtomBlock;
        const float* qcur = a.W + (long long)kb * Npad * kAtomBlock;
        const bool has_prev = kb > 0, has_cur = kb < KB;
        const int stride = blockDim.x;
        float ra = 0.0f, rb = 0.0f;
        W8 ua, va, ub, vb;
#define DICT_LOAD(S_, R_, U, V)                                             \
        do {                                                                \
            const long long i_ = ilist[S_];                                 \
            R_ = rho[S_];                                                   \
            if (has_prev) U = load_w8(qprev + i_ * kAtomBlock);             \
            if (has_cur) V = load_w8(qcur + i_ * kAtomBlock);               \
        } while (0)
#define DICT_APPLY(S_, R_, U, V)                                            \
        do {                                                                \
            if (has_prev) {                                                 \
                _Pragma("unroll") for (int k = 0; k < kAtomBlock; ++k)      \
                    R_ = fmaf(-dprev[k], U.v[k], R_);                       \
                rho[S_] = R_;                                               \
            }                                                               \
            if (has_cur) {                                                  \
                _Pragma("unroll") for (int k = 0; k < kAtomBlock; ++k) {    \
                    G[k] = fmaf(V.v[k], R_, G[k]);                          \
                    _Pragma("unroll") for (int l = 0; l <= k; ++l)          \
                        C[k * (k + 1) / 2 + l] = fmaf(V.v[k], V.v[l], C[k * (k + 1) / 2 + l]); \
                }                                                           \
            }                                                               \
        } while (0)
        int s = threadIdx.x;
        if (s < cnt) DICT_LOAD(s, ra, ua, va);
        while (s < cnt) {
            const int sb = s + stride;
            if (sb < cnt) DICT_LOAD(sb, rb, ub, vb);
            DICT_APPLY(s, ra, ua, va);
            if (sb >= cnt) break;
            const int sa = sb + stride;
            if (sa < cnt) DICT_LOAD(sa, ra, ua, va);
            DICT_APPLY(sb, rb, ub, vb);
            s = sa;
        }
#undef DICT_LOAD
#undef DICT_APPLY
        if (kb == KB) break;
#pragma unroll
        for (int v = 0; v < kRed; ++v) {
            float x = v < kAtomBlock ? G[v] : C[v - kAtomBlock];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (lane == 0) red[warp][v] = x;
        }
        __syncthreads();
        if (threadIdx.x < kRed) {
            double acc = 0.0;
            for (int w = 0; w < kDictWarps; ++w) acc += (double)red[w][threadIdx.x];
            fin[threadIdx.x] = acc;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int kk = 0; kk < kAtomBlock; ++kk) {
                const int k = kb * kAtomBlock + kk;
                if (k >= K) {
                    s_delta[kk] = 0.0f;
                    continue;
                }
                const float d_old = a.D[(long long)k * P + p];
                const double ckk = fin[kAtomBlock + kk * (kk + 1) / 2 + kk];
                double num = fin[kk] + (double)d_old * ckk;            // sum w_k r^{-k}
                for (int l = 0; l < kk; ++l) num -= (double)s_delta[l] * fin[kAtomBlock + kk * (kk + 1) / 2 + l];
                const double prec = (double)P + ge * ckk;
                const double dnew = ge * num / prec + xi[k] / sqrt(prec);
                const float dnew_f = (float)dnew;
                a.D[(long long)k * P + p] = dnew_f;
                s_delta[kk] = dnew_f - d_old;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kAtomBlock; ++kk) dprev[kk] = s_delta[kk];
    }
    __syncthreads();
    float r2 = 0.0f;
    for (int s = threadIdx.x; s < cnt; s += blockDim.x) {
        const float v = rho[s];
        r2 = fmaf(v, v, r2);
        if (RHO) a.R[base + s] = v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r2 += __shfl_down_sync(0xffffffffu, r2, o);
    if (lane == 0) red[warp][0] = r2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double acc = 0.0;
        for (int w = 0; w < kDictWarps; ++w) acc += (double)red[w][0];
        a.part_r2[p] = acc;
    }
}

template <bool RHO, bool LIST>
__global__ void __launch_bounds__(kDictThreads, 1) dict_kernel(const DictArgs a)
{
    dict_body<RHO, LIST>(a, blockIdx.x);
}

// Batched instances: CTA b draws chain (b - cta_start[i]) of instance i.
template <bool RHO, bool LIST>
__global__ void __launch_bounds__(kDictThreads, 1)
    dict_multi_kernel(const DictArgs* __restrict__ args, const int* __restrict__ cta_start, int n)
{
    int p = 0;
    const DictArgs& a = *stage_instance_args(args, cta_start, n, &p);
    dict_body<RHO, LIST>(a, p);
}

template <bool RHO, bool LIST>
static cudaError_t launch_mode(const DictArgs& a, size_t smem, cudaStream_t s)
{
    void* fn = (void*)dict_kernel<RHO, LIST>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void* args[] = {(void*)&a};
    return cudaLaunchKernel(fn, dim3(a.g.P), dim3(kDictThreads), args, smem, s);
}

// The storage mode for a chain of at most max_slots slots: 2 = residual and
// patch list in shared memory, 1 = residual only, 0 = global memory; and its
// dynamic shared memory.
int dict_mode(int max_slots, size_t* smem)
{
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return -1;
    const size_t fixed = sizeof(float) * kDictWarps * kRed + sizeof(double) * (kRed + kDictMaxK) +
                         sizeof(float) * kAtomBlock + 256;
    const size_t slots = (size_t)max_slots;
    if (slots * 8 + fixed <= (size_t)optin) { *smem = slots * 8; return 2; }
    if (slots * 4 + fixed <= (size_t)optin) { *smem = slots * 4; return 1; }
    *smem = 0;
    return 0;
}

cudaError_t launch_dict_multi(const DictArgs* args, const int* cta_start, int n, int mode, size_t smem, int grid,
                              cudaStream_t s)
{
    void* fn = mode == 2 ? (void*)dict_multi_kernel<true, true>
             : mode == 1 ? (void*)dict_multi_kernel<true, false> : (void*)dict_multi_kernel<false, false>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void* kargs[] = {(void*)&args, (void*)&cta_start, (void*)&n};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kDictThreads), kargs, smem, s);
}

cudaError_t launch_dict(const DictArgs& a, int max_slots, cudaStream_t s)
{
    if (a.g.K > kDictMaxK) return cudaErrorInvalidValue;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const size_t fixed = sizeof(float) * kDictWarps * kRed + sizeof(double) * (kRed + kDictMaxK) +
                         sizeof(float) * kAtomBlock + 256;
    const size_t slots = (size_t)max_slots;
    if (slots * 8 + fixed <= (size_t)optin) return launch_mode<true, true>(a, slots * 8, s);
    if (slots * 4 + fixed <= (size_t)optin) return launch_mode<true, false>(a, slots * 4, s);
    return launch_mode<false, false>(a, 0, s);
}

}  // namespace sensai
