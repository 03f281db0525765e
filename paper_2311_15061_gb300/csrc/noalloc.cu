// noalloc.cu -- overlap-add reconstruction that allocates no device memory.
//
// sensai_reconstruct_static() serves callers that cannot allocate GPU memory
// themselves: a plugin inside a host application whose memory pool owns the
// whole device, or a live-acquisition callback with a hard time budget in
// which a cudaMalloc (which may block and synchronise the device) is not
// allowed.  They pass their own device buffers for the dictionary, the codes
// and the output frame; the only scratch this path needs, the per-patch
// reconstructions, lives in the fixed file-scope array below.
//
// The array (kStaticScratchFloats floats, 16 MiB) exists on every GPU that
// loads this library and stays there until the process exits.  Every call
// shares it and it keeps the last call's contents; each call overwrites every
// entry it reads, so nothing has to be cleared, but two calls that overlap on
// the GPU (different streams, or different host threads on one device) race
// on it and must be serialised by the caller.  The device address of the
// array is looked up once per device, on the first call made with that device
// current; that first call should come before any stream capture.
#include <mutex>

#include "internal.cuh"

namespace sensai {

constexpr long long kStaticScratchFloats = 1LL << 22;   // 16 MiB of float32
constexpr int kStaticMaxDevices = 64;

static __device__ __align__(256) float g_static_recon[kStaticScratchFloats];

namespace {

std::mutex g_static_mutex;
float* g_static_ptr[kStaticMaxDevices] = {};

// Y[p][i] = sum_k S[i][k] d_kp, codes given patch-major (zero where
// inactive).  One thread per patch, 32 pixels at a time; warp-broadcast
// shared-memory reads of the dictionary.
__global__ void __launch_bounds__(256) static_patch_recon_kernel(Geom g, const float* D, const float* S, float* Y)
{
    extern __shared__ float Ds[];  // K x ldP, zero padded
    const int K = g.K, P = g.P;
    const int ldP = (P + 31) & ~31;
    for (int idx = threadIdx.x; idx < K * ldP; idx += blockDim.x) {
        const int k = idx / ldP, p = idx - k * ldP;
        Ds[idx] = p < P ? D[(long long)k * P + p] : 0.0f;
    }
    __syncthreads();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    const float* srow = S + i * K;
    for (int p0 = 0; p0 < P; p0 += 32) {
        float acc[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) acc[q] = 0.0f;
        for (int k = 0; k < K; ++k) {
            const float w = srow[k];
            if (w != 0.0f) {
                const float* dk = Ds + k * ldP + p0;
#pragma unroll
                for (int q = 0; q < 32; ++q) acc[q] = fmaf(dk[q], w, acc[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < 32; ++q)
            if (p0 + q < P) Y[(long long)(p0 + q) * g.N + i] = acc[q];
    }
}

__device__ __forceinline__ void static_cover_range(const Geom& g, int d, long long y, long long* first,
                                                   long long* last)
{
    const long long lastp = (g.G[d] - 1) * g.S[d];
    long long lo = y - g.B[d] + 1;
    if (lo < 0) lo = 0;
    const long long hi = y < lastp ? y : lastp;
    *first = (lo + g.S[d] - 1) / g.S[d];
    *last = hi / g.S[d];
}

// Pixel q = mean over its covering patches i of Y[q - origin(i)][i].
__global__ void static_ola_gather_kernel(Geom g, const float* Y, float* out)
{
    const long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= g.nframe) return;
    long long y[kMaxDim], f[kMaxDim], l[kMaxDim], cur[kMaxDim];
    long long rem = u;
    for (int d = g.ndim - 1; d >= 0; --d) {
        y[d] = rem % g.M[d];
        rem /= g.M[d];
        static_cover_range(g, d, y[d], &f[d], &l[d]);
        if (l[d] < f[d]) {
            out[u] = 0.0f;
            return;
        }
        cur[d] = f[d];
    }
    float acc = 0.0f;
    int count = 0;
    for (;;) {
        long long i = 0;
        int p = 0;
        for (int d = 0; d < g.ndim; ++d) {
            i = i * g.G[d] + cur[d];
            p = p * g.B[d] + (int)(y[d] - cur[d] * g.S[d]);
        }
        acc += Y[(long long)p * g.N + i];
        ++count;
        int d = g.ndim - 1;
        while (d >= 0 && ++cur[d] > l[d]) {
            cur[d] = f[d];
            --d;
        }
        if (d < 0) break;
    }
    out[u] = acc / (float)count;
}

sensai_status static_fail(sensai_status st, const char* msg)
{
    record_error(msg);
    return st;
}

// Device memory of the current device dev, or managed memory.  Device memory
// of another GPU is refused: without peer access a kernel touching it faults.
bool device_resident(const void* p, int dev)
{
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (attr.type == cudaMemoryTypeManaged) return true;
    return attr.type == cudaMemoryTypeDevice && attr.device == dev;
}

}  // namespace

}  // namespace sensai

using namespace sensai;

extern "C" sensai_status sensai_reconstruct_static(const sensai_params* prm, const float* D, const float* S,
                                                   float* out, void* stream)
{
    record_error("");
    if (!prm || !D || !S || !out) return static_fail(SENSAI_EINVAL, "null argument");
    const sensai_params& p = *prm;
    if (p.ndim < 1 || p.ndim > kMaxDim) return static_fail(SENSAI_EINVAL, "ndim must be 1..4");
    if (p.K < 1 || p.K > 1024) return static_fail(SENSAI_EINVAL, "K must be 1..1024");
    Geom g{};
    g.ndim = p.ndim;
    g.K = p.K;
    // The same limits as sensai_create (N and the frame below 2^31, P at most
    // 1024), checked as the products grow so that none of them can overflow
    // and the grid sizes below fit in 32 bits.
    const long long kLimit = 1LL << 31;
    long long P = 1, N = 1, nframe = 1;
    for (int d = 0; d < p.ndim; ++d) {
        if (p.M[d] < 1 || p.B[d] < 1 || p.B[d] > p.M[d] || p.stride[d] < 1 ||
            (p.M[d] - p.B[d]) % p.stride[d] != 0)
            return static_fail(SENSAI_EINVAL, "invalid frame / patch / stride geometry");
        if (p.M[d] >= kLimit || nframe * p.M[d] >= kLimit)
            return static_fail(SENSAI_EINVAL, "frame too large (2^31 pixels or more)");
        g.M[d] = p.M[d];
        g.B[d] = p.B[d];
        g.S[d] = p.stride[d];
        g.G[d] = (p.M[d] - p.B[d]) / p.stride[d] + 1;
        P *= p.B[d];
        N *= g.G[d];
        nframe *= p.M[d];
        if (P > 1024) return static_fail(SENSAI_EINVAL, "patch size P exceeds 1024");
    }
    if (N >= kLimit) return static_fail(SENSAI_EINVAL, "too many patches (2^31 or more)");
    if (P * N > kStaticScratchFloats)
        return static_fail(SENSAI_EINVAL,
                           "P x N exceeds the 4194304-float static scratch of sensai_reconstruct_static");
    long long s = 1;
    for (int d = p.ndim - 1; d >= 0; --d) {
        g.fs[d] = s;
        s *= g.M[d];
    }
    g.P = (int)P;
    g.N = N;
    g.NW = (int)((N + 31) / 32);
    g.nframe = nframe;
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStaticMaxDevices)
        return static_fail(SENSAI_ECUDA, "no usable current CUDA device");
    if (!device_resident(D, dev) || !device_resident(S, dev) || !device_resident(out, dev))
        return static_fail(SENSAI_EINVAL, "D, S and out must be device pointers on the current device");
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return static_fail(SENSAI_ECUDA, "cudaDeviceGetAttribute failed");
    const int ldP = (g.P + 31) & ~31;
    const size_t smem = sizeof(float) * (size_t)g.K * ldP;
    if (smem > (size_t)optin) return static_fail(SENSAI_EINVAL, "dictionary does not fit in shared memory");

    float* Y = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_static_mutex);
        if (!g_static_ptr[dev]) {
            float* ptr = nullptr;
            const cudaError_t e = cudaGetSymbolAddress((void**)&ptr, g_static_recon);
            if (e != cudaSuccess || !ptr) return static_fail(SENSAI_ECUDA, "cudaGetSymbolAddress of the static scratch failed");
            g_static_ptr[dev] = ptr;
        }
        Y = g_static_ptr[dev];
    }
    const cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaFuncSetAttribute((void*)static_patch_recon_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return static_fail(SENSAI_ECUDA, cudaGetErrorString(e));
    static_patch_recon_kernel<<<(unsigned int)((N + 255) / 256), 256, smem, st>>>(g, D, S, Y);
    static_ola_gather_kernel<<<(unsigned int)((nframe + 255) / 256), 256, 0, st>>>(g, Y, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return static_fail(SENSAI_ECUDA, cudaGetErrorString(e));
    return SENSAI_OK;
}
