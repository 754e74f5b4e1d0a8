// pkr_noalloc.cu -- the convergence residual between two potentials,
// computed without allocating any memory.
//
// The regular path reduces the residual through per-block partial sums in a
// scratch buffer that a plan allocates with cudaMalloc.  Some callers cannot
// allocate: runtimes that own all device memory through their own pool and
// forbid side allocations, and latency-critical loops that must not enter the
// allocator (cudaMalloc and cudaFree can synchronise the device).  For them
// this file keeps the scratch in a file-scope static device array: every GPU
// that loads the library holds these 24.6 KB until the process exits, and all
// calls on a device share them.  A call ends by copying the three results to
// the host and synchronising its stream.
#include <cuda_runtime.h>

#include <mutex>

#include "pkr_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 1024;   // partials: 3 doubles per block
constexpr int kOut = 3 * kMaxBlocks;

// Scratch shared by every call on a device: block partials, then out[3].
static __device__ __align__(256) double g_residual_scratch[3 * kMaxBlocks + 3];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

__device__ __forceinline__ double wsum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double wmax(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

__global__ void __launch_bounds__(kThreads)
residual_partials_kernel(const double* __restrict__ a, const double* __restrict__ b, int64_t V,
                         double* scratch)
{
    __shared__ double s0[kThreads / 32], s1[kThreads / 32], s2[kThreads / 32];
    double d2 = 0.0, n2 = 0.0, mx = 0.0;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < V; i += stride) {
        const double x = a[i];
        const double d = x - b[i];
        d2 += d * d;
        n2 += x * x;
        mx = fmax(mx, fabs(d));
    }
    d2 = wsum(d2);
    n2 = wsum(n2);
    mx = wmax(mx);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s0[w] = d2;
        s1[w] = n2;
        s2[w] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t0 = 0.0, t1 = 0.0, t2 = 0.0;
        for (int k = 0; k < kThreads / 32; ++k) {
            t0 += s0[k];
            t1 += s1[k];
            t2 = fmax(t2, s2[k]);
        }
        scratch[3 * blockIdx.x + 0] = t0;
        scratch[3 * blockIdx.x + 1] = t1;
        scratch[3 * blockIdx.x + 2] = t2;
    }
}

__global__ void __launch_bounds__(kThreads)
residual_finalize_kernel(double* scratch, int nblocks)
{
    __shared__ double s0[kThreads / 32], s1[kThreads / 32], s2[kThreads / 32];
    double d2 = 0.0, n2 = 0.0, mx = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += kThreads) {
        d2 += scratch[3 * i + 0];
        n2 += scratch[3 * i + 1];
        mx = fmax(mx, scratch[3 * i + 2]);
    }
    d2 = wsum(d2);
    n2 = wsum(n2);
    mx = wmax(mx);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s0[w] = d2;
        s1[w] = n2;
        s2[w] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t0 = 0.0, t1 = 0.0, t2 = 0.0;
        for (int k = 0; k < kThreads / 32; ++k) {
            t0 += s0[k];
            t1 += s1[k];
            t2 = fmax(t2, s2[k]);
        }
        double* out = scratch + kOut;
        out[0] = t2;
        out[1] = (t1 > 0.0) ? sqrt(t0) / sqrt(t1) : (t0 == 0.0 ? 0.0 : INFINITY);
        out[2] = sqrt(t1);
        if (!(t0 == t0) || !(t1 == t1)) {
            out[0] = NAN;
            out[1] = NAN;
        }
    }
}

// Device address of the static scratch on the current device, looked up once
// per device (host code cannot pass the symbol itself to a kernel).
int scratch_for_current_device(double** ptr)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PKR_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return PKR_ECUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_residual_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return PKR_ECUDA;
        }
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *ptr = g_scratch_ptr[dev];
    return PKR_OK;
}

}  // namespace

extern "C" int pkr_residual_noalloc(const double* phi_new, const double* phi_old, int64_t V,
                                    double out[3], void* stream)
{
    if (!phi_new || !phi_old || !out) return PKR_EINVAL;
    if (V < 1 || V > PKR_NOALLOC_MAX_SITES) return PKR_EINVAL;
    double* scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc != PKR_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    int64_t blocks = (V + kThreads - 1) / kThreads;
    if (blocks > kMaxBlocks) blocks = kMaxBlocks;
    residual_partials_kernel<<<(int)blocks, kThreads, 0, st>>>(phi_new, phi_old, V, scratch);
    residual_finalize_kernel<<<1, kThreads, 0, st>>>(scratch, (int)blocks);
    if (cudaGetLastError() != cudaSuccess) return PKR_ECUDA;
    if (cudaMemcpyAsync(out, scratch + kOut, 3 * sizeof(double), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return PKR_ECUDA;
    return PKR_OK;
}
