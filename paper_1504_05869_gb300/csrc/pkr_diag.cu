// pkr_diag.cu -- memory ceiling of the sweep's access pattern (diagnostic).
//
// The sweep reads Q population planes at per-velocity offsets (the pull)
// and writes Q planes at the site itself.  This kernel moves exactly those
// bytes in the same way -- per-lane 8- or 4-byte cp.async copies of a
// 32-site tile into shared memory, then streaming stores -- with no
// arithmetic, so its bandwidth is the ceiling any sweep built on this access
// pattern can reach.  The offsets can be kept per axis: none (a plain copy of
// Q planes), y and z only (every warp access stays aligned to the tile), x
// only, or all three (the sweep's pull).
#include <cuda_runtime.h>

#include "pkr_internal.h"
#include "pkr_sweep.cuh"

namespace pkr {
namespace {

// SX, SYZ: keep the x, and the y and z, components of the pull offsets.  The
// geometry is the staged sweep's default one for large sets: 2 velocity groups
// x 2 tiles per block of 4 warps (each warp stages half of a tile's
// velocities).  The addresses are formed as the sweep forms them: the wrapped
// row and column offsets of the tile's sites for every displacement -R..R
// once per tile, then two adds per velocity.
template <class L, typename T, int SX, int SYZ>
__global__ void __launch_bounds__(128)
pull_copy_kernel(const T* __restrict__ A, T* __restrict__ B, int64_t V, int nx, int ny, int nz,
                 int ntiles)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int Q = L::Q;
    constexpr int RC = reach_of<L>();
    constexpr int W = 2 * RC + 1;
    constexpr int ST = 32 * (int)sizeof(T);
    constexpr int CH = (Q + 1) / 2;       // most velocities a warp stages
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int grp = w & 1;                 // velocity group
    const int sub = w >> 1;                // tile slot of the block
    const int nxy = nx * ny;
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(smem_raw) +
                          (uint32_t)(w * CH * ST + lane * (int)sizeof(T));
    for (int t = blockIdx.x * 2 + sub; t < ntiles; t += gridDim.x * 2) {
        const int64_t s64 = (int64_t)t * 32 + lane;
        const bool valid = s64 < V;
        const int s = valid ? (int)s64 : 0;
        const int r = (int)((unsigned)s / (unsigned)nx);
        const int x = s - r * nx;
        const int z = (int)((unsigned)r / (unsigned)ny);
        const int y = r - z * ny;
        int xs[W], yo[W], zo[W];
        static_for<0, W>([&](auto DI) {
            constexpr int d = decltype(DI)::value - RC;
            xs[d + RC] = wrap_off<d>(x, nx);
            yo[d + RC] = wrap_off<d>(y, ny) * nx;
            zo[d + RC] = wrap_off<d>(z, nz) * nxy;
        });
        static_for<0, 2>([&](auto GI) {
            constexpr int g = decltype(GI)::value;
            constexpr int lo = g * Q / 2, hi = (g + 1) * Q / 2;
            if (grp != g) return;
            static_for<lo, hi>([&](auto I) {
                constexpr int i = decltype(I)::value;
                constexpr int ox = SX ? vx_of<L>(i) + RC : RC;
                constexpr int oy = SYZ ? vy_of<L>(i) + RC : RC;
                constexpr int oz = SYZ ? vz_of<L>(i) + RC : RC;
                const T* src = A + ((int64_t)i * V + (zo[oz] + yo[oy] + xs[ox]));
                cp_async<sizeof(T)>(base + (uint32_t)((i - lo) * ST), src,
                                    valid ? (int)sizeof(T) : 0);
            });
            cp_async_wait_all();
            if (valid) {
                T* dst = B + ((int64_t)lo * V + s);
#pragma unroll 8
                for (int i = lo; i < hi; ++i) {
                    T v;
                    if constexpr (sizeof(T) == 8) {
                        asm volatile("ld.shared.b64 %0, [%1];"
                                     : "=l"(*reinterpret_cast<long long*>(&v))
                                     : "r"(base + (uint32_t)((i - lo) * ST)));
                    } else {
                        asm volatile("ld.shared.b32 %0, [%1];" : "=r"(*reinterpret_cast<int*>(&v))
                                     : "r"(base + (uint32_t)((i - lo) * ST)));
                    }
                    __stcs(dst, v);
                    dst += V;
                }
            }
        });
        __syncwarp();
    }
}

// The pull with the x offsets served by aligned runs: the block's two tiles
// are x-adjacent (64 sites of one row, nx a multiple of 64), warp (g, s)
// copies the aligned 32-element block s of the pair for each velocity of
// group g, plus one aligned 4-element halo on the side the velocity's x
// component needs, into that velocity's 72-element row in shared memory;
// after the two warps of the group meet, each reads its sites shifted by
// -v_x from the row and stores them.  Per velocity and pair: two aligned
// 256-byte runs and one 32-byte halo (five cache lines; six for two
// shifted runs).
template <class L, typename T>
__global__ void __launch_bounds__(128)
paired_copy_kernel(const T* __restrict__ A, T* __restrict__ B, int64_t V, int nx, int ny, int nz,
                   int npairs)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int Q = L::Q;
    constexpr int RC = reach_of<L>();
    constexpr int W = 2 * RC + 1;
    constexpr int RW = 72 * (int)sizeof(T);   // bytes of one velocity's row
    static_assert(RC <= 4, "halo of 4 elements");
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int grp = w & 1;
    const int sub = w >> 1;
    const int nxy = nx * ny;
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(smem_raw);
    for (int pr = blockIdx.x; pr < npairs; pr += gridDim.x) {
        const int s0 = pr * 64;
        const int r = (int)((unsigned)s0 / (unsigned)nx);
        const int x0 = s0 - r * nx;
        const int z = (int)((unsigned)r / (unsigned)ny);
        const int y = r - z * ny;
        int yo[W], zo[W];
        static_for<0, W>([&](auto DI) {
            constexpr int d = decltype(DI)::value - RC;
            yo[d + RC] = wrap_off<d>(y, ny) * nx;
            zo[d + RC] = wrap_off<d>(z, nz) * nxy;
        });
        const int xm = x0 + 32 * sub + lane;                       // aligned block s
        const int xl = x0 >= 4 ? x0 - 4 + lane : nx - 4 + lane;   // left halo (lanes < 4)
        const int xr = x0 + 64 < nx ? x0 + 64 + lane : lane;       // right halo (lanes < 4)
        static_for<0, 2>([&](auto GI) {
            constexpr int g = decltype(GI)::value;
            constexpr int lo = g * Q / 2, hi = (g + 1) * Q / 2;
            if (grp != g) return;
            static_for<lo, hi>([&](auto I) {
                constexpr int i = decltype(I)::value;
                constexpr int vx = vx_of<L>(i);
                constexpr int oy = vy_of<L>(i) + RC;
                constexpr int oz = vz_of<L>(i) + RC;
                const T* row = A + ((int64_t)i * V + (zo[oz] + yo[oy]));
                const uint32_t rb = base + (uint32_t)(i * RW);
                cp_async<sizeof(T)>(rb + (uint32_t)((4 + 32 * sub + lane) * sizeof(T)), row + xm,
                                    (int)sizeof(T));
                if constexpr (vx > 0) {
                    if (sub == 0 && lane < 4)
                        cp_async<sizeof(T)>(rb + (uint32_t)(lane * sizeof(T)), row + xl,
                                            (int)sizeof(T));
                } else if constexpr (vx < 0) {
                    if (sub == 1 && lane < 4)
                        cp_async<sizeof(T)>(rb + (uint32_t)((68 + lane) * sizeof(T)), row + xr,
                                            (int)sizeof(T));
                }
            });
            cp_async_wait_all();
            asm volatile("bar.sync %0, 64;" ::"r"(1 + g) : "memory");
            T* dst = B + ((int64_t)lo * V + s0 + 32 * sub + lane);
            static_for<lo, hi>([&](auto I) {
                constexpr int i = decltype(I)::value;
                constexpr int vx = vx_of<L>(i);
                const uint32_t ad =
                    base + (uint32_t)(i * RW + (4 + 32 * sub + lane - vx) * (int)sizeof(T));
                T v;
                if constexpr (sizeof(T) == 8) {
                    asm volatile("ld.shared.b64 %0, [%1];"
                                 : "=l"(*reinterpret_cast<long long*>(&v)) : "r"(ad));
                } else {
                    asm volatile("ld.shared.b32 %0, [%1];" : "=r"(*reinterpret_cast<int*>(&v))
                                 : "r"(ad));
                }
                __stcs(dst, v);
                dst += V;
            });
            // the rows are refilled for the next pair only after both warps read them
            asm volatile("bar.sync %0, 64;" ::"r"(1 + g) : "memory");
        });
    }
}

// The aligned x-pairs sweep's own staging (PairFill: halo = reach, values
// written shifted by v_x), then each warp reads its sites at H + p of every
// row of its group and stores them.  Same blocks and rows as the sweep, no
// arithmetic, rows refilled after the pair.
template <class L, typename T>
__global__ void __launch_bounds__(128)
sweep_staging_copy_kernel(const T* __restrict__ A, T* __restrict__ B, int64_t V, int nx, int ny,
                          int nz, int npairs)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using PR = Pair<L, T>;
    constexpr int Q = L::Q;
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int grp = w & 1;
    const int sub = w >> 1;
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(smem_raw);
    PairFill<L, T> fill;
    for (int pr = blockIdx.x; pr < npairs; pr += gridDim.x) {
        fill.locate(pr, nx, ny, nz, lane);
        static_for<0, 2>([&](auto GI) {
            constexpr int g = decltype(GI)::value;
            constexpr int lo = g * Q / 2, hi = (g + 1) * Q / 2;
            if (grp != g) return;
            static_for<lo, hi>([&](auto I) {
                fill.template pull<decltype(I)::value>(A, V, base, sub, lane, (int)sizeof(T));
            });
            cp_async_wait_all();
            asm volatile("bar.sync %0, 64;" ::"r"(1 + g) : "memory");
            T* dst = B + ((int64_t)lo * V + pr * 64 + 32 * sub + lane);
            static_for<lo, hi>([&](auto I) {
                constexpr int i = decltype(I)::value;
                const uint32_t ad =
                    base + (uint32_t)(i * PR::ROWB + (PR::H + 32 * sub + lane) * (int)sizeof(T));
                T v;
                if constexpr (sizeof(T) == 8) {
                    asm volatile("ld.shared.b64 %0, [%1];"
                                 : "=l"(*reinterpret_cast<long long*>(&v)) : "r"(ad));
                } else {
                    asm volatile("ld.shared.b32 %0, [%1];" : "=r"(*reinterpret_cast<int*>(&v))
                                 : "r"(ad));
                }
                __stcs(dst, v);
                dst += V;
            });
            asm volatile("bar.sync %0, 64;" ::"r"(1 + g) : "memory");
        });
    }
}

template <class L, typename T, bool SWEEP>
int run_paired_copy(const int64_t n[3], int reps, double* gbs, cudaStream_t st)
{
    const int64_t V = n[0] * n[1] * n[2];
    const size_t bytes = (size_t)L::Q * (size_t)V * sizeof(T);
    const int npairs = (int)(V / 64);
    const size_t smem = SWEEP ? Pair<L, T>::smem_bytes() : (size_t)L::Q * 72 * sizeof(T);
    auto kern = SWEEP ? sweep_staging_copy_kernel<L, T> : paired_copy_kernel<L, T>;
    if (set_sweep_smem(kern, smem) != cudaSuccess) return PKR_ECUDA;
    int dev = 0, nsm = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 128, smem) != cudaSuccess ||
        occ < 1)
        return PKR_ECUDA;
    size_t freeb = 0, totb = 0;
    if (cudaMemGetInfo(&freeb, &totb) != cudaSuccess) return PKR_ECUDA;
    if (2 * bytes + (64 << 20) > freeb) return PKR_ENOMEM;
    void *A = nullptr, *B = nullptr;
    if (cudaMalloc(&A, bytes) != cudaSuccess || cudaMalloc(&B, bytes) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(A);
        return PKR_ENOMEM;
    }
    int rc = PKR_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int grid = nsm * occ;
    if (grid > npairs) grid = npairs;
    if (cudaMemsetAsync(A, 0, bytes, st) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        rc = PKR_ECUDA;
    for (int k = 0; rc == PKR_OK && k < reps + 1; ++k) {
        if (k == 1 && cudaEventRecord(e0, st) != cudaSuccess) rc = PKR_ECUDA;
        kern<<<grid, 128, smem, st>>>(static_cast<const T*>(A), static_cast<T*>(B), V, (int)n[0],
                                     (int)n[1], (int)n[2], npairs);
        if (cudaGetLastError() != cudaSuccess) rc = PKR_ECUDA;
    }
    float ms = 0.f;
    if (rc == PKR_OK && (cudaEventRecord(e1, st) != cudaSuccess ||
                         cudaEventSynchronize(e1) != cudaSuccess ||
                         cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        rc = PKR_ECUDA;
    if (rc == PKR_OK) *gbs = 2.0 * (double)bytes * reps / (ms * 1e-3) / 1e9;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(st);
    cudaFree(A);
    cudaFree(B);
    return rc;
}

template <class L, typename T, int SX, int SYZ>
int run_pull_copy(const int64_t n[3], int reps, double* gbs, cudaStream_t st)
{
    const int64_t V = n[0] * n[1] * n[2];
    const size_t bytes = (size_t)L::Q * (size_t)V * sizeof(T);
    const int ntiles = (int)((V + 31) / 32);
    const size_t smem = (size_t)4 * ((L::Q + 1) / 2) * 32 * sizeof(T);
    auto kern = pull_copy_kernel<L, T, SX, SYZ>;
    if (set_sweep_smem(kern, smem) != cudaSuccess) return PKR_ECUDA;
    int dev = 0, nsm = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 128, smem) != cudaSuccess ||
        occ < 1)
        return PKR_ECUDA;
    size_t freeb = 0, totb = 0;
    if (cudaMemGetInfo(&freeb, &totb) != cudaSuccess) return PKR_ECUDA;
    if (2 * bytes + (64 << 20) > freeb) return PKR_ENOMEM;
    void *A = nullptr, *B = nullptr;
    if (cudaMalloc(&A, bytes) != cudaSuccess || cudaMalloc(&B, bytes) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(A);
        return PKR_ENOMEM;
    }
    int rc = PKR_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int grid = nsm * occ;
    if (grid > (ntiles + 1) / 2) grid = (ntiles + 1) / 2;
    if (cudaMemsetAsync(A, 0, bytes, st) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        rc = PKR_ECUDA;
    for (int k = 0; rc == PKR_OK && k < reps + 1; ++k) {
        if (k == 1 && cudaEventRecord(e0, st) != cudaSuccess) rc = PKR_ECUDA;
        kern<<<grid, 128, smem, st>>>(static_cast<const T*>(A), static_cast<T*>(B), V,
                                    (int)n[0], (int)n[1], (int)n[2], ntiles);
        if (cudaGetLastError() != cudaSuccess) rc = PKR_ECUDA;
    }
    float ms = 0.f;
    if (rc == PKR_OK && (cudaEventRecord(e1, st) != cudaSuccess ||
                         cudaEventSynchronize(e1) != cudaSuccess ||
                         cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        rc = PKR_ECUDA;
    if (rc == PKR_OK) *gbs = 2.0 * (double)bytes * reps / (ms * 1e-3) / 1e9;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(st);
    cudaFree(A);
    cudaFree(B);
    return rc;
}

template <class L, typename T>
int pull_copy_t(const int64_t n[3], int axes, int reps, double* gbs, cudaStream_t st)
{
    switch (axes) {
    case 0: return run_pull_copy<L, T, 0, 0>(n, reps, gbs, st);
    case 1: return run_pull_copy<L, T, 1, 0>(n, reps, gbs, st);
    case 2: return run_pull_copy<L, T, 0, 1>(n, reps, gbs, st);
    case 3: return run_pull_copy<L, T, 1, 1>(n, reps, gbs, st);
    case 7: return n[0] % 64 == 0 ? run_paired_copy<L, T, false>(n, reps, gbs, st) : PKR_EINVAL;
    case 8: return n[0] % 64 == 0 ? run_paired_copy<L, T, true>(n, reps, gbs, st) : PKR_EINVAL;
    }
    return PKR_EINVAL;
}

template <class L>
int pull_copy_l(const int64_t n[3], int elem, int axes, int reps, double* gbs, cudaStream_t st)
{
    // the per-tile offsets wrap each side once: every edge at least the reach
    for (int k = 0; k < 3; ++k)
        if (n[k] < reach_of<L>()) return PKR_EINVAL;
    if (elem == 8) return pull_copy_t<L, double>(n, axes, reps, gbs, st);
    if (elem == 4) return pull_copy_t<L, float>(n, axes, reps, gbs, st);
    return PKR_EINVAL;
}

}  // namespace
}  // namespace pkr

extern "C" int pkr_pull_copy_ceiling(int lattice, const int64_t n[3], int elem_bytes,
                                     int shift_axes, int reps, double* gbs, void* stream)
{
    using namespace pkr;
    if (!n || !gbs || reps < 1 || ((shift_axes & ~3) != 0 && shift_axes != 7 && shift_axes != 8))
        return PKR_EINVAL;
    if (n[0] < 1 || n[1] < 1 || n[2] < 1) return PKR_EINVAL;
    const int64_t V = n[0] * n[1] * n[2];
    if (V > (int64_t)0x7fffffff) return PKR_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    switch (lattice) {
    case PKR_D3Q19: return pull_copy_l<D3Q19>(n, elem_bytes, shift_axes, reps, gbs, st);
    case PKR_D3Q111: return pull_copy_l<D3Q111>(n, elem_bytes, shift_axes, reps, gbs, st);
    }
    return PKR_EINVAL;
}
