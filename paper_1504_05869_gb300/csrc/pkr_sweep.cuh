// pkr_sweep.cuh -- the fused stream-and-collide sweep (one time step of the
// high-order kinetic relaxation scheme) as a templated CUDA kernel.
//
// One launch performs, at every site x of the periodic grid:
//   pull-stream   g_i(x) = A_i(x - v_i)                       (all Q velocities)
//   density       Phi(x) = sum_i g_i(x)
//   BGK + source  B_i(x) = (1 - w) g_i(x) + w phi_i Phi(x) + chi_i S(x)
// and, on residual sweeps, compares Phi with the previous step's Phi and
// emits per-block partial sums of |dPhi|^2, |Phi|^2 and max |dPhi|.
//
// Work decomposition.  Sites are taken in the flat order (z*ny + y)*nx + x in
// tiles of 32 (one warp lane per site).  The Q velocities of a tile are split
// among G warps (each holds ~Q/G pulled values in registers); the G partial
// sums of Phi meet in shared memory, then every warp relaxes and stores its
// own velocities.  A block carries M such tiles.  Blocks are persistent and
// stride over the tiles.  Every velocity component is a compile-time
// constant, so the pull address of a velocity is two integer adds on
// per-tile wrapped row/column offsets.  Plane i of an array lives at i*V.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "pkr_internal.h"

namespace pkr {

template <class L>
__host__ __device__ constexpr int vx_of(int i) { return L::T.v[i].x; }
template <class L>
__host__ __device__ constexpr int vy_of(int i) { return L::T.v[i].y; }
template <class L>
__host__ __device__ constexpr int vz_of(int i) { return L::T.v[i].z; }
template <class L>
__host__ __device__ constexpr int cls_of(int i) { return L::T.cls[i]; }
template <class L>
__host__ __device__ constexpr int reach_of() { return L::T.reach; }

// Velocity groups per tile (G) and tiles per block (M) of each lattice.
template <class L> struct Split { static constexpr int G = 1, M = 4; };
template <> struct Split<D2Q81> { static constexpr int G = 3, M = 1; };
template <> struct Split<D2Q169> { static constexpr int G = 6, M = 1; };
template <> struct Split<D3Q111> { static constexpr int G = 4, M = 1; };

template <int I, int N, typename F>
__device__ __forceinline__ void static_for(F&& f)
{
    if constexpr (I < N) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, N>(f);
    }
}

template <typename T> struct AccType { using type = T; };

__device__ __forceinline__ int wrap_near(int c, int n)
{
    c = c < 0 ? c + n : c;
    return c >= n ? c - n : c;
}
__device__ __forceinline__ int wrap_any(int c, int n)
{
    int r = c % n;
    return r < 0 ? r + n : r;
}

// Exact sum of binary64 values, rounded once.  The values are aligned to
// the largest exponent E among them in a 128-bit two's-complement integer
// whose unit is 2^(E - 1139) (64 bits below the unit in the last place of
// the largest value; anything smaller than that is dropped), added exactly
// with integer instructions, and the total is converted back to binary64.
// On this GPU the FP64 pipe issues about two operations per clock per SM, so
// a density sum of ~28 values per thread costs ~28 pipe slots in binary64
// but only four here (two conversions, one FMA and one scaling).  Inf/NaN or
// values all below 2^-895 take the plain binary64 path.
template <int N>
__device__ __forceinline__ double exact_sum(const double* v)
{
    int emax = 0;
#pragma unroll
    for (int k = 0; k < N; ++k) emax = max(emax, (__double2hiint(v[k]) >> 20) & 0x7ff);
    if (emax == 0x7ff || emax < 128) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < N; ++k) s += v[k];
        return s;
    }
    unsigned long long lo = 0ull;
    long long hi = 0ll;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const unsigned long long bits = (unsigned long long)__double_as_longlong(v[k]);
        const int e = (int)((bits >> 52) & 0x7ffull);
        const unsigned long long m =
            (bits & 0xfffffffffffffull) | (e ? (1ull << 52) : 0ull);
        const int sh = (e ? e : 1) - emax + 64;   // <= 64
        const int sl = sh > 0 ? sh : 0;
        const int sr = sh < 0 ? -sh : 0;
        const unsigned long long ms = sr < 64 ? (m >> sr) : 0ull;
        unsigned long long tlo = sl < 64 ? (ms << sl) : 0ull;
        unsigned long long thi = sl > 0 ? (ms >> (64 - sl)) : 0ull;
        // two's complement negation of (thi:tlo) when the sign bit is set
        const unsigned long long neg = bits >> 63;
        const unsigned long long mask = 0ull - neg;
        tlo = (tlo ^ mask) + neg;
        thi = (thi ^ mask) + ((neg && tlo == 0ull) ? 1ull : 0ull);
        const unsigned long long nlo = lo + tlo;
        hi += (long long)thi + (nlo < lo ? 1ll : 0ll);
        lo = nlo;
    }
    const double r = fma((double)hi, 18446744073709551616.0, (double)lo);
    return r * __longlong_as_double((long long)(emax - 116) << 52);
}

template <int N>
__device__ __forceinline__ float exact_sum(const float* v)
{
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < N; ++k) s += v[k];
    return s;
}

__device__ __forceinline__ void store_stream(double* p, double v) { __stcs(p, v); }
__device__ __forceinline__ void store_stream(float* p, float v) { __stcs(p, v); }

template <class L, typename T>
__global__ void __launch_bounds__(Split<L>::G * Split<L>::M * 32)
sweep_kernel(const SweepArgs a, const Coefs<typename AccType<T>::type> c)
{
    using R = typename AccType<T>::type;
    constexpr int Q = L::Q;
    constexpr int G = Split<L>::G;
    constexpr int M = Split<L>::M;
    constexpr int RC = reach_of<L>();
    constexpr int W = 2 * RC + 1;
    constexpr int CH = (Q + G - 1) / G;

    __shared__ R red[2][M][G][32];
    __shared__ double rpart[M][3];

    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int grp = wid % G;
    const int sub = wid / G;
    const T* __restrict__ A = static_cast<const T*>(a.A);
    T* __restrict__ B = static_cast<T*>(a.B);
    const T* __restrict__ S = static_cast<const T*>(a.S);
    const int64_t V = a.V;
    const int nxy = a.nx * a.ny;

    double rd2 = 0.0, rn2 = 0.0, rmx = 0.0;
    int buf = 0;
    const int nbt = (a.ntiles + M - 1) / M;
    for (int bt = blockIdx.x; bt < nbt; bt += gridDim.x, buf ^= 1) {
        const int tile = bt * M + sub;
        const int64_t s64 = (int64_t)tile * 32 + lane;
        const bool valid = (tile < a.ntiles) && (s64 < V);
        const int s = valid ? (int)s64 : 0;
        const int x = s % a.nx;
        const int r = s / a.nx;
        const int y = r % a.ny;
        const int z = r / a.ny;

        int xs[W], yo[W], zo[W];
#pragma unroll
        for (int d = -RC; d <= RC; ++d) {
            if (a.small) {
                xs[d + RC] = wrap_any(x - d, a.nx);
                yo[d + RC] = wrap_any(y - d, a.ny) * a.nx;
                zo[d + RC] = wrap_any(z - d, a.nz) * nxy;
            } else {
                xs[d + RC] = wrap_near(x - d, a.nx);
                yo[d + RC] = wrap_near(y - d, a.ny) * a.nx;
                zo[d + RC] = wrap_near(z - d, a.nz) * nxy;
            }
        }

        T g[CH];
        R part = R(0);
        const bool load = valid && !a.zero_in;
        static_for<0, G>([&](auto GI) {
            constexpr int gi = decltype(GI)::value;
            constexpr int lo = gi * Q / G;
            constexpr int hi = (gi + 1) * Q / G;
            if (grp == gi) {
                static_for<lo, hi>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    constexpr int ox = vx_of<L>(i) + RC;
                    constexpr int oy = vy_of<L>(i) + RC;
                    constexpr int oz = vz_of<L>(i) + RC;
                    T val = T(0);
                    if (load) val = A[(int64_t)i * V + (zo[oz] + yo[oy] + xs[ox])];
                    g[i - lo] = val;
                });
                part = exact_sum<hi - lo>(g);
            }
        });

        red[buf][sub][grp][lane] = part;
        __syncthreads();
        R Phi = red[buf][sub][0][lane];
#pragma unroll
        for (int k = 1; k < G; ++k) Phi = fma(red[buf][sub][k][lane], R(1), Phi);
        const R Sx = valid ? (R)S[s] : R(0);

        static_for<0, G>([&](auto GI) {
            constexpr int gi = decltype(GI)::value;
            constexpr int lo = gi * Q / G;
            constexpr int hi = (gi + 1) * Q / G;
            if (grp == gi) {
                static_for<lo, hi>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    constexpr int cl = cls_of<L>(i);
                    const R e = fma(c.wphi[cl], Phi, c.chi[cl] * Sx);
                    const R p = fma(c.om1, (R)g[i - lo], e);
                    if (valid) store_stream(&B[(int64_t)i * V + s], (T)p);
                });
            }
        });

        if (a.mode != kPlain && grp == 0 && valid) {
            const double ph = (double)Phi;
            if (a.mode == kCheck) {
                const double d = ph - a.Phi[s];
                rd2 += d * d;
                rn2 += ph * ph;
                rmx = fmax(rmx, fabs(d));
            }
            a.Phi[s] = ph;
        }
    }

    if (a.mode == kCheck) {
        if (grp == 0) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                rd2 += __shfl_down_sync(0xffffffffu, rd2, o);
                rn2 += __shfl_down_sync(0xffffffffu, rn2, o);
                rmx = fmax(rmx, __shfl_down_sync(0xffffffffu, rmx, o));
            }
            if (lane == 0) {
                rpart[sub][0] = rd2;
                rpart[sub][1] = rn2;
                rpart[sub][2] = rmx;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double t0 = 0.0, t1 = 0.0, t2 = 0.0;
            for (int k = 0; k < M; ++k) {
                t0 += rpart[k][0];
                t1 += rpart[k][1];
                t2 = fmax(t2, rpart[k][2]);
            }
            a.partials[3 * blockIdx.x + 0] = t0;
            a.partials[3 * blockIdx.x + 1] = t1;
            a.partials[3 * blockIdx.x + 2] = t2;
        }
    }
}

template <class L, typename T>
int launch_sweep_t(const SweepArgs& a, const void* coefs, int grid, void* stream)
{
    using R = typename AccType<T>::type;
    constexpr int threads = Split<L>::G * Split<L>::M * 32;
    sweep_kernel<L, T><<<grid, threads, 0, (cudaStream_t)stream>>>(
        a, *static_cast<const Coefs<R>*>(coefs));
    return (int)cudaGetLastError();
}

template <class L, typename T>
int occupancy_t(int* blocks)
{
    constexpr int threads = Split<L>::G * Split<L>::M * 32;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, sweep_kernel<L, T>, threads, 0);
}

#define PKR_INSTANTIATE_SWEEP(L)                                                        \
    template int launch_sweep_t<L, double>(const SweepArgs&, const void*, int, void*); \
    template int launch_sweep_t<L, float>(const SweepArgs&, const void*, int, void*);  \
    template int occupancy_t<L, double>(int*);                                          \
    template int occupancy_t<L, float>(int*);

}  // namespace pkr
