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
// tiles of 32; one warp owns a tile and all Q velocities of it (one lane per
// site).  Blocks are persistent and stride over the tiles.  Every velocity
// component is a compile-time constant, so the pull address of a velocity is
// two integer adds on per-tile wrapped row/column offsets.  Plane i of an
// array lives at i*V.
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
template <class L>
__host__ __device__ constexpr int ncls_of() { return L::T.ncls; }
// First velocity of symmetry class c (Q for c = ncls).
template <class L>
__host__ __device__ constexpr int cls_begin(int c)
{
    for (int i = 0; i < L::Q; ++i)
        if (L::T.cls[i] == c) return i;
    return L::Q;
}

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

__device__ __forceinline__ void store_stream(double* p, double v) { __stcs(p, v); }
__device__ __forceinline__ void store_stream(float* p, float v) { __stcs(p, v); }

// ---------------------------------------------------------------------------
// Staged sweep: one warp owns a tile of 32 consecutive sites and all Q
// velocities.  The Q pulled values of the tile are copied global -> shared
// with per-lane asynchronous copies (cp.async, zero-fill for lanes past the
// end and for the first step), so a warp keeps Q x 256 bytes in flight
// without spending registers on them.  Each lane then reads back only its own
// column: no block barrier is needed.  The density is the exact sum above;
// the equilibrium-plus-source term is formed once per symmetry class.
// ---------------------------------------------------------------------------
template <int BYTES>
__device__ __forceinline__ void cp_async(uint32_t dst, const void* src, int src_bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(dst), "l"(src),
                 "n"(BYTES), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

template <class L, typename T>
struct Staged {
    static constexpr int WARPS = 2;                 // warps per block
    static constexpr int Q = L::Q;
    static constexpr size_t smem_bytes() { return (size_t)WARPS * Q * 32 * sizeof(T); }
};

// Density of one site from its Q pulled values in shared memory (stride 32)
// without binary64 additions.  The values are aligned to the largest
// exponent E among them in a 64-bit two's-complement fixed-point sum whose
// unit is 2^(E - 1075 - GB), i.e. GB guard bits below the last place of the
// largest value (GB = 63 - 53 - ceil(log2 Q) leaves room for Q terms).  Each
// term is rounded to that unit (error <= 2^-(GB+1) ulp of the largest value,
// below the half-ulp that every plain binary64 addition may lose), the sum is
// exact, and one conversion plus one exact power-of-two scaling return it to
// binary64.  On this GPU the FP64 pipe issues about two operations per clock
// per SM, so this costs two of its slots per site instead of Q - 1.  Inf/NaN
// inputs, or values all below 2^-1011, take the plain binary64 path.
__host__ __device__ constexpr int ceil_log2(int q)
{
    int r = 0;
    while ((1 << r) < q) ++r;
    return r;
}

// Shared-memory loads issued as volatile asm: a batch of them can go out
// back to back, and the compiler cannot hoist all Q of them into registers.
__device__ __forceinline__ double lds_f64(uint32_t addr)
{
    double v;
    asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ int lds_hi32(uint32_t addr)
{
    int v;
    asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(addr + 4));
    return v;
}
__device__ __forceinline__ float lds_f32(uint32_t addr)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
    return v;
}

// One term of the fixed-point density: the value rounded to the unit
// 2^(emax - 1075 - GB), sign applied.
template <int GB>
__device__ __forceinline__ long long fixed_term(double v, int emax)
{
    const long long b = __double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7ff);
    const long long m = e ? (((b & 0xfffffffffffffll) | (1ll << 52)) << GB) : 0ll;
    const int rs = emax - e;
    const long long t = rs < 63 ? ((m + ((1ll << rs) >> 1)) >> rs) : 0ll;
    return b < 0 ? -t : t;
}

template <int Q>
__device__ __forceinline__ double density_fixed(uint32_t col)   // col: shared address, stride 256 B
{
    constexpr int GB = 63 - 53 - ceil_log2(Q);
    constexpr int U = 8;
    static_assert(GB >= 1, "too many velocities for the 64-bit density sum");
    // largest exponent: max of the high words with the sign cleared
    int h0 = 0, h1 = 0, h2 = 0, h3 = 0;
#pragma unroll 2
    for (int k = 0; k + 3 < Q; k += 4) {
        h0 = max(h0, lds_hi32(col + (k + 0) * 256) & 0x7fffffff);
        h1 = max(h1, lds_hi32(col + (k + 1) * 256) & 0x7fffffff);
        h2 = max(h2, lds_hi32(col + (k + 2) * 256) & 0x7fffffff);
        h3 = max(h3, lds_hi32(col + (k + 3) * 256) & 0x7fffffff);
    }
#pragma unroll
    for (int k = Q - Q % 4; k < Q; ++k) h0 = max(h0, lds_hi32(col + k * 256) & 0x7fffffff);
    const int emax = max(max(h0, h1), max(h2, h3)) >> 20;
    if (emax == 0x7ff || emax < 64) {
        double s = 0.0;
        for (int k = 0; k < Q; ++k) s += lds_f64(col + k * 256);
        return s;
    }
    long long a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    for (int k = 0; k + U - 1 < Q; k += U) {
        double v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = lds_f64(col + (k + u) * 256);
        a0 += fixed_term<GB>(v[0], emax) + fixed_term<GB>(v[4], emax);
        a1 += fixed_term<GB>(v[1], emax) + fixed_term<GB>(v[5], emax);
        a2 += fixed_term<GB>(v[2], emax) + fixed_term<GB>(v[6], emax);
        a3 += fixed_term<GB>(v[3], emax) + fixed_term<GB>(v[7], emax);
    }
#pragma unroll
    for (int k = Q - Q % U; k < Q; ++k) a0 += fixed_term<GB>(lds_f64(col + k * 256), emax);
    return (double)((a0 + a1) + (a2 + a3)) *
           __longlong_as_double((long long)(emax - 52 - GB) << 52);
}

template <int Q>
__device__ __forceinline__ float density_fixed_f32(uint32_t col)   // stride 128 B
{
    // binary32 storage: plain sum in four interleaved partials (fixed order)
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll 2
    for (int k = 0; k + 3 < Q; k += 4) {
        s0 += lds_f32(col + (k + 0) * 128);
        s1 += lds_f32(col + (k + 1) * 128);
        s2 += lds_f32(col + (k + 2) * 128);
        s3 += lds_f32(col + (k + 3) * 128);
    }
#pragma unroll
    for (int k = Q - Q % 4; k < Q; ++k) s0 += lds_f32(col + k * 128);
    return (s0 + s1) + (s2 + s3);
}

template <typename T> __device__ __forceinline__ T lds_val(uint32_t addr);
template <> __device__ __forceinline__ double lds_val<double>(uint32_t addr) { return lds_f64(addr); }
template <> __device__ __forceinline__ float lds_val<float>(uint32_t addr) { return lds_f32(addr); }

template <int Q, typename T> struct Density;
template <int Q> struct Density<Q, double> {
    static __device__ __forceinline__ double run(uint32_t col) { return density_fixed<Q>(col); }
};
template <int Q> struct Density<Q, float> {
    static __device__ __forceinline__ float run(uint32_t col) { return density_fixed_f32<Q>(col); }
};

template <class L, typename T>
__global__ void __launch_bounds__(Staged<L, T>::WARPS * 32)
sweep_staged_kernel(const SweepArgs a, const Coefs<typename AccType<T>::type> c)
{
    using R = typename AccType<T>::type;
    constexpr int Q = L::Q;
    constexpr int WARPS = Staged<L, T>::WARPS;
    constexpr int RC = reach_of<L>();
    constexpr int W = 2 * RC + 1;
    constexpr int NC = ncls_of<L>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double rpart[WARPS][3];

    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    T* col = reinterpret_cast<T*>(smem_raw) + (size_t)wib * Q * 32 + lane;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(col);
    const T* __restrict__ A = static_cast<const T*>(a.A);
    T* __restrict__ B = static_cast<T*>(a.B);
    const T* __restrict__ S = static_cast<const T*>(a.S);
    const int64_t V = a.V;
    const int nxy = a.nx * a.ny;

    double rd2 = 0.0, rn2 = 0.0, rmx = 0.0;
    const int nw = gridDim.x * WARPS;
    for (int tile = blockIdx.x * WARPS + wib; tile < a.ntiles; tile += nw) {
        const int64_t s64 = (int64_t)tile * 32 + lane;
        const bool valid = s64 < V;
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
        const int nbytes = (valid && !a.zero_in) ? (int)sizeof(T) : 0;
        static_for<0, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int ox = vx_of<L>(i) + RC;
            constexpr int oy = vy_of<L>(i) + RC;
            constexpr int oz = vz_of<L>(i) + RC;
            const T* src = A + ((int64_t)i * V + (zo[oz] + yo[oy] + xs[ox]));
            cp_async<sizeof(T)>(sbase + (uint32_t)(i * 32 * sizeof(T)), src, nbytes);
        });
        cp_async_wait_all();

        const R Phi = Density<Q, T>::run(sbase);
        const R Sx = valid ? (R)S[s] : R(0);
        if (valid) {
            // relax and store, one symmetry class at a time (velocities of a
            // class are contiguous and share phi_c, chi_c)
            static_for<0, NC>([&](auto CI) {
                constexpr int cl = decltype(CI)::value;
                constexpr int i0 = cls_begin<L>(cl);
                constexpr int i1 = cls_begin<L>(cl + 1);
                const R e = fma(c.wphi[cl], Phi, c.chi[cl] * Sx);
                T* dst = B + ((int64_t)i0 * V + s);
                int i = i0;
                for (; i + 3 < i1; i += 4) {
                    const R g0 = lds_val<T>(sbase + (i + 0) * 32 * sizeof(T));
                    const R g1 = lds_val<T>(sbase + (i + 1) * 32 * sizeof(T));
                    const R g2 = lds_val<T>(sbase + (i + 2) * 32 * sizeof(T));
                    const R g3 = lds_val<T>(sbase + (i + 3) * 32 * sizeof(T));
                    store_stream(dst, (T)fma(c.om1, g0, e));
                    store_stream(dst + V, (T)fma(c.om1, g1, e));
                    store_stream(dst + 2 * V, (T)fma(c.om1, g2, e));
                    store_stream(dst + 3 * V, (T)fma(c.om1, g3, e));
                    dst += 4 * V;
                }
                for (; i < i1; ++i) {
                    store_stream(dst, (T)fma(c.om1, (R)lds_val<T>(sbase + i * 32 * sizeof(T)), e));
                    dst += V;
                }
            });
        }
        if (a.mode != kPlain && valid) {
            const double ph = (double)Phi;
            if (a.mode == kCheck) {
                const double d = ph - a.Phi[s];
                rd2 += d * d;
                rn2 += ph * ph;
                rmx = fmax(rmx, fabs(d));
            }
            a.Phi[s] = ph;
        }
        __syncwarp();
    }

    if (a.mode == kCheck) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            rd2 += __shfl_down_sync(0xffffffffu, rd2, o);
            rn2 += __shfl_down_sync(0xffffffffu, rn2, o);
            rmx = fmax(rmx, __shfl_down_sync(0xffffffffu, rmx, o));
        }
        if (lane == 0) {
            rpart[wib][0] = rd2;
            rpart[wib][1] = rn2;
            rpart[wib][2] = rmx;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double t0 = 0.0, t1 = 0.0, t2 = 0.0;
            for (int k = 0; k < WARPS; ++k) {
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
int launch_sweep_t(int variant, const SweepArgs& a, const void* coefs, int grid, void* stream)
{
    using R = typename AccType<T>::type;
    const Coefs<R>& c = *static_cast<const Coefs<R>*>(coefs);
    (void)variant;
    constexpr int threads = Staged<L, T>::WARPS * 32;
    const size_t smem = Staged<L, T>::smem_bytes();
    sweep_staged_kernel<L, T><<<grid, threads, smem, (cudaStream_t)stream>>>(a, c);
    return (int)cudaGetLastError();
}

template <class L, typename T>
int occupancy_t(int variant, int* blocks)
{
    (void)variant;
    constexpr int threads = Staged<L, T>::WARPS * 32;
    const size_t smem = Staged<L, T>::smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(sweep_staged_kernel<L, T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, sweep_staged_kernel<L, T>,
                                                              threads, smem);
}

#define PKR_INSTANTIATE_SWEEP(L)                                                             \
    template int launch_sweep_t<L, double>(int, const SweepArgs&, const void*, int, void*); \
    template int launch_sweep_t<L, float>(int, const SweepArgs&, const void*, int, void*);  \
    template int occupancy_t<L, double>(int, int*);                                          \
    template int occupancy_t<L, float>(int, int*);

}  // namespace pkr
