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
#include <cuda_fp16.h>
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
__host__ __device__ __forceinline__ void static_for(F&& f)
{
    if constexpr (I < N) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, N>(f);
    }
}

template <typename T> struct AccType { using type = T; };
template <> struct AccType<long long> { using type = double; };
// Type of the stored source: binary64 for fixed-point populations.
template <typename T> struct SrcType { using type = T; };
template <> struct SrcType<long long> { using type = double; };

__device__ __forceinline__ int wrap_near(int c, int n)
{
    c = c < 0 ? c + n : c;
    return c >= n ? c - n : c;
}
// c - D wrapped into [0, n) for c in [0, n) and |D| <= n: only one side can
// be crossed, and which one is known at compile time.
template <int D>
__device__ __forceinline__ int wrap_off(int c, int n)
{
    const int v = c - D;
    if constexpr (D > 0) return v < 0 ? v + n : v;
    else if constexpr (D < 0) return v >= n ? v - n : v;
    else return v;
}
__device__ __forceinline__ int wrap_any(int c, int n)
{
    int r = c % n;
    return r < 0 ? r + n : r;
}

__device__ __forceinline__ void store_stream(double* p, double v) { __stcs(p, v); }
__device__ __forceinline__ void store_stream(float* p, float v) { __stcs(p, v); }
__device__ __forceinline__ void store_stream(long long* p, long long v) { __stcs(p, v); }

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
// The copies issued since the last commit form one group.
__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
// Every committed group but the most recent one has landed.
__device__ __forceinline__ void cp_async_wait_all_but_last()
{
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
}
// Every committed group has landed.
__device__ __forceinline__ void cp_async_wait_committed()
{
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// A sweep kernel's dynamic shared memory.  The split of each SM's L1/shared
// array is left to the CUDA driver, which takes the smallest shared part that
// holds the kernel's full occupancy: the rest stays L1, where the 4- and
// 8-byte asynchronous copies of the pull land on their way to shared memory.
// Forcing the largest shared part (228 KB, 28 KB of L1) measured 19% slower
// for the staged sweep at 256^3 in 64-bit fixed point, whose three blocks
// (60.5 KB each) fit the 196 KB split with 60 KB of L1.
template <typename K>
cudaError_t set_sweep_smem(K kern, size_t smem)
{
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// Launch geometry of the staged sweep.  A tile's Q velocities are split
// among G warps (velocity groups): splitting cuts the shared memory a warp
// stages by G and so lets an SM hold more warps, at the price of two
// named-barrier meetings per tile.  A block carries TILES tiles.  Several
// (G, TILES) variants are compiled per lattice and storage type; a plan picks
// one (default table below, or pkr_plan_autotune).
template <class L, typename T, int G_, int TILES_>
struct Staged {
    static constexpr int Q = L::Q;
    static constexpr int G = G_;
    static constexpr int TILES = TILES_;
    static constexpr int WARPS = G * TILES;
    static constexpr int CH = (Q + G - 1) / G;     // most velocities a warp stages
    static constexpr size_t smem_bytes() { return (size_t)WARPS * CH * 32 * sizeof(T); }
    static constexpr int lo(int g) { return g * Q / G; }
};

// Variant list: (G, TILES) pairs.  Small sets are never split.
struct Geo {
    int G, TILES;
};
template <class L>
struct Variants {
    static constexpr int N = (L::Q > 64) ? 6 : 2;
    static constexpr Geo at(int k)
    {
        if (L::Q > 64) {
            constexpr Geo big[6] = {{1, 2}, {2, 1}, {2, 2}, {3, 1}, {3, 2}, {4, 1}};
            return big[k];
        }
        constexpr Geo small[2] = {{1, 2}, {1, 4}};
        return small[k];
    }
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

// One term of the fixed-point density at twice its resolution: t = floor(2y)
// for y = v / 2^(emax - 1075 - GB), the mantissa shifted right as a magnitude
// and the sign applied by complement afterwards (for arithmetic shifts
// ~(x >> r) == (~x) >> r, so a negative term becomes floor(2y - 2^-r), which
// moves only exact ties).  floor((t + 1) / 2) = (t + (t & 1)) / 2 is then y
// rounded to the nearest integer, ties away from zero.  A shift of 54 + GB or
// more (zero, subnormal or negligible values) leaves 0 or -1, i.e. a rounded 0.
template <int GB>
__device__ __forceinline__ long long fixed_term2(double v, int emax)
{
    const long long b = __double_as_longlong(v);
    const int hi = (int)(b >> 32);
    const int e = (hi >> 20) & 0x7ff;
    const unsigned long long m =
        ((unsigned long long)(b & 0xfffffffffffffll) | (1ull << 52)) << (GB + 1);
    // PTX shr.b64 clamps shift amounts above 64 to 64 (result 0): no min needed
    unsigned long long r;
    asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(m), "r"(emax - e));
    return (long long)r ^ (long long)(hi >> 31);
}

// Largest exponent among N staged binary64 values (VS bytes apart).
template <int N, int VS = 256>
__device__ __forceinline__ int max_exponent(uint32_t col)
{
    int h0 = 0, h1 = 0;
#pragma unroll 2
    for (int k = 0; k + 3 < N; k += 4) {
        h0 = __vimax3_s32(h0, lds_hi32(col + (k + 0) * VS) & 0x7fffffff,
                          lds_hi32(col + (k + 1) * VS) & 0x7fffffff);
        h1 = __vimax3_s32(h1, lds_hi32(col + (k + 2) * VS) & 0x7fffffff,
                          lds_hi32(col + (k + 3) * VS) & 0x7fffffff);
    }
#pragma unroll
    for (int k = N - N % 4; k < N; ++k) h0 = max(h0, lds_hi32(col + k * VS) & 0x7fffffff);
    return max(h0, h1) >> 20;
}

// Fixed-point sum of N staged binary64 values aligned to emax (GB guard bits):
// the sum of the terms rounded to the unit, kept as four partial sums (term k
// in partial k mod 4) of the doubled terms t_k and of their low bits (sum of
// rounded terms = (sum t_k + sum (t_k & 1)) / 2, exact, and even per partial).
// |t_k| < 2^(54 + GB), so a partial of fewer than 2^(9 - GB) terms cannot
// overflow; with GB = 10 - ceil(log2 Q) that holds for every N <= Q.
template <int GB, int N, int VS = 256>
__device__ __forceinline__ long long fixed_sum(uint32_t col, int emax)
{
    constexpr int U = 8;
    static_assert((N + 3) / 4 < (1 << (9 - GB)), "fixed-point partial may overflow");
    long long a[4] = {0, 0, 0, 0};
    int p[4] = {0, 0, 0, 0};
    for (int k = 0; k + U - 1 < N; k += U) {
        double v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = lds_f64(col + (k + u) * VS);
        long long t[U];
#pragma unroll
        for (int u = 0; u < U; ++u) t[u] = fixed_term2<GB>(v[u], emax);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            a[u] += t[u] + t[u + 4];
            p[u] += (int)(t[u] & 1) + (int)(t[u + 4] & 1);
        }
    }
#pragma unroll
    for (int k = N - N % U; k < N; ++k) {
        const long long t = fixed_term2<GB>(lds_f64(col + k * VS), emax);
        a[k % 4] += t;
        p[k % 4] += (int)(t & 1);
    }
    return ((a[0] + p[0]) >> 1) + ((a[1] + p[1]) >> 1) + ((a[2] + p[2]) >> 1) +
           ((a[3] + p[3]) >> 1);
}

template <int N, int VS = 256>
__device__ __forceinline__ double plain_sum(uint32_t col)
{
    double s = 0.0;
    for (int k = 0; k < N; ++k) s += lds_f64(col + k * VS);
    return s;
}

// emax out of the range the fixed-point sum handles: Inf/NaN, or every value
// below 2^-960 (take the plain binary64 sum then).
__device__ __forceinline__ bool plain_path(int emax) { return emax == 0x7ff || emax < 64; }

template <int GB>
__device__ __forceinline__ double fixed_value(long long acc, int emax)
{
    // acc x 2^(emax - 1075 - GB): the power of two is added to the exponent
    // field of the converted value on the integer pipe (the binary64 pipe is
    // the scarce one).  emax >= 64 here (plain_path), so a non-zero result is
    // normal; past the binary64 range it is +-inf, as the product would be.
    const double d = (double)acc;
    const long long b = __double_as_longlong(d);
    const int k = emax - 1075 - GB;
    const int be = (int)((b >> 52) & 0x7ff) + k;
    if (acc == 0) return d;
    if (be >= 0x7ff) return acc > 0 ? __longlong_as_double(0x7ff0000000000000ll)
                                    : __longlong_as_double((long long)0xfff0000000000000ull);
    return __longlong_as_double(b + ((long long)k << 52));
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
template <> __device__ __forceinline__ long long lds_val<long long>(uint32_t addr)
{
    long long v;
    asm volatile("ld.shared.s64 %0, [%1];" : "=l"(v) : "r"(addr));
    return v;
}

// One grid as a tile step sees it.
template <typename T>
struct TileGrid {
    const T* A;     // populations in (pulled)
    T* B;           // populations out
    const typename SrcType<T>::type* S;   // source
    double* Phi;    // density (written on write/check sweeps)
    int64_t V;
    int nx, ny, nz, small;
    double soff;    // constant added to S in this step (mass correction)
    int fr, fw;     // fixed-point storage: exponents of the read and written arrays
    long long cfx;  // fixed-point storage: round((1 - omega) 2^62)
};

__device__ __forceinline__ long long lds_s64(uint32_t addr)
{
    long long v;
    asm volatile("ld.shared.s64 %0, [%1];" : "=l"(v) : "r"(addr));
    return v;
}

// Sum of N staged 64-bit fixed-point values (VS bytes apart) in four
// interleaved partials: integer addition is exact and associative (two's
// complement wraps cancel), so the split leaves the sum unchanged and cuts
// the dependent chain of 64-bit adds to a quarter.  U: groups of four per
// loop trip (code size against loop overhead; timed per kernel at 256^3).
template <int N, int VS, int U>
__device__ __forceinline__ long long fx_sum(uint32_t col)
{
    long long a0 = 0, a1 = 0, a2 = 0, a3 = 0;
#pragma unroll U
    for (int k = 0; k + 3 < N; k += 4) {
        a0 += lds_s64(col + (k + 0) * VS);
        a1 += lds_s64(col + (k + 1) * VS);
        a2 += lds_s64(col + (k + 2) * VS);
        a3 += lds_s64(col + (k + 3) * VS);
    }
#pragma unroll
    for (int k = N - N % 4; k < N; ++k) a0 += lds_s64(col + k * VS);
    return (a0 + a1) + (a2 + a3);
}

// round(q c / 2^62), rounding half up (c = (1 - omega) 2^62 for the relaxation)
__device__ __forceinline__ long long fx_mul(long long q, long long c)
{
    const __int128 prod = (__int128)q * (__int128)c + ((__int128)1 << 61);
    return (long long)(prod >> 62);
}

// 2^e as a binary64 (|e| < 1000)
__device__ __forceinline__ double pow2(int e)
{
    return __longlong_as_double((long long)(1023 + e) << 52);
}

// The part of a tile step that follows the pull, for velocity group g of G
// (velocities lo(g) .. lo(g + 1) - 1), as the warp-specialised sweep runs it;
// tile_step below carries the same operations inline (its binary64 sweep
// measured 1.9% slower when it called this function instead): the group's
// share of the density
// (the G warps of a tile meet at named barrier `bar`, twice in binary64 and
// once otherwise; every meeting sits outside lane-dependent branches), the
// relaxation and store of the group's velocities, and, in group 0, the
// density output and the residual terms.  sbase: this lane's column of the
// group's staged values (velocity lo(g) first, the next VS bytes further on);
// xacc, xexp: the tile's exchange rows.  after_class(std::integral_constant
// <int, cl>) runs, in every lane, once the group's velocities of symmetry
// class cl are relaxed and stored (classes the group holds, in order).
// SPLIT >= 0: the group's staged values from SPLIT on may still be in flight
// when the call starts; before_tail() (run in every lane) makes them
// visible, and the density reads the values before SPLIT first.  The
// fixed-point and binary64 density sums are exact, so the split leaves them
// unchanged; binary32 runs before_tail() before its ordered sum.
struct NoHook {
    template <class C>
    __device__ __forceinline__ void operator()(C) const {}
};
struct NoTail {
    __device__ __forceinline__ void operator()() const {}
};
template <class L, typename T, int G, int g, int VS = 32 * (int)sizeof(T), int SPLIT = -1,
          class Hook = NoHook, class Tail = NoTail>
__device__ __forceinline__ void group_compute(const TileGrid<T>& tg,
                                              const Coefs<typename AccType<T>::type>& c,
                                              int mode, bool valid, int s,
                                              typename AccType<T>::type Sx, int lane,
                                              uint32_t sbase, int bar, long long (&xacc)[G][32],
                                              int (&xexp)[G][32], double& d2, double& n2,
                                              double& mx, double& ms, unsigned long long& fxm,
                                              const Hook& after_class = Hook{},
                                              const Tail& before_tail = Tail{})
{
    using R = typename AccType<T>::type;
    constexpr int lo = g * L::Q / G;
    constexpr int hi = (g + 1) * L::Q / G;
    constexpr int n = hi - lo;
    constexpr int NC = ncls_of<L>();
    constexpr int GB = 63 - 53 - ceil_log2(L::Q);
    T* __restrict__ B = tg.B;
    const int64_t V = tg.V;
    R Phi;
    if constexpr (std::is_same<T, long long>::value) {
        // fixed point: the density is an exact integer sum
        long long part;
        if constexpr (SPLIT > 0 && SPLIT < n) {
            part = fx_sum<SPLIT, VS, 1>(sbase);
            before_tail();
            part += fx_sum<n - SPLIT, VS, 1>(sbase + SPLIT * VS);
        } else {
            if constexpr (SPLIT >= 0) before_tail();
            part = fx_sum<n, VS, 1>(sbase);
        }
        if constexpr (G > 1) {
            xacc[g][lane] = part;
            asm volatile("bar.sync %0, %1;" ::"r"(bar), "n"(G * 32) : "memory");
            part = 0;
#pragma unroll
            for (int k = 0; k < G; ++k) part += xacc[k][lane];
        }
        Phi = (double)part * pow2(-tg.fr);
    } else if constexpr (std::is_same<T, double>::value) {
        int emax;
        if constexpr (SPLIT > 0 && SPLIT < n) {
            emax = max_exponent<SPLIT, VS>(sbase);
            before_tail();
            emax = max(emax, max_exponent<n - SPLIT, VS>(sbase + SPLIT * VS));
        } else {
            if constexpr (SPLIT >= 0) before_tail();
            emax = max_exponent<n, VS>(sbase);
        }
        if constexpr (G > 1) {
            xexp[g][lane] = emax;
            asm volatile("bar.sync %0, %1;" ::"r"(bar), "n"(G * 32) : "memory");
#pragma unroll
            for (int k = 0; k < G; ++k) emax = max(emax, xexp[k][lane]);
        }
        const bool plain = plain_path(emax);
        long long part = plain ? __double_as_longlong(plain_sum<n, VS>(sbase))
                               : fixed_sum<GB, n, VS>(sbase, emax);
        if constexpr (G > 1) {
            xacc[g][lane] = part;
            asm volatile("bar.sync %0, %1;" ::"r"(bar), "n"(G * 32) : "memory");
            if (plain) {
                double t = 0.0;
#pragma unroll
                for (int k = 0; k < G; ++k) t += __longlong_as_double(xacc[k][lane]);
                Phi = t;
            } else {
                long long t = 0;
#pragma unroll
                for (int k = 0; k < G; ++k) t += xacc[k][lane];
                Phi = fixed_value<GB>(t, emax);
            }
        } else {
            Phi = plain ? __longlong_as_double(part) : fixed_value<GB>(part, emax);
        }
    } else {
        if constexpr (SPLIT >= 0) before_tail();
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll 2
        for (int k = 0; k + 3 < n; k += 4) {
            s0 += lds_f32(sbase + (k + 0) * VS);
            s1 += lds_f32(sbase + (k + 1) * VS);
            s2 += lds_f32(sbase + (k + 2) * VS);
            s3 += lds_f32(sbase + (k + 3) * VS);
        }
#pragma unroll
        for (int k = n - n % 4; k < n; ++k) s0 += lds_f32(sbase + k * VS);
        float part = (s0 + s1) + (s2 + s3);
        if constexpr (G > 1) {
            // binary32 partials meet in group order (fixed, deterministic)
            xacc[g][lane] = (long long)__float_as_int(part);
            asm volatile("bar.sync %0, %1;" ::"r"(bar), "n"(G * 32) : "memory");
            part = 0.f;
#pragma unroll
            for (int k = 0; k < G; ++k) part += __int_as_float((int)xacc[k][lane]);
        }
        Phi = part;
    }

    // relax and store this group's velocities, one symmetry class at a
    // time (velocities of a class are contiguous and share phi_c, chi_c)
    static_for<0, NC>([&](auto CI) {
        constexpr int cl = decltype(CI)::value;
        constexpr int cb = cls_begin<L>(cl), ce = cls_begin<L>(cl + 1);
        constexpr int i0 = cb > lo ? cb : lo;
        constexpr int i1 = ce < hi ? ce : hi;
        if (valid) {
            if constexpr (i0 < i1 && std::is_same<T, long long>::value) {
                const double e = fma(c.wphi[cl], Phi, c.chi[cl] * Sx);
                const long long ei = __double2ll_rn(e * pow2(tg.fw));
                // the written array's scale is 2^-k that of the read one (k >= 0,
                // the rescale only lowers it): fold 2^-k into the coefficient
                const int k = tg.fr - tg.fw;
                const long long cw = k == 0 ? tg.cfx : ((tg.cfx >> (k - 1)) + 1) >> 1;
                T* dst = B + ((int64_t)i0 * V + s);
#pragma unroll 2
                for (int i = i0; i < i1; ++i) {
                    const long long p = fx_mul(lds_s64(sbase + (i - lo) * VS), cw) + ei;
                    fxm |= (unsigned long long)(p ^ (p >> 63));
                    store_stream(dst, (T)p);
                    dst += V;
                }
            } else if constexpr (i0 < i1) {
                const R e = fma(c.wphi[cl], Phi, c.chi[cl] * Sx);
                T* dst = B + ((int64_t)i0 * V + s);
                int i = i0;
                for (; i + 3 < i1; i += 4) {
                    const R g0 = lds_val<T>(sbase + (i + 0 - lo) * VS);
                    const R g1 = lds_val<T>(sbase + (i + 1 - lo) * VS);
                    const R g2 = lds_val<T>(sbase + (i + 2 - lo) * VS);
                    const R g3 = lds_val<T>(sbase + (i + 3 - lo) * VS);
                    store_stream(dst, (T)fma(c.om1, g0, e));
                    store_stream(dst + V, (T)fma(c.om1, g1, e));
                    store_stream(dst + 2 * V, (T)fma(c.om1, g2, e));
                    store_stream(dst + 3 * V, (T)fma(c.om1, g3, e));
                    dst += 4 * V;
                }
                for (; i < i1; ++i) {
                    const R gi = lds_val<T>(sbase + (i - lo) * VS);
                    store_stream(dst, (T)fma(c.om1, gi, e));
                    dst += V;
                }
            }
        }
        if constexpr (i0 < i1) after_class(CI);
    });
    // density output and residual contributions (one group per tile)
    if (g == 0 && mode != kPlain && valid) {
        const double ph = (double)Phi;
        if (mode == kCheck) {
            const double d = ph - tg.Phi[s];
            d2 += d * d;
            n2 += ph * ph;
            mx = fmax(mx, fabs(d));
            ms += ph;
        }
        tg.Phi[s] = ph;
    }
}

// One 32-site tile of one grid, executed by the G warps of a tile slot:
// pull (cp.async), density, relax + store, density output.  On check sweeps
// the lane's contributions to |dPhi|^2, |Phi|^2, max |dPhi| and sum Phi are
// added to d2, n2, mx, ms (velocity group 0 only).
template <class L, typename T, int G, int TILES>
__device__ __forceinline__ void tile_step(const TileGrid<T>& tg,
                                          const Coefs<typename AccType<T>::type>& c, int tile,
                                          int mode, bool zero_in, int lane, int grp, int sub,
                                          uint32_t sbase, long long (&xacc)[TILES][G][32],
                                          int (&xexp)[TILES][G][32], double& d2, double& n2,
                                          double& mx, double& ms, unsigned long long& fxm)
{
    using R = typename AccType<T>::type;
    using ST = Staged<L, T, G, TILES>;
    constexpr int RC = reach_of<L>();
    constexpr int W = 2 * RC + 1;
    constexpr int NC = ncls_of<L>();
    constexpr int GB = 63 - 53 - ceil_log2(L::Q);
    static_assert(GB >= 1, "too many velocities for the 64-bit density sum");
    const T* __restrict__ A = tg.A;
    T* __restrict__ B = tg.B;
    const int64_t V = tg.V;
    const int nx = tg.nx, ny = tg.ny, nz = tg.nz;
    const int nxy = nx * ny;

    const int64_t s64 = (int64_t)tile * 32 + lane;
    const bool valid = s64 < V;
    const int s = valid ? (int)s64 : 0;
    const int r = (int)((unsigned)s / (unsigned)nx);
    const int x = s - r * nx;
    const int z = (int)((unsigned)r / (unsigned)ny);
    const int y = r - z * ny;
    int xs[W], yo[W], zo[W];
    if (tg.small) {
#pragma unroll
        for (int d = -RC; d <= RC; ++d) {
            xs[d + RC] = wrap_any(x - d, nx);
            yo[d + RC] = wrap_any(y - d, ny) * nx;
            zo[d + RC] = wrap_any(z - d, nz) * nxy;
        }
    } else {
        static_for<0, W>([&](auto DI) {
            constexpr int d = decltype(DI)::value - RC;
            xs[d + RC] = wrap_off<d>(x, nx);
            yo[d + RC] = wrap_off<d>(y, ny) * nx;
            zo[d + RC] = wrap_off<d>(z, nz) * nxy;
        });
    }
    const int nbytes = (valid && !zero_in) ? (int)sizeof(T) : 0;
    // the source offset (mass correction) is used by binary32 storage only
    R Sx = R(0);
    if (valid) {
        if constexpr (std::is_same<T, float>::value) Sx = (R)((double)tg.S[s] + tg.soff);
        else Sx = (R)tg.S[s];
    }

    static_for<0, G>([&](auto GI) {
        constexpr int g = decltype(GI)::value;
        constexpr int lo = ST::lo(g);
        constexpr int hi = ST::lo(g + 1);
        constexpr int n = hi - lo;
        if (grp != g) return;
        // pull: one asynchronous copy per velocity of this group
        static_for<lo, hi>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int ox = vx_of<L>(i) + RC;
            constexpr int oy = vy_of<L>(i) + RC;
            constexpr int oz = vz_of<L>(i) + RC;
            const T* src = A + ((int64_t)i * V + (zo[oz] + yo[oy] + xs[ox]));
            cp_async<sizeof(T)>(sbase + (uint32_t)((i - lo) * 32 * sizeof(T)), src, nbytes);
        });
        cp_async_wait_all();

        // density (the G warps of a tile meet twice at named barrier 1 + sub;
        // both barriers sit outside every lane-dependent branch)
        R Phi;
        if constexpr (std::is_same<T, long long>::value) {
            // fixed point: the density is an exact integer sum
            long long part = fx_sum<n, 256, 4>(sbase);
            if constexpr (G > 1) {
                xacc[sub][g][lane] = part;
                asm volatile("bar.sync %0, %1;" ::"r"(1 + sub), "n"(G * 32) : "memory");
                part = 0;
#pragma unroll
                for (int k = 0; k < G; ++k) part += xacc[sub][k][lane];
            }
            Phi = (double)part * pow2(-tg.fr);
        } else if constexpr (std::is_same<T, double>::value) {
            int emax = max_exponent<n>(sbase);
            if constexpr (G > 1) {
                xexp[sub][g][lane] = emax;
                asm volatile("bar.sync %0, %1;" ::"r"(1 + sub), "n"(G * 32) : "memory");
#pragma unroll
                for (int k = 0; k < G; ++k) emax = max(emax, xexp[sub][k][lane]);
            }
            const bool plain = plain_path(emax);
            long long part = plain ? __double_as_longlong(plain_sum<n>(sbase))
                                   : fixed_sum<GB, n>(sbase, emax);
            if constexpr (G > 1) {
                xacc[sub][g][lane] = part;
                asm volatile("bar.sync %0, %1;" ::"r"(1 + sub), "n"(G * 32) : "memory");
                if (plain) {
                    double t = 0.0;
#pragma unroll
                    for (int k = 0; k < G; ++k) t += __longlong_as_double(xacc[sub][k][lane]);
                    Phi = t;
                } else {
                    long long t = 0;
#pragma unroll
                    for (int k = 0; k < G; ++k) t += xacc[sub][k][lane];
                    Phi = fixed_value<GB>(t, emax);
                }
            } else {
                Phi = plain ? __longlong_as_double(part) : fixed_value<GB>(part, emax);
            }
        } else {
            float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll 2
            for (int k = 0; k + 3 < n; k += 4) {
                s0 += lds_f32(sbase + (k + 0) * 128);
                s1 += lds_f32(sbase + (k + 1) * 128);
                s2 += lds_f32(sbase + (k + 2) * 128);
                s3 += lds_f32(sbase + (k + 3) * 128);
            }
#pragma unroll
            for (int k = n - n % 4; k < n; ++k) s0 += lds_f32(sbase + k * 128);
            float part = (s0 + s1) + (s2 + s3);
            if constexpr (G > 1) {
                // binary32 partials meet in group order (fixed, deterministic)
                xacc[sub][g][lane] = (long long)__float_as_int(part);
                asm volatile("bar.sync %0, %1;" ::"r"(1 + sub), "n"(G * 32) : "memory");
                part = 0.f;
#pragma unroll
                for (int k = 0; k < G; ++k) part += __int_as_float((int)xacc[sub][k][lane]);
            }
            Phi = part;
        }

        // relax and store this group's velocities, one symmetry class at a
        // time (velocities of a class are contiguous and share phi_c, chi_c)
        if (valid) {
            static_for<0, NC>([&](auto CI) {
                constexpr int cl = decltype(CI)::value;
                constexpr int cb = cls_begin<L>(cl), ce = cls_begin<L>(cl + 1);
                constexpr int i0 = cb > lo ? cb : lo;
                constexpr int i1 = ce < hi ? ce : hi;
                if constexpr (i0 < i1 && std::is_same<T, long long>::value) {
                    const double e = fma(c.wphi[cl], Phi, c.chi[cl] * Sx);
                    const long long ei = __double2ll_rn(e * pow2(tg.fw));
                    // the written array's scale is 2^-k that of the read one (k >= 0,
                    // the rescale only lowers it): fold 2^-k into the coefficient
                    const int k = tg.fr - tg.fw;
                    const long long cw = k == 0 ? tg.cfx : ((tg.cfx >> (k - 1)) + 1) >> 1;
                    T* dst = B + ((int64_t)i0 * V + s);
#pragma unroll 2
                    for (int i = i0; i < i1; ++i) {
                        const long long p = fx_mul(lds_s64(sbase + (i - lo) * 256), cw) + ei;
                        fxm |= (unsigned long long)(p ^ (p >> 63));
                        store_stream(dst, (T)p);
                        dst += V;
                    }
                } else if constexpr (i0 < i1) {
                    const R e = fma(c.wphi[cl], Phi, c.chi[cl] * Sx);
                    T* dst = B + ((int64_t)i0 * V + s);
                    int i = i0;
                    for (; i + 3 < i1; i += 4) {
                        const R g0 = lds_val<T>(sbase + (i + 0 - lo) * 32 * sizeof(T));
                        const R g1 = lds_val<T>(sbase + (i + 1 - lo) * 32 * sizeof(T));
                        const R g2 = lds_val<T>(sbase + (i + 2 - lo) * 32 * sizeof(T));
                        const R g3 = lds_val<T>(sbase + (i + 3 - lo) * 32 * sizeof(T));
                        store_stream(dst, (T)fma(c.om1, g0, e));
                        store_stream(dst + V, (T)fma(c.om1, g1, e));
                        store_stream(dst + 2 * V, (T)fma(c.om1, g2, e));
                        store_stream(dst + 3 * V, (T)fma(c.om1, g3, e));
                        dst += 4 * V;
                    }
                    for (; i < i1; ++i) {
                        const R gi = lds_val<T>(sbase + (i - lo) * 32 * sizeof(T));
                        store_stream(dst, (T)fma(c.om1, gi, e));
                        dst += V;
                    }
                }
            });
        }
        // density output and residual contributions (one group per tile)
        if (g == 0 && mode != kPlain && valid) {
            const double ph = (double)Phi;
            if (mode == kCheck) {
                const double d = ph - tg.Phi[s];
                d2 += d * d;
                n2 += ph * ph;
                mx = fmax(mx, fabs(d));
                ms += ph;
            }
            tg.Phi[s] = ph;
        }
    });
    __syncwarp();
}

template <class L, typename T, int G_, int TILES_>
__global__ void __launch_bounds__(G_ * TILES_ * 32)
sweep_staged_kernel(const SweepArgs a, const Coefs<typename AccType<T>::type> c)
{
    if (a.stop != nullptr && *a.stop != 0) return;   // the run stopped before this step
    constexpr int G = G_;
    constexpr int TILES = TILES_;
    using ST = Staged<L, T, G, TILES>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double rpart[TILES][4];
    // per-group partial densities of a tile, two sets used by turns: a warp
    // writes the next tile's partial only after the exchange barrier of that
    // tile, so a partner still reading this tile's set cannot see it change
    __shared__ long long xacc[2][TILES][G][32];
    __shared__ int xexp[TILES][G][32];         // per-group largest exponents

    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int grp = wib % G;     // velocity group of this warp
    const int sub = wib / G;     // tile slot of this warp in the block
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(
        reinterpret_cast<T*>(smem_raw) + (size_t)wib * ST::CH * 32 + lane);
    const bool fx = std::is_same<T, long long>::value;
    const TileGrid<T> tg{static_cast<const T*>(a.A), static_cast<T*>(a.B),
                         static_cast<const typename SrcType<T>::type*>(a.S), a.Phi, a.V, a.nx,
                         a.ny, a.nz, a.small, a.soff, fx ? a.fxF[a.cur] : 0,
                         fx ? a.fxF[a.cur ^ 1] : 0, a.cfx};

    double rd2 = 0.0, rn2 = 0.0, rmx = 0.0, rms = 0.0;
    unsigned long long fxm = 0ull;
    const int nt = gridDim.x * TILES;
    int par = 0;
    for (int tile = blockIdx.x * TILES + sub; tile < a.ntiles; tile += nt, par ^= 1)
        tile_step<L, T, G, TILES>(tg, c, tile, a.mode, a.zero_in != 0, lane, grp, sub, sbase,
                                  xacc[par], xexp, rd2, rn2, rmx, rms, fxm);
    if constexpr (std::is_same<T, long long>::value) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            fxm |= __shfl_down_sync(0xffffffffu, fxm, o);
        }
        if (lane == 0 && fxm) atomicOr(a.fxmax, fxm);
    }

    if (a.mode == kCheck) {
        if (grp == 0) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                rd2 += __shfl_down_sync(0xffffffffu, rd2, o);
                rn2 += __shfl_down_sync(0xffffffffu, rn2, o);
                rmx = fmax(rmx, __shfl_down_sync(0xffffffffu, rmx, o));
                rms += __shfl_down_sync(0xffffffffu, rms, o);
            }
            if (lane == 0) {
                rpart[sub][0] = rd2;
                rpart[sub][1] = rn2;
                rpart[sub][2] = rmx;
                rpart[sub][3] = rms;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0;
            for (int k = 0; k < TILES; ++k) {
                t0 += rpart[k][0];
                t1 += rpart[k][1];
                t2 = fmax(t2, rpart[k][2]);
                t3 += rpart[k][3];
            }
            a.partials[4 * blockIdx.x + 0] = t0;
            a.partials[4 * blockIdx.x + 1] = t1;
            a.partials[4 * blockIdx.x + 2] = t2;
            a.partials[4 * blockIdx.x + 3] = t3;
        }
    }
}

// ---------------------------------------------------------------------------
// Batch sweep: one persistent launch advances every live grid of a batch by
// one step.  Batch-wide tile t belongs to the grid whose tile_begin is the
// largest one <= t (binary search over the descriptors).  A grid's age (steps
// since it joined) picks its buffers and its own residual schedule: it writes
// Phi when (age + 2) % K == 0 and checks when (age + 1) % K == 0 (age >= 1),
// so a grid's trajectory and stopping step do not depend on what else is in
// the batch.  On check steps each tile leaves its four partial sums in
// tile_partials (with the sum of Phi); pkr_batch_reduce sums them per grid in
// a fixed order.
// ---------------------------------------------------------------------------
template <class L, typename T, int G_, int TILES_>
__global__ void __launch_bounds__(G_ * TILES_ * 32)
sweep_batch_kernel(BatchState* st, int K)
{
    using R = typename AccType<T>::type;
    constexpr int G = G_;
    constexpr int TILES = TILES_;
    using ST = Staged<L, T, G, TILES>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ long long xacc[2][TILES][G][32];   // two sets used by turns (staged sweep)
    __shared__ int xexp[TILES][G][32];

    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int grp = wib % G;
    const int sub = wib / G;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(
        reinterpret_cast<T*>(smem_raw) + (size_t)wib * ST::CH * 32 + lane);
    const BatchGrid<R>* grids = static_cast<const BatchGrid<R>*>(st->grids);
    const int ngrids = st->ngrids;
    const int ntiles = st->ntiles;
    const long long step = st->step;
    double* tpart = st->tile_partials;

    const int nt = gridDim.x * TILES;
    int par = 0;
    for (int tile = blockIdx.x * TILES + sub; tile < ntiles; tile += nt, par ^= 1) {
        int lo = 0, hi = ngrids - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (grids[mid].tile_begin <= tile) lo = mid;
            else hi = mid - 1;
        }
        const BatchGrid<R>& gd = grids[lo];
        const long long age = step - gd.join;
        const int cur = (int)(age & 1);
        const bool zero_in = (age == 0);
        int mode = kPlain;
        if (age >= 1 && (age + 1) % K == 0) mode = kCheck;
        else if (zero_in || (age + 2) % K == 0) mode = kWritePhi;
        constexpr bool fx = std::is_same<T, long long>::value;
        // binary32: the step after a check removes the mass that check measured
        const double soff = (gd.soff && age >= 1 && age % K == 0) ? *gd.soff : 0.0;
        const TileGrid<T> tg{static_cast<const T*>(gd.pop[cur]), static_cast<T*>(gd.pop[cur ^ 1]),
                             static_cast<const typename SrcType<T>::type*>(gd.S), gd.Phi, gd.V,
                             gd.nx, gd.ny, gd.nz, gd.small, soff, fx ? gd.fxF[cur] : 0,
                             fx ? gd.fxF[cur ^ 1] : 0, fx ? gd.cfx : 0};
        double d2 = 0.0, n2 = 0.0, mx = 0.0, ms = 0.0;
        unsigned long long fxm = 0ull;
        tile_step<L, T, G, TILES>(tg, gd.c, tile - gd.tile_begin, mode, zero_in, lane, grp, sub,
                                  sbase, xacc[par], xexp, d2, n2, mx, ms, fxm);
        if constexpr (fx) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) fxm |= __shfl_down_sync(0xffffffffu, fxm, o);
            if (lane == 0 && fxm) atomicOr(gd.fxmax, fxm);
        }
        if (mode == kCheck && grp == 0) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                d2 += __shfl_down_sync(0xffffffffu, d2, o);
                n2 += __shfl_down_sync(0xffffffffu, n2, o);
                mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
                ms += __shfl_down_sync(0xffffffffu, ms, o);
            }
            if (lane == 0) {
                tpart[4 * (int64_t)tile + 0] = d2;
                tpart[4 * (int64_t)tile + 1] = n2;
                tpart[4 * (int64_t)tile + 2] = mx;
                tpart[4 * (int64_t)tile + 3] = ms;
            }
        }
    }
}

template <class L, typename T, int K>
int launch_batch_variant(BatchState* st, int check_every, int grid, void* stream)
{
    constexpr Geo geo = Variants<L>::at(K);
    using ST = Staged<L, T, geo.G, geo.TILES>;
    sweep_batch_kernel<L, T, geo.G, geo.TILES><<<grid, ST::WARPS * 32, ST::smem_bytes(),
                                                 (cudaStream_t)stream>>>(st, check_every);
    return (int)cudaGetLastError();
}

template <class L, typename T, int K>
int batch_occupancy_variant(int* blocks)
{
    constexpr Geo geo = Variants<L>::at(K);
    using ST = Staged<L, T, geo.G, geo.TILES>;
    auto kern = sweep_batch_kernel<L, T, geo.G, geo.TILES>;
    cudaError_t e = set_sweep_smem(kern, ST::smem_bytes());
    if (e != cudaSuccess) return (int)e;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern, ST::WARPS * 32,
                                                              ST::smem_bytes());
}

template <class L, typename T>
int launch_batch_t(int variant, BatchState* st, int check_every, int grid, void* stream)
{
    int rc = (int)cudaErrorInvalidValue;
    static_for<0, Variants<L>::N>([&](auto K) {
        if (variant == decltype(K)::value)
            rc = launch_batch_variant<L, T, decltype(K)::value>(st, check_every, grid, stream);
    });
    return rc;
}

template <class L, typename T>
int batch_occupancy_t(int variant, int* blocks)
{
    int rc = (int)cudaErrorInvalidValue;
    static_for<0, Variants<L>::N>([&](auto K) {
        if (variant == decltype(K)::value)
            rc = batch_occupancy_variant<L, T, decltype(K)::value>(blocks);
    });
    return rc;
}

// ---------------------------------------------------------------------------
// binary16 storage.  A population value v lives as the binary16 number
// v / sc[k] in array k, with sc[k] a power of two set before each step so
// that the step's largest |p| has 4x headroom below 65504; every arithmetic
// operation is binary32.  cp.async has no 2-byte form, so each lane copies
// the aligned 4-byte word that holds its value and picks the half by the
// parity of the element index.  One warp per tile, all Q velocities.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned int lds_b32(uint32_t addr)
{
    unsigned int v;
    asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}

template <class L, int TILES>
__global__ void __launch_bounds__(TILES * 32)
sweep_h16_kernel(const SweepArgs a, const Coefs<float> c)
{
    constexpr int Q = L::Q;
    constexpr int RC = reach_of<L>();
    constexpr int W = 2 * RC + 1;
    constexpr int NC = ncls_of<L>();
    constexpr int NPB = (Q + 31) / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double rpart[TILES][4];
    __shared__ float mpart[TILES];

    const int lane = threadIdx.x & 31;
    const int sub = threadIdx.x >> 5;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem_raw) +
                           (uint32_t)((sub * Q * 32 + lane) * 4);
    const __half* __restrict__ A = static_cast<const __half*>(a.A);
    __half* __restrict__ B = static_cast<__half*>(a.B);
    const float* __restrict__ S = static_cast<const float*>(a.S);
    const int64_t V = a.V;
    const int nxy = a.nx * a.ny;
    const float sr = a.sc[a.cur];
    const float inv_sw = 1.0f / a.sc[a.cur ^ 1];
    const int vodd = (int)(V & 1);

    double rd2 = 0.0, rn2 = 0.0, rmx = 0.0, rms = 0.0;
    float pmax = 0.f;
    int of = 0;
    const int nt = gridDim.x * TILES;
    for (int tile = blockIdx.x * TILES + sub; tile < a.ntiles; tile += nt) {
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
        const int nbytes = (valid && !a.zero_in) ? 4 : 0;
        unsigned int pb[NPB];
#pragma unroll
        for (int k = 0; k < NPB; ++k) pb[k] = 0u;
        static_for<0, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int ox = vx_of<L>(i) + RC;
            constexpr int oy = vy_of<L>(i) + RC;
            constexpr int oz = vz_of<L>(i) + RC;
            const int off = zo[oz] + yo[oy] + xs[ox];
            const int par = (off ^ ((i & 1) & vodd)) & 1;     // parity of i*V + off
            const __half* src = A + ((int64_t)i * V + off - par);
            cp_async<4>(sbase + (uint32_t)(i * 128), src, nbytes);
            pb[i / 32] |= (unsigned int)par << (i % 32);
        });
        cp_async_wait_all();

        // pick each lane's half and rewrite the slot as a binary32 value, so
        // the passes below are those of binary32 storage
#pragma unroll
        for (int w = 0; w < NPB; ++w) {
            const unsigned int bits = pb[w];
            const int nb = (Q - 32 * w) < 32 ? (Q - 32 * w) : 32;
#pragma unroll 4
            for (int b = 0; b < nb; ++b) {
                const uint32_t ad = sbase + (uint32_t)((32 * w + b) * 128);
                const unsigned int wd = lds_b32(ad);
                const unsigned int h = ((bits >> b) & 1u) ? (wd >> 16) : (wd & 0xffffu);
                const float v = __half2float(__ushort_as_half((unsigned short)h));
                asm volatile("st.shared.f32 [%0], %1;" ::"r"(ad), "f"(v) : "memory");
            }
        }
        // the slots hold unscaled values: the array's scale sr (a power of
        // two, so exactly) multiplies the sum and the relaxation factor
        const float Phi = density_fixed_f32<Q>(sbase) * sr;
        const float om1s = c.om1 * sr;
        const float Sx = valid ? (float)((double)S[s] + a.soff) : 0.f;
        if (valid) {
            static_for<0, NC>([&](auto CI) {
                constexpr int cl = decltype(CI)::value;
                constexpr int i0 = cls_begin<L>(cl), i1 = cls_begin<L>(cl + 1);
                const float e = fmaf(c.wphi[cl], Phi, c.chi[cl] * Sx);
                unsigned short* dst = reinterpret_cast<unsigned short*>(B) + ((int64_t)i0 * V + s);
#pragma unroll 4
                for (int i = i0; i < i1; ++i) {
                    const float p = fmaf(om1s, lds_f32(sbase + (uint32_t)(i * 128)), e);
                    pmax = fmaxf(pmax, fabsf(p));
                    __stcs(dst, __half_as_ushort(__float2half_rn(p * inv_sw)));
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
                rms += ph;
            }
            a.Phi[s] = ph;
        }
        __syncwarp();
    }

#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pmax = fmaxf(pmax, __shfl_down_sync(0xffffffffu, pmax, o));
    if (lane == 0) mpart[sub] = pmax;
    if (a.mode == kCheck) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            rd2 += __shfl_down_sync(0xffffffffu, rd2, o);
            rn2 += __shfl_down_sync(0xffffffffu, rn2, o);
            rmx = fmax(rmx, __shfl_down_sync(0xffffffffu, rmx, o));
            rms += __shfl_down_sync(0xffffffffu, rms, o);
        }
        if (lane == 0) {
            rpart[sub][0] = rd2;
            rpart[sub][1] = rn2;
            rpart[sub][2] = rmx;
            rpart[sub][3] = rms;
        }
    }
    // a stored value beyond the binary16 range (it became +-inf) overflowed
    of = !(pmax * inv_sw <= 65504.f);
    if (__any_sync(0xffffffffu, of) && lane == 0) atomicOr(a.oflow, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int k = 0; k < TILES; ++k) m = fmaxf(m, mpart[k]);
        atomicMax(a.pmax, __float_as_uint(m));
        if (a.mode == kCheck) {
            double t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0;
            for (int k = 0; k < TILES; ++k) {
                t0 += rpart[k][0];
                t1 += rpart[k][1];
                t2 = fmax(t2, rpart[k][2]);
                t3 += rpart[k][3];
            }
            a.partials[4 * blockIdx.x + 0] = t0;
            a.partials[4 * blockIdx.x + 1] = t1;
            a.partials[4 * blockIdx.x + 2] = t2;
            a.partials[4 * blockIdx.x + 3] = t3;
        }
    }
}

// ---------------------------------------------------------------------------
// binary16 storage, two sites per lane.  A warp owns a tile of 64 consecutive
// sites of one x row (nx a multiple of 64, every edge at least the lattice's
// reach) and lane l the pair of sites x0 + 2l, x0 + 2l + 1: one aligned
// 4-byte word of every plane.  For velocity i the pulled elements start at
// x0 - v_x, whose parity is that of v_x, known at compile time: an even start
// is 32 aligned words (lane l's pair is word l), an odd one 33 (lane l's pair
// is the high half of word l and the low half of word l + 1).  Each lane
// copies word l of the run (lane 0 also word 32 of an odd run) into the
// velocity's 33-word slot.  After the copies each odd run is repacked in
// place into aligned pairs, and both passes read one word per velocity and
// lane, converted where it is used.  Per site, the density, relaxation, scaling,
// overflow bound and rounding are those of sweep_h16_kernel, operation for
// operation, so the two give the same results bit for bit.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned int prmt(unsigned int a, unsigned int b, unsigned int sel)
{
    unsigned int r;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(sel));
    return r;
}

// Lane's pair of a velocity from its slot (sw: this lane's word, 4 l), after
// the repack: one aligned word, low half the even site, high half the odd one.
__device__ __forceinline__ float2 h16_word(uint32_t sw)
{
    const unsigned int w = lds_b32(sw);
    return __half22float2(*reinterpret_cast<const __half2*>(&w));
}

template <class L, int TILES>
__global__ void __launch_bounds__(TILES * 32, 7)   // 128 registers: 7 blocks per SM
sweep_h16p_kernel(const SweepArgs a, const Coefs<float> c)
{
    constexpr int Q = L::Q;
    constexpr int RC = reach_of<L>();
    constexpr int W = 2 * RC + 1;
    constexpr int NC = ncls_of<L>();
    constexpr int SW = 33 * 4;                 // bytes of one velocity's slot
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double rpart[TILES][4];
    __shared__ float mpart[TILES];

    const int lane = threadIdx.x & 31;
    const int sub = threadIdx.x >> 5;
    const uint32_t slot = (uint32_t)__cvta_generic_to_shared(smem_raw) + (uint32_t)(sub * Q * SW);
    const uint32_t sw = slot + (uint32_t)(lane * 4);
    // one scratch word per lane past the slots of the block's tiles
    const uint32_t dummy = (uint32_t)__cvta_generic_to_shared(smem_raw) +
                           (uint32_t)(TILES * Q * SW + threadIdx.x * 4);
    const unsigned int* __restrict__ A = static_cast<const unsigned int*>(a.A);   // words
    unsigned int* __restrict__ B = static_cast<unsigned int*>(a.B);
    const float* __restrict__ S = static_cast<const float*>(a.S);
    const int64_t V = a.V;
    const int64_t Vw = V >> 1;                 // words per plane (V is even)
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int nw = nx >> 1;                    // words per row
    const float sr = a.sc[a.cur];
    const float inv_sw = 1.0f / a.sc[a.cur ^ 1];
    const int ntiles = (int)(V >> 6);

    double rd2 = 0.0, rn2 = 0.0, rmx = 0.0, rms = 0.0;
    float pmax = 0.f;
    const int nt = gridDim.x * TILES;
    for (int tile = blockIdx.x * TILES + sub; tile < ntiles; tile += nt) {
        const int s0 = tile * 64;              // first site: x0 = s0 mod nx, even
        const int r = (int)((unsigned)s0 / (unsigned)nx);
        const int x0 = s0 - r * nx;
        const int z = (int)((unsigned)r / (unsigned)ny);
        const int y = r - z * ny;
        int yo[W], zo[W];
        static_for<0, W>([&](auto DI) {
            constexpr int d = decltype(DI)::value - RC;
            yo[d + RC] = wrap_off<d>(y, ny) * nw;
            zo[d + RC] = wrap_off<d>(z, nz) * (ny * nw);
        });
        const int nb = a.zero_in ? 0 : 4;
        // lane's word of the run for each x displacement -R..R (the first
        // word of a run is (x0 - vx) rounded down to even, halved)
        int wl[W];
        static_for<0, W>([&](auto DI) {
            constexpr int vx = decltype(DI)::value - RC;
            int w = ((x0 - vx) >> 1) + lane;   // arithmetic shift: floor
            wl[vx + RC] = w < 0 ? w + nw : (w >= nw ? w - nw : w);
        });
        const unsigned int* plane = A;          // plane i, advanced per velocity
        static_for<0, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int vx = vx_of<L>(i);
            constexpr int oy = vy_of<L>(i) + RC;
            constexpr int oz = vz_of<L>(i) + RC;
            const unsigned int* row = plane + (zo[oz] + yo[oy]);
            plane += Vw;
            cp_async<4>(sw + (uint32_t)(i * SW), row + wl[vx + RC], nb);
            if constexpr (vx & 1) {
                // word 32 of an odd run, copied by lane 0; the other lanes
                // issue the same instruction with nothing to read, into a
                // word of their own (no branch in the unrolled pull)
                int w1 = ((x0 - vx) >> 1) + 32;
                w1 = w1 >= nw ? w1 - nw : w1;
                cp_async<4>(lane == 0 ? slot + (uint32_t)(i * SW + 128) : dummy, row + w1,
                            lane == 0 ? nb : 0);
            }
        });
        cp_async_wait_all();
        __syncwarp();
        // repack every odd run in place into aligned pairs: word l := high
        // half of word l, low half of word l + 1 (all lanes read before any
        // writes), so both passes below read one aligned word per velocity
        static_for<0, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            if constexpr (vx_of<L>(i) & 1) {
                const uint32_t ad = sw + (uint32_t)(i * SW);
                const unsigned int w = prmt(lds_b32(ad), lds_b32(ad + 4), 0x5432);
                __syncwarp();
                asm volatile("st.shared.b32 [%0], %1;" ::"r"(ad), "r"(w) : "memory");
            }
        });
        __syncwarp();

        // density: per site the four interleaved binary32 partials of
        // density_fixed_f32 (velocity k to partial k mod 4, the last Q mod 4
        // to partial 0), then the array's scale
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, b0 = 0.f, b1 = 0.f, b2 = 0.f, b3 = 0.f;
#pragma unroll 2
        for (int k = 0; k + 3 < Q; k += 4) {
            const float2 v0 = h16_word(sw + (uint32_t)((k + 0) * SW));
            const float2 v1 = h16_word(sw + (uint32_t)((k + 1) * SW));
            const float2 v2 = h16_word(sw + (uint32_t)((k + 2) * SW));
            const float2 v3 = h16_word(sw + (uint32_t)((k + 3) * SW));
            a0 += v0.x; b0 += v0.y;
            a1 += v1.x; b1 += v1.y;
            a2 += v2.x; b2 += v2.y;
            a3 += v3.x; b3 += v3.y;
        }
#pragma unroll
        for (int k = Q - Q % 4; k < Q; ++k) {
            const float2 v = h16_word(sw + (uint32_t)(k * SW));
            a0 += v.x; b0 += v.y;
        }
        const float PhiA = ((a0 + a1) + (a2 + a3)) * sr;
        const float PhiB = ((b0 + b1) + (b2 + b3)) * sr;
        // the written array's scale inv_sw is a power of two, so it enters the
        // relaxation factor and the per-class terms exactly: the products
        // below are the stored values p / sc, bit for bit those of p * inv_sw
        const float om1w = c.om1 * sr * inv_sw;
        const int s = s0 + 2 * lane;
        const float2 S2 = *reinterpret_cast<const float2*>(S + s);
        const float SxA = (float)((double)S2.x + a.soff);
        const float SxB = (float)((double)S2.y + a.soff);
        unsigned int* dst = B + (s >> 1);       // plane i's word of the pair, per velocity
        static_for<0, NC>([&](auto CI) {
            constexpr int cl = decltype(CI)::value;
            constexpr int i0 = cls_begin<L>(cl), i1 = cls_begin<L>(cl + 1);
            const float eA = fmaf(c.wphi[cl], PhiA, c.chi[cl] * SxA) * inv_sw;
            const float eB = fmaf(c.wphi[cl], PhiB, c.chi[cl] * SxB) * inv_sw;
#pragma unroll 4
            for (int i = i0; i < i1; ++i) {
                const float2 v = h16_word(sw + (uint32_t)(i * SW));
                const float qA = fmaf(om1w, v.x, eA);   // p / sc of the written array
                const float qB = fmaf(om1w, v.y, eB);
                pmax = fmaxf(pmax, fmaxf(fabsf(qA), fabsf(qB)));
                const __half2 h = __floats2half2_rn(qA, qB);
                __stcs(dst, *reinterpret_cast<const unsigned int*>(&h));
                dst += Vw;
            }
        });
        if (a.mode != kPlain) {
            const double phA = (double)PhiA, phB = (double)PhiB;
            if (a.mode == kCheck) {
                const double2 old = *reinterpret_cast<const double2*>(a.Phi + s);
                const double dA = phA - old.x, dB = phB - old.y;
                rd2 += dA * dA;
                rd2 += dB * dB;
                rn2 += phA * phA;
                rn2 += phB * phB;
                rmx = fmax(rmx, fmax(fabs(dA), fabs(dB)));
                rms += phA;
                rms += phB;
            }
            *reinterpret_cast<double2*>(a.Phi + s) = make_double2(phA, phB);
        }
        __syncwarp();
    }

    // pmax holds max |p| / sc (the stored magnitudes): back to max |p|, exactly
    pmax = pmax / inv_sw;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pmax = fmaxf(pmax, __shfl_down_sync(0xffffffffu, pmax, o));
    if (lane == 0) mpart[sub] = pmax;
    if (a.mode == kCheck) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            rd2 += __shfl_down_sync(0xffffffffu, rd2, o);
            rn2 += __shfl_down_sync(0xffffffffu, rn2, o);
            rmx = fmax(rmx, __shfl_down_sync(0xffffffffu, rmx, o));
            rms += __shfl_down_sync(0xffffffffu, rms, o);
        }
        if (lane == 0) {
            rpart[sub][0] = rd2;
            rpart[sub][1] = rn2;
            rpart[sub][2] = rmx;
            rpart[sub][3] = rms;
        }
    }
    // a stored value beyond the binary16 range (it became +-inf) overflowed
    const int of = !(pmax * inv_sw <= 65504.f);
    if (__any_sync(0xffffffffu, of) && lane == 0) atomicOr(a.oflow, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int k = 0; k < TILES; ++k) m = fmaxf(m, mpart[k]);
        atomicMax(a.pmax, __float_as_uint(m));
        if (a.mode == kCheck) {
            double t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0;
            for (int k = 0; k < TILES; ++k) {
                t0 += rpart[k][0];
                t1 += rpart[k][1];
                t2 = fmax(t2, rpart[k][2]);
                t3 += rpart[k][3];
            }
            a.partials[4 * blockIdx.x + 0] = t0;
            a.partials[4 * blockIdx.x + 1] = t1;
            a.partials[4 * blockIdx.x + 2] = t2;
            a.partials[4 * blockIdx.x + 3] = t3;
        }
    }
}

// binary16 geometries: 0 one site per lane (any grid), 1 two sites per lane
// (nx a multiple of 64 and no edge below the reach; the plan checks).
constexpr int kH16Tiles = 2;
template <class L>
constexpr size_t h16_smem(int variant)
{
    return variant == 1 ? (size_t)kH16Tiles * (L::Q * 33 * 4 + 32 * 4)
                        : (size_t)kH16Tiles * L::Q * 32 * 4;
}

template <class L>
int launch_sweep_h16(int variant, const SweepArgs& a, const void* coefs, int grid, void* stream)
{
    const Coefs<float>& c = *static_cast<const Coefs<float>*>(coefs);
    if (variant == 1)
        sweep_h16p_kernel<L, kH16Tiles><<<grid, kH16Tiles * 32, h16_smem<L>(1),
                                         (cudaStream_t)stream>>>(a, c);
    else
        sweep_h16_kernel<L, kH16Tiles><<<grid, kH16Tiles * 32, h16_smem<L>(0),
                                        (cudaStream_t)stream>>>(a, c);
    return (int)cudaGetLastError();
}

template <class L>
int occupancy_h16(int variant, int* blocks, int* tiles_per_block)
{
    const size_t smem = h16_smem<L>(variant);
    auto kern = variant == 1 ? sweep_h16p_kernel<L, kH16Tiles> : sweep_h16_kernel<L, kH16Tiles>;
    cudaError_t e = set_sweep_smem(kern, smem);
    if (e != cudaSuccess) return (int)e;
    // tiles_per_block counts 32-site tiles: a two-site tile is two of them
    *tiles_per_block = variant == 1 ? 2 * kH16Tiles : kH16Tiles;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern, kH16Tiles * 32, smem);
}

// ---------------------------------------------------------------------------
// omega = 1 (tau_lb = 1, the paper's setting): the collision forgets the
// pulled populations, f_i = phi_i Phi + chi_i S, so one step is the scalar
// stencil  Phi'(x) = sum_i w_i Phi(x - v_i) + St(x)  with w_i = phi_i and
// St = sum_i chi_i S(x - v_i) (the same kernel with w_i = chi_i, St = 0,
// builds St once).  One thread per site; the Q neighbour reads hit L1/L2.
// On check steps it adds |dPhi|^2, |Phi|^2, max |dPhi| and sum Phi of its
// block to partials (4 doubles per block).
// ---------------------------------------------------------------------------
template <class L>
__global__ void __launch_bounds__(256)
stencil_kernel(const double* __restrict__ Pin, double* __restrict__ Pout,
               const double* __restrict__ St, const Coefs<double> c, int64_t V, int nx, int ny,
               int nz, int small, int check, double* partials, const int* stop)
{
    if (stop != nullptr && *stop != 0) return;   // the run stopped before this step
    constexpr int Q = L::Q;
    constexpr int RC = reach_of<L>();
    constexpr int W = 2 * RC + 1;
    __shared__ double red[8][4];
    const int nxy = nx * ny;
    double d2 = 0.0, n2 = 0.0, mx = 0.0, ms = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s64 < V; s64 += stride) {
        const int s = (int)s64;
        const int x = s % nx;
        const int r = s / nx;
        const int y = r % ny;
        const int z = r / ny;
        int xs[W], yo[W], zo[W];
#pragma unroll
        for (int d = -RC; d <= RC; ++d) {
            if (small) {
                xs[d + RC] = wrap_any(x - d, nx);
                yo[d + RC] = wrap_any(y - d, ny) * nx;
                zo[d + RC] = wrap_any(z - d, nz) * nxy;
            } else {
                xs[d + RC] = wrap_near(x - d, nx);
                yo[d + RC] = wrap_near(y - d, ny) * nx;
                zo[d + RC] = wrap_near(z - d, nz) * nxy;
            }
        }
        double acc = St ? St[s] : 0.0;
        static_for<0, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int ox = vx_of<L>(i) + RC;
            constexpr int oy = vy_of<L>(i) + RC;
            constexpr int oz = vz_of<L>(i) + RC;
            acc = fma(c.wphi[cls_of<L>(i)], __ldg(Pin + (zo[oz] + yo[oy] + xs[ox])), acc);
        });
        Pout[s] = acc;
        if (check) {
            const double d = acc - Pin[s];
            d2 += d * d;
            n2 += acc * acc;
            mx = fmax(mx, fabs(d));
            ms += acc;
        }
    }
    if (check) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            d2 += __shfl_down_sync(0xffffffffu, d2, o);
            n2 += __shfl_down_sync(0xffffffffu, n2, o);
            mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
            ms += __shfl_down_sync(0xffffffffu, ms, o);
        }
        const int w = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0) {
            red[w][0] = d2;
            red[w][1] = n2;
            red[w][2] = mx;
            red[w][3] = ms;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
                t0 += red[k][0];
                t1 += red[k][1];
                t2 = fmax(t2, red[k][2]);
                t3 += red[k][3];
            }
            partials[4 * blockIdx.x + 0] = t0;
            partials[4 * blockIdx.x + 1] = t1;
            partials[4 * blockIdx.x + 2] = t2;
            partials[4 * blockIdx.x + 3] = t3;
        }
    }
}

template <class L>
int launch_stencil(const double* Pin, double* Pout, const double* St, const Coefs<double>& c,
                   int64_t V, int nx, int ny, int nz, int small, int check, double* partials,
                   int grid, void* stream, const int* stop)
{
    const int block = (int64_t)grid * 64 >= V ? 64 : 256;   // see stencil_block
    stencil_kernel<L><<<grid, block, 0, (cudaStream_t)stream>>>(Pin, Pout, St, c, V, nx, ny, nz,
                                                                small, check, partials, stop);
    return (int)cudaGetLastError();
}

}  // namespace pkr

#include "pkr_sweep_pair.cuh"
#include "pkr_sweep_ws.cuh"

namespace pkr {

template <class L, typename T, int K>
int launch_variant(const SweepArgs& a, const void* coefs, int grid, void* stream)
{
    using R = typename AccType<T>::type;
    constexpr Geo geo = Variants<L>::at(K);
    using ST = Staged<L, T, geo.G, geo.TILES>;
    sweep_staged_kernel<L, T, geo.G, geo.TILES><<<grid, ST::WARPS * 32, ST::smem_bytes(),
                                                  (cudaStream_t)stream>>>(
        a, *static_cast<const Coefs<R>*>(coefs));
    return (int)cudaGetLastError();
}

template <class L, typename T, int K>
int occupancy_variant(int* blocks, int* tiles_per_block)
{
    constexpr Geo geo = Variants<L>::at(K);
    using ST = Staged<L, T, geo.G, geo.TILES>;
    auto kern = sweep_staged_kernel<L, T, geo.G, geo.TILES>;
    cudaError_t e = set_sweep_smem(kern, ST::smem_bytes());
    if (e != cudaSuccess) return (int)e;
    *tiles_per_block = geo.TILES;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern, ST::WARPS * 32,
                                                              ST::smem_bytes());
}

// Run-time dispatch over the compiled variants of (L, T): the staged
// geometries of Variants<L>, then the warp-specialised ones of WsVariants<L>.
template <class L, typename T>
int launch_sweep_t(int variant, const SweepArgs& a, const void* coefs, int grid, void* stream)
{
    int rc = (int)cudaErrorInvalidValue;
    static_for<0, Variants<L>::N>([&](auto K) {
        if (variant == decltype(K)::value)
            rc = launch_variant<L, T, decltype(K)::value>(a, coefs, grid, stream);
    });
    static_for<0, WsVariants<L>::N>([&](auto K) {
        if (variant == Variants<L>::N + decltype(K)::value)
            rc = launch_ws_variant<L, T, decltype(K)::value>(a, coefs, grid, stream);
    });
    static_for<0, PairVariant<L>::N>([&](auto K) {
        if (variant == Variants<L>::N + WsVariants<L>::N + decltype(K)::value)
            rc = launch_pair_variant<L, T, decltype(K)::value>(a, coefs, grid, stream);
    });
    return rc;
}

template <class L, typename T>
int occupancy_t(int variant, int* blocks, int* tiles_per_block)
{
    int rc = (int)cudaErrorInvalidValue;
    static_for<0, Variants<L>::N>([&](auto K) {
        if (variant == decltype(K)::value)
            rc = occupancy_variant<L, T, decltype(K)::value>(blocks, tiles_per_block);
    });
    static_for<0, WsVariants<L>::N>([&](auto K) {
        if (variant == Variants<L>::N + decltype(K)::value)
            rc = occupancy_ws_variant<L, T, decltype(K)::value>(blocks, tiles_per_block);
    });
    static_for<0, PairVariant<L>::N>([&](auto K) {
        if (variant == Variants<L>::N + WsVariants<L>::N + decltype(K)::value)
            rc = occupancy_pair_variant<L, T, decltype(K)::value>(blocks, tiles_per_block);
    });
    return rc;
}

// Variants of a plan's sweep (staged, warp-specialised, then the aligned x
// pairs, which need nx a multiple of 64 and every edge at least the reach)
// and of the batch sweep (staged only).
template <class L>
int variant_count_t() { return Variants<L>::N + WsVariants<L>::N + PairVariant<L>::N; }
// first aligned x-pairs variant (they are the last PairVariant<L>::N), or -1
template <class L>
int pair_variant_t() { return PairVariant<L>::N > 0 ? Variants<L>::N + WsVariants<L>::N : -1; }
template <class L>
int batch_variant_count_t() { return Variants<L>::N; }

#define PKR_INSTANTIATE_SWEEP(L)                                                             \
    template int launch_sweep_t<L, double>(int, const SweepArgs&, const void*, int, void*); \
    template int launch_sweep_t<L, long long>(int, const SweepArgs&, const void*, int, void*); \
    template int occupancy_t<L, long long>(int, int*, int*);                                 \
    template int launch_sweep_t<L, float>(int, const SweepArgs&, const void*, int, void*);  \
    template int occupancy_t<L, double>(int, int*, int*);                                    \
    template int occupancy_t<L, float>(int, int*, int*);                                     \
    template int variant_count_t<L>();                                                      \
    template int batch_variant_count_t<L>();                                                \
    template int pair_variant_t<L>();                                                       \
    template int launch_sweep_h16<L>(int, const SweepArgs&, const void*, int, void*);        \
    template int occupancy_h16<L>(int, int*, int*);                                          \
    template int launch_stencil<L>(const double*, double*, const double*, const Coefs<double>&,  \
                                   int64_t, int, int, int, int, int, double*, int, void*,       \
                                   const int*);                                                 \
    template int launch_batch_t<L, double>(int, BatchState*, int, int, void*);               \
    template int launch_batch_t<L, float>(int, BatchState*, int, int, void*);                \
    template int launch_batch_t<L, long long>(int, BatchState*, int, int, void*);            \
    template int batch_occupancy_t<L, double>(int, int*);                                    \
    template int batch_occupancy_t<L, long long>(int, int*);                                 \
    template int batch_occupancy_t<L, float>(int, int*);

}  // namespace pkr
