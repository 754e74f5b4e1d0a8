// pkr_sweep_pair.cuh -- the staged sweep with the pull's x offsets served
// from aligned runs (included by pkr_sweep.cuh; same step, same arithmetic as
// the 2 velocity groups x 2 tiles geometry, bit for bit).
//
// In the staged sweep every warp copies, for each velocity, the 32 values
// x0 - v_x .. x0 - v_x + 31 of its row: for v_x != 0 the 256-byte run starts
// off a 128-byte line and touches three lines: more L1/L2 requests than a
// whole-line run (a copy through that staging reaches 0.72 of the peak).
// Here a block's two tiles are x-adjacent (64 sites of one row: nx a multiple
// of 64).  For velocity i the group's two warps copy the two aligned 32-site
// blocks x0 .. x0 + 63 of the velocity's source row, plus H halo values on
// the side v_x needs (x0 - H .. x0 - 1 for v_x > 0, x0 + 64 .. x0 + 63 + H
// for v_x < 0; H = the lattice's reach), into the velocity's row of 64 + 2H
// values in shared memory, each value x written at position H + (x - x0) +
// v_x.  The rows are as short as the reach allows because the copies land
// in L1 on their way to shared memory: with H = 3 three D3Q111 blocks of
// 8-byte rows (62.2 KB + 2.1-2.6 KB of exchange rows each) fit the 196 KB
// shared split of the SM and leave 60 KB of L1; with H = 4 they took the
// 228 KB split (28 KB of L1), 13 % slower in 64-bit fixed point and 6 % in
// binary64 (256^3, early refill).  Site x0 + p then finds its pulled value
// x0 + p - v_x at position H + p: the rows read like the staged sweep's
// columns, 64 + 2H values apart, and the density and relaxation code
// (group_compute) runs unchanged.  The two warps of a velocity group meet at
// a named barrier after the copies (each reads values the other copied) and
// again before rows are refilled: after the whole pair, or, in the
// early-refill form, after each symmetry class, whose rows then take the
// block's next pair while the remaining classes are relaxed.
#pragma once

namespace pkr {

template <class L, typename T>
struct Pair {
    static constexpr int Q = L::Q;
    static constexpr int H = reach_of<L>();                // halo values per side
    static constexpr int RL = 64 + 2 * H;                  // values per row
    static constexpr int ROWB = RL * (int)sizeof(T);       // bytes per row
    static constexpr size_t smem_bytes() { return (size_t)Q * ROWB; }
};

// The pair geometry applies: x rows of whole 64-site pairs, every edge at
// least the reach (the per-tile offsets wrap each side at most once).  Two
// forms, both with 2 velocity groups: k = 0 fills a pair's rows, computes,
// and only then fills the rows again for the block's next pair; k = 1
// refills a symmetry class's rows for the next pair as soon as both warps of
// the group have relaxed that class, so the copies of the next pair are in
// flight while the rest of this pair is computed.
template <class L>
struct PairVariant {
    static constexpr int N = (L::Q > 64) ? 2 : 0;
    static constexpr int groups(int) { return 2; }
    static constexpr bool early_refill(int k) { return k == 1; }
};

// Filling the rows of one pair, in the warp (sub = tile of the pair) and
// lane that run it: locate() takes the pair's first x, the y and z row
// offsets of the pull and this lane's halo positions (one value per lane
// < H); pull<i>() issues the copies of velocity i, value x to position
// H + (x - x0) + v_x of row i (nbytes = 0: zero fill).  Every copy is one
// value per lane: 16-byte chunks for the rows whose values land 16-byte
// aligned (H + v_x even), copied past L1, measured no faster in 64-bit fixed
// point and 4 % slower in binary64 at 256^3.
template <class L, typename T>
struct PairFill {
    static constexpr int RC = reach_of<L>();
    static constexpr int W = 2 * RC + 1;
    static constexpr int H = Pair<L, T>::H;
    static constexpr int ROWB = Pair<L, T>::ROWB;
    static constexpr int ES = (int)sizeof(T);
    int yo[W], zo[W];
    int x0 = 0, xl = 0, xr = 0;

    __device__ __forceinline__ void locate(int p, int nx, int ny, int nz, int lane)
    {
        const int s0 = p * 64;
        const int r = (int)((unsigned)s0 / (unsigned)nx);
        x0 = s0 - r * nx;
        const int z = (int)((unsigned)r / (unsigned)ny);
        const int y = r - z * ny;
        const int nxy = nx * ny;
        static_for<0, W>([&](auto DI) {
            constexpr int d = decltype(DI)::value - RC;
            yo[d + RC] = wrap_off<d>(y, ny) * nx;
            zo[d + RC] = wrap_off<d>(z, nz) * nxy;
        });
        xl = (x0 >= H ? x0 - H : x0 - H + nx) + lane;
        xr = (x0 + 64 < nx ? x0 + 64 : 0) + lane;
    }

    template <int i>
    __device__ __forceinline__ void pull(const T* __restrict__ A, int64_t V, uint32_t base,
                                         int sub, int lane, int nbytes) const
    {
        constexpr int vx = vx_of<L>(i);
        constexpr int oy = vy_of<L>(i) + RC;
        constexpr int oz = vz_of<L>(i) + RC;
        const T* row = A + ((int64_t)i * V + (zo[oz] + yo[oy]));
        const uint32_t rb = base + (uint32_t)(i * ROWB);
        cp_async<sizeof(T)>(rb + (uint32_t)((H + 32 * sub + lane + vx) * ES),
                            row + (x0 + 32 * sub + lane), nbytes);
        if constexpr (vx > 0) {
            if (sub == 0 && lane < H)
                cp_async<sizeof(T)>(rb + (uint32_t)((lane + vx) * ES), row + xl, nbytes);
        } else if constexpr (vx < 0) {
            if (sub == 1 && lane < H)
                cp_async<sizeof(T)>(rb + (uint32_t)((H + 64 + lane + vx) * ES), row + xr,
                                    nbytes);
        }
    }
};

// First velocity of the last symmetry class that velocities lo .. hi - 1 hold.
template <class L>
__host__ __device__ constexpr int tail_begin(int lo, int hi)
{
    const int b = cls_begin<L>(cls_of<L>(hi - 1));
    return b > lo ? b : lo;
}

template <class L, typename T, int G, bool EARLY>
__global__ void __launch_bounds__(64 * G)
sweep_pair_kernel(const SweepArgs a, const Coefs<typename AccType<T>::type> c)
{
    if (a.stop != nullptr && *a.stop != 0) return;   // the run stopped before this step
    using R = typename AccType<T>::type;
    using PR = Pair<L, T>;
    constexpr int Q = L::Q;
    constexpr int H = PR::H;
    constexpr int ROWB = PR::ROWB;
    constexpr int ES = (int)sizeof(T);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double rpart[2][4];
    // per-group partial densities of a tile, two sets used by turns (a warp
    // writes the next pair's partial only after that pair's exchange barrier)
    __shared__ long long xacc[2][2][G][32];
    __shared__ int xexp[2][G][32];   // per-group largest exponents

    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int grp = wib % G;     // velocity group of this warp
    const int sub = wib / G;     // tile of the pair: sites x0 + 32 sub + lane
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(smem_raw);
    const bool fx = std::is_same<T, long long>::value;
    const T* __restrict__ A = static_cast<const T*>(a.A);
    const TileGrid<T> tg{A, static_cast<T*>(a.B),
                         static_cast<const typename SrcType<T>::type*>(a.S), a.Phi, a.V, a.nx,
                         a.ny, a.nz, a.small, a.soff, fx ? a.fxF[a.cur] : 0,
                         fx ? a.fxF[a.cur ^ 1] : 0, a.cfx};
    const int64_t V = a.V;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int npairs = (int)(V >> 6);
    const int nbytes = a.zero_in ? 0 : ES;

    PairFill<L, T> fill;   // the pair whose rows are being filled
    auto pull = [&](auto I) {
        fill.template pull<decltype(I)::value>(A, V, base, sub, lane, nbytes);
    };

    // early refill: the copies of each symmetry class form one cp.async
    // group, so a pair can start on every row but its group's last class
    // (refilled last, at the end of the previous pair) while those land.
    // Binary64 does (2.76 against 2.73 GLUPS at 256^3); fixed point and
    // binary32 measured 0.3 % and 0.6 % slower with the split and wait for
    // every row first.
    constexpr bool TAIL = std::is_same<T, double>::value;
    if constexpr (EARLY) {
        if ((int)blockIdx.x < npairs) {
            fill.locate((int)blockIdx.x, nx, ny, nz, lane);
            static_for<0, G>([&](auto GI) {
                constexpr int g = decltype(GI)::value;
                constexpr int lo = g * Q / G, hi = (g + 1) * Q / G;
                constexpr int tb = tail_begin<L>(lo, hi);
                if (grp == g) {
                    static_for<lo, tb>(pull);
                    if constexpr (TAIL) cp_async_commit();
                    static_for<tb, hi>(pull);
                    if constexpr (TAIL) cp_async_commit();
                }
            });
        }
    }

    double rd2 = 0.0, rn2 = 0.0, rmx = 0.0, rms = 0.0;
    unsigned long long fxm = 0ull;
    int par = 0;
    for (int pr = blockIdx.x; pr < npairs; pr += gridDim.x, par ^= 1) {
        const int s = pr * 64 + 32 * sub + lane;   // this lane's site
        // the source offset (mass correction) is used by binary32 storage only
        R Sx;
        if constexpr (std::is_same<T, float>::value) Sx = (R)((double)tg.S[s] + tg.soff);
        else Sx = (R)tg.S[s];
        const bool more = pr + (int)gridDim.x < npairs;   // the block has a next pair
        if constexpr (EARLY) {
            if (more) fill.locate(pr + (int)gridDim.x, nx, ny, nz, lane);
        } else {
            fill.locate(pr, nx, ny, nz, lane);
        }

        static_for<0, G>([&](auto GI) {
            constexpr int g = decltype(GI)::value;
            constexpr int lo = g * Q / G, hi = (g + 1) * Q / G;
            if (grp != g) return;
            if constexpr (!EARLY) {
                static_for<lo, hi>(pull);
                cp_async_wait_all();
            } else if constexpr (TAIL) {
                cp_async_wait_all_but_last();   // all rows but the last class's
            } else {
                cp_async_wait_all();
            }
            // the group's other warp copied half of the values this one reads
            asm volatile("bar.sync %0, 64;" ::"r"(3 + g) : "memory");
            const uint32_t sb = base + (uint32_t)(lo * ROWB + (H + 32 * sub + lane) * ES);
            if constexpr (EARLY) {
                constexpr int tb = tail_begin<L>(lo, hi);
                group_compute<L, T, G, g, ROWB, TAIL ? tb - lo : -1>(
                    tg, c, a.mode, true, s, Sx, lane, sb, 1 + sub, xacc[par][sub], xexp[sub], rd2,
                    rn2, rmx, rms, fxm,
                    [&](auto CI) {
                        constexpr int cl = decltype(CI)::value;
                        constexpr int cb = cls_begin<L>(cl), ce = cls_begin<L>(cl + 1);
                        constexpr int i0 = cb > lo ? cb : lo;
                        constexpr int i1 = ce < hi ? ce : hi;
                        // both warps are done with the class's rows
                        asm volatile("bar.sync %0, 64;" ::"r"(3 + g) : "memory");
                        if (more) {
                            static_for<i0, i1>(pull);
                            if constexpr (TAIL) cp_async_commit();
                        }
                    },
                    [&]() {
                        // the last class's rows, of both warps of the group
                        cp_async_wait_committed();
                        asm volatile("bar.sync %0, 64;" ::"r"(3 + g) : "memory");
                    });
            } else {
                group_compute<L, T, G, g, ROWB>(tg, c, a.mode, true, s, Sx, lane, sb, 1 + sub,
                                                xacc[par][sub], xexp[sub], rd2, rn2, rmx, rms,
                                                fxm);
                // both warps are done with the rows before either refills them
                asm volatile("bar.sync %0, 64;" ::"r"(3 + g) : "memory");
            }
        });
        __syncwarp();
    }
    if constexpr (std::is_same<T, long long>::value) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) fxm |= __shfl_down_sync(0xffffffffu, fxm, o);
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
            for (int k = 0; k < 2; ++k) {
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

template <class L, typename T, int K>
int launch_pair_variant(const SweepArgs& a, const void* coefs, int grid, void* stream)
{
    using R = typename AccType<T>::type;
    constexpr int G = PairVariant<L>::groups(K);
    constexpr bool EARLY = PairVariant<L>::early_refill(K);
    sweep_pair_kernel<L, T, G, EARLY><<<grid, 64 * G, Pair<L, T>::smem_bytes(), (cudaStream_t)stream>>>(
        a, *static_cast<const Coefs<R>*>(coefs));
    return (int)cudaGetLastError();
}

template <class L, typename T, int K>
int occupancy_pair_variant(int* blocks, int* tiles_per_block)
{
    constexpr int G = PairVariant<L>::groups(K);
    constexpr bool EARLY = PairVariant<L>::early_refill(K);
    auto kern = sweep_pair_kernel<L, T, G, EARLY>;
    const size_t smem = Pair<L, T>::smem_bytes();
    cudaError_t e = set_sweep_smem(kern, smem);
    if (e != cudaSuccess) return (int)e;
    *tiles_per_block = 2;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern, 64 * G, smem);
}

}  // namespace pkr
