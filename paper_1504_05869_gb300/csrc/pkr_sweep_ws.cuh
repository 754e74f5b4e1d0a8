// pkr_sweep_ws.cuh -- warp-specialised form of the fused stream-and-collide
// sweep (included by pkr_sweep.cuh; same step, same arithmetic, bit for bit).
//
// The staged sweep runs pull, density and relaxation of a tile in one set of
// warps, one phase after the other: a warp that waits for its pulled values
// leaves the FP64 pipe idle, and shared memory (one tile of Q values per
// tile slot) caps the number of warps that could cover for it.  On GB300 the
// binary64 relaxation (one FMA per velocity and site on a pipe of about two
// FMAs per clock per SM) keeps that pipe more than half busy at the HBM
// roofline, so the pull latency has to leave the warps that feed it.
//
// Here a block (one per SM) owns NS = NG x SPG tile slots in shared memory
// and two kinds of warps:
//   loader warp f (f < NS) owns slot f: for each tile it is given it pulls
//     the Q values of the tile's 32 sites and their source values into the
//     slot (per-lane cp.async, zero-fill past the end and, for the
//     populations, on the first step), waits for the copies and marks the
//     slot ready;
//   compute group g (NG groups of G warps, one velocity group per warp, as
//     in the staged sweep) takes the block's tiles j = g, g + NG, ... in
//     order, its m-th tile in its slot g SPG + (m mod SPG): it forms the
//     exact density, relaxes and stores (group_compute, the staged sweep's
//     own code), then marks the slot free.
// With SPG = 2 a group's next tile is loaded while it works on the current
// one, and NG groups interleave their integer (density) and FP64
// (relaxation) phases on every SM sub-partition.
//
// Slot hand-offs are named barriers with fixed arrival counts: ready[f]
// (barrier 1 + f) and free[f] (barrier 1 + NS + f), each met by the 32
// threads of loader f and the 32 G threads of the one group that uses slot f.
// For a slot that receives m tiles the loader arrives m times on ready and
// waits m times on free (before each reuse, and once after its last tile);
// the group waits m times on ready and arrives m times on free.  Every phase
// therefore completes, and a phase cannot start before the previous one of
// the same barrier has completed (a loader refills a slot only after free,
// which needs the group to have passed ready for the slot's previous tile).
// The G warps of group g also meet at barrier 1 + 2 NS + g inside each tile
// (density exchange), as the G warps of a staged tile do.
#pragma once

namespace pkr {

__device__ __forceinline__ void nbar_sync(int id, int n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void nbar_arrive(int id, int n)
{
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

template <class L, typename T, int NG_, int G_, int SPG_>
struct Ws {
    using SRC = typename SrcType<T>::type;
    static constexpr int Q = L::Q;
    static constexpr int NG = NG_;
    static constexpr int G = G_;
    // one slot: Q pulled values and the source value of 32 sites
    static constexpr int VAL_BYTES = Q * 32 * (int)sizeof(T);
    static constexpr int SLOT = VAL_BYTES + 32 * (int)sizeof(SRC);
    // slots per group: as asked, or fewer where 220 KB cannot hold them
    static constexpr int SPG_FIT = (220 * 1024) / (NG * SLOT);
    static constexpr int SPG = SPG_ < SPG_FIT ? SPG_ : SPG_FIT;
    static constexpr int NS = NG * SPG;
    static constexpr int WARPS = NS + NG * G;
    static constexpr int NB = 32 * (1 + G);   // threads meeting at a slot barrier
    static constexpr size_t smem_bytes() { return (size_t)NS * SLOT; }
    static_assert(SPG >= 1, "no slot fits");
    static_assert(2 * NS + NG + 1 <= 16, "more named barriers than a block has");
};

// Warp-specialised geometries per lattice, (groups, warps per group, slots
// per group), after the staged ones in the lattice's variant list.
struct WsGeo {
    int NG, G, SPG;
};
template <class L>
struct WsVariants {
    static constexpr int N = (L::Q > 64) ? 1 : 0;
    static constexpr WsGeo at(int) { return WsGeo{3, 4, 2}; }
};

// Loader, one tile: pull the tile's Q values and its source values into a
// slot and wait for them.  sb: this lane's column of the slot's values; cb:
// this lane's source word.
template <class L, typename T>
__device__ __forceinline__ void ws_pull(const SweepArgs& a, int tile, int lane, uint32_t sb,
                                        uint32_t cb)
{
    using SRC = typename SrcType<T>::type;
    constexpr int Q = L::Q;
    constexpr int RC = reach_of<L>();
    constexpr int W = 2 * RC + 1;
    constexpr int ST = 32 * (int)sizeof(T);
    const T* __restrict__ A = static_cast<const T*>(a.A);
    const int64_t V = a.V;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int nxy = nx * ny;

    const int64_t s64 = (int64_t)tile * 32 + lane;
    const bool valid = s64 < V;
    const int s = valid ? (int)s64 : 0;
    const int r = (int)((unsigned)s / (unsigned)nx);
    const int x = s - r * nx;
    const int z = (int)((unsigned)r / (unsigned)ny);
    const int y = r - z * ny;
    int xs[W], yo[W], zo[W];
    if (a.small) {
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
    const int nbytes = (valid && !a.zero_in) ? (int)sizeof(T) : 0;
    cp_async<sizeof(SRC)>(cb, static_cast<const SRC*>(a.S) + s, valid ? (int)sizeof(SRC) : 0);
    static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int ox = vx_of<L>(i) + RC;
        constexpr int oy = vy_of<L>(i) + RC;
        constexpr int oz = vz_of<L>(i) + RC;
        const T* src = A + ((int64_t)i * V + (zo[oz] + yo[oy] + xs[ox]));
        cp_async<sizeof(T)>(sb + (uint32_t)(i * ST), src, nbytes);
    });
    cp_async_wait_all();
}

template <class L, typename T, int NG, int G, int SPG>
__global__ void __launch_bounds__(Ws<L, T, NG, G, SPG>::WARPS * 32, 1)
sweep_ws_kernel(const SweepArgs a, const Coefs<typename AccType<T>::type> c)
{
    if (a.stop != nullptr && *a.stop != 0) return;   // the run stopped before this step
    using R = typename AccType<T>::type;
    using WS = Ws<L, T, NG, G, SPG>;
    using SRC = typename WS::SRC;
    constexpr int NS = WS::NS;
    constexpr int NB = WS::NB;
    constexpr int SP = WS::SPG;
    constexpr int ST = 32 * (int)sizeof(T);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ long long xacc[2][NG][G][32];   // per-group partial densities, two sets by turns
    __shared__ int xexp[NG][G][32];         // per-group largest exponents
    __shared__ double rpart[NG][4];

    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const uint32_t sm0 = (uint32_t)__cvta_generic_to_shared(smem_raw);
    // tiles of this block: blockIdx.x + j gridDim.x for j < nb
    const int nb = (int)blockIdx.x < a.ntiles
                       ? (a.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1
                       : 0;

    if (wib < NS) {
        const int f = wib;
        const int g = f / SP;
        const uint32_t sb = sm0 + (uint32_t)(f * WS::SLOT + lane * (int)sizeof(T));
        const uint32_t cb = sm0 + (uint32_t)(f * WS::SLOT + WS::VAL_BYTES + lane * (int)sizeof(SRC));
        bool first = true;
        for (int j = g + NG * (f % SP); j < nb; j += NS) {
            if (!first) nbar_sync(1 + NS + f, NB);      // the slot's previous tile is done
            ws_pull<L, T>(a, (int)blockIdx.x + j * (int)gridDim.x, lane, sb, cb);
            __syncwarp();
            nbar_arrive(1 + f, NB);                     // slot ready
            first = false;
        }
        if (!first) nbar_sync(1 + NS + f, NB);          // balances the last free arrival
    } else {
        const int w = wib - NS;
        const int g = w / G;     // compute group
        const int q = w % G;     // velocity group of this warp
        const bool fx = std::is_same<T, long long>::value;
        const TileGrid<T> tg{static_cast<const T*>(a.A), static_cast<T*>(a.B),
                             static_cast<const SRC*>(a.S), a.Phi, a.V, a.nx, a.ny, a.nz,
                             a.small, a.soff, fx ? a.fxF[a.cur] : 0, fx ? a.fxF[a.cur ^ 1] : 0,
                             a.cfx};
        double d2 = 0.0, n2 = 0.0, mx = 0.0, ms = 0.0;
        unsigned long long fxm = 0ull;
        int sl = 0, par = 0;
        for (int j = g; j < nb; j += NG, par ^= 1) {
            const int f = g * SP + sl;
            const int tile = (int)blockIdx.x + j * (int)gridDim.x;
            const int64_t s64 = (int64_t)tile * 32 + lane;
            const bool valid = s64 < a.V;
            const int s = valid ? (int)s64 : 0;
            const uint32_t sb = sm0 + (uint32_t)(f * WS::SLOT + lane * (int)sizeof(T));
            const uint32_t cb =
                sm0 + (uint32_t)(f * WS::SLOT + WS::VAL_BYTES + lane * (int)sizeof(SRC));
            nbar_sync(1 + f, NB);                       // slot ready
            // the source offset (mass correction) is used by binary32 storage only
            R Sx = R(0);
            if (valid) {
                if constexpr (std::is_same<T, float>::value)
                    Sx = (R)((double)lds_f32(cb) + a.soff);
                else Sx = (R)lds_f64(cb);
            }
            static_for<0, G>([&](auto QI) {
                constexpr int qq = decltype(QI)::value;
                if (q == qq)
                    group_compute<L, T, G, qq>(tg, c, a.mode, valid, s, Sx, lane,
                                               sb + (uint32_t)((qq * L::Q / G) * ST),
                                               1 + 2 * NS + g, xacc[par][g], xexp[g], d2, n2, mx, ms,
                                               fxm);
            });
            __syncwarp();                               // lanes past the end rejoin
            nbar_arrive(1 + NS + f, NB);                // slot free
            sl = sl + 1 == SP ? 0 : sl + 1;
        }
        if constexpr (std::is_same<T, long long>::value) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) fxm |= __shfl_down_sync(0xffffffffu, fxm, o);
            if (lane == 0 && fxm) atomicOr(a.fxmax, fxm);
        }
        if (a.mode == kCheck && q == 0) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                d2 += __shfl_down_sync(0xffffffffu, d2, o);
                n2 += __shfl_down_sync(0xffffffffu, n2, o);
                mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
                ms += __shfl_down_sync(0xffffffffu, ms, o);
            }
            if (lane == 0) {
                rpart[g][0] = d2;
                rpart[g][1] = n2;
                rpart[g][2] = mx;
                rpart[g][3] = ms;
            }
        }
    }

    if (a.mode == kCheck) {
        __syncthreads();
        if (threadIdx.x == 0) {
            double t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0;
            for (int k = 0; k < NG; ++k) {
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
int launch_ws_variant(const SweepArgs& a, const void* coefs, int grid, void* stream)
{
    using R = typename AccType<T>::type;
    constexpr WsGeo geo = WsVariants<L>::at(K);
    using WS = Ws<L, T, geo.NG, geo.G, geo.SPG>;
    sweep_ws_kernel<L, T, geo.NG, geo.G, geo.SPG>
        <<<grid, WS::WARPS * 32, WS::smem_bytes(), (cudaStream_t)stream>>>(
            a, *static_cast<const Coefs<R>*>(coefs));
    return (int)cudaGetLastError();
}

template <class L, typename T, int K>
int occupancy_ws_variant(int* blocks, int* tiles_per_block)
{
    constexpr WsGeo geo = WsVariants<L>::at(K);
    using WS = Ws<L, T, geo.NG, geo.G, geo.SPG>;
    auto kern = sweep_ws_kernel<L, T, geo.NG, geo.G, geo.SPG>;
    cudaError_t e = set_sweep_smem(kern, WS::smem_bytes());
    if (e != cudaSuccess) return (int)e;
    *tiles_per_block = 1;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern, WS::WARPS * 32,
                                                              WS::smem_bytes());
}

}  // namespace pkr
