// pkr_api.cpp -- the C ABI (include/pkr.h): plans, the convergence loop and
// the one-shot solve.  Host code only; every step of the solve runs in the
// kernels of pkr_kernels.cu and sweep_*.cu.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "pkr_internal.h"

using namespace pkr;

namespace pkr {
template <class L, typename T> int launch_sweep_t(int, const SweepArgs&, const void*, int, void*);
template <class L, typename T> int occupancy_t(int, int*, int*);
template <class L> int variant_count_t();
template <class L> int pair_variant_t();
template <class L> int launch_sweep_h16(int, const SweepArgs&, const void*, int, void*);
template <class L> int occupancy_h16(int, int*, int*);
template <class L>
int launch_stencil(const double*, double*, const double*, const Coefs<double>&, int64_t, int, int,
                   int, int, int, double*, int, void*, const int*);
}  // namespace pkr

#define PKR_CK(call)                                     \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return PKR_ECUDA;         \
    } while (0)

namespace {

template <class L>
int dispatch_launch(int var, int prec, const SweepArgs& a, const void* c, int grid, void* st)
{
    if (prec == PKR_FP64) return launch_sweep_t<L, double>(var, a, c, grid, st);
    if (prec == PKR_FX64) return launch_sweep_t<L, long long>(var, a, c, grid, st);
    return launch_sweep_t<L, float>(var, a, c, grid, st);
}
template <class L>
int dispatch_occ(int var, int prec, int* b, int* tpb)
{
    if (prec == PKR_FP64) return occupancy_t<L, double>(var, b, tpb);
    if (prec == PKR_FX64) return occupancy_t<L, long long>(var, b, tpb);
    return occupancy_t<L, float>(var, b, tpb);
}

int64_t tiles_of(const int64_t n[3]) { return (n[0] * n[1] * n[2] + 31) / 32; }

// The sweeps that work on 64-site pieces of x rows apply (the
// two-sites-per-lane binary16 sweep and the aligned x-pairs sweep): x rows
// of whole 64-site tiles, every edge at least the lattice's reach.
bool x_pairs(const pkr_problem* p, const LatticeInfo& li)
{
    if (p->n[0] % 64 != 0) return false;
    for (int k = 0; k < li.dim; ++k)
        if (p->n[k] < li.reach) return false;
    return true;
}

// Index of the aligned x-pairs variant of a lattice's plan sweep, or -1.
int pair_variant(int lattice)
{
    switch (lattice) {
    case PKR_D1Q5: return pair_variant_t<D1Q5>();
    case PKR_D1Q9: return pair_variant_t<D1Q9>();
    case PKR_D1Q13: return pair_variant_t<D1Q13>();
    case PKR_D2Q25: return pair_variant_t<D2Q25>();
    case PKR_D2Q81: return pair_variant_t<D2Q81>();
    case PKR_D2Q169: return pair_variant_t<D2Q169>();
    case PKR_D3Q19: return pair_variant_t<D3Q19>();
    case PKR_D3Q111: return pair_variant_t<D3Q111>();
    }
    return -1;
}

int variant_count(int lattice);

// The aligned x-pairs variants are the last ones of a lattice's list.
bool is_pair_variant(int lattice, int variant)
{
    const int p = pair_variant(lattice);
    return p >= 0 && variant >= p && variant < variant_count(lattice);
}

int variant_count(int lattice)
{
    switch (lattice) {
    case PKR_D1Q5: return variant_count_t<D1Q5>();
    case PKR_D1Q9: return variant_count_t<D1Q9>();
    case PKR_D1Q13: return variant_count_t<D1Q13>();
    case PKR_D2Q25: return variant_count_t<D2Q25>();
    case PKR_D2Q81: return variant_count_t<D2Q81>();
    case PKR_D2Q169: return variant_count_t<D2Q169>();
    case PKR_D3Q19: return variant_count_t<D3Q19>();
    case PKR_D3Q111: return variant_count_t<D3Q111>();
    }
    return -1;
}

// Default geometry per lattice, from timing the variants on GB300.  Index
// into the lattice's variant list: for Q > 64 the staged geometries
// {(G,TILES)} = {(1,2),(2,1),(2,2),(3,1),(3,2),(4,1)}, the warp-specialised
// sweep, then the aligned x-pairs sweep and its early-refill form; else
// {(1,2),(1,4)} (D3Q19: the two within 0.2 %).  Large sets whose x rows are
// whole 64-site pairs take the early-refill x-pairs sweep once the grid
// gives every block a few pairs (GLUPS, early refill against (2,2): D3Q111
// at 256^3 3.09 / 2.84 in 64-bit fixed point, 2.61 / 2.50 in binary64, 5.54
// / 5.38 in binary32; D2Q81 at 2048^2 3.85 / 3.69 and 3.60 / 3.35; D2Q169 at
// 2048^2 1.44 / 1.33 in binary64 but 1.35 / 1.48 in fixed point, where two
// blocks of 103 KB per SM leave 28 KB of L1).  Other grids take 2 velocity
// groups x 2 tiles, or, with few tiles per SM, 4 groups x 1 tile (more warps
// share each tile, so each step's chain is shorter).  All geometries give
// the same binary64 result.
int default_variant(int lattice, int precision, int64_t V, int nsm, bool xpairs)
{
    if (variant_count(lattice) <= 2) return 0;
    const int pv = pair_variant(lattice);
    if (xpairs && pv >= 0 && V / 64 >= (int64_t)8 * nsm &&
        !(lattice == PKR_D2Q169 && precision == PKR_FX64))
        return pv + 1;
    return (V + 31) / 32 <= (int64_t)4 * nsm ? 5 : 2;
}

int elem_bytes(int precision)
{
    return (precision == PKR_FP64 || precision == PKR_FX64) ? 8 : precision == PKR_FP32 ? 4 : 2;
}
// binary64 and fixed-point plans keep S in binary64, the others in binary32.
bool wide_source(int precision) { return precision == PKR_FP64 || precision == PKR_FX64; }
int source_bytes(int precision) { return wide_source(precision) ? 8 : 4; }

double now_ms()
{
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

int validate(const pkr_problem* p, LatticeInfo* li, double* tau)
{
    if (!p) return PKR_EINVAL;
    if (p->dim < 1 || p->dim > 3) return PKR_EINVAL;
    if (p->precision != PKR_FP64 && p->precision != PKR_FP32 && p->precision != PKR_FP16 &&
        p->precision != PKR_FX64)
        return PKR_EINVAL;
    // (PKR_MIXED / PKR_MIXED16 are resolved by pkr_solve into a ladder of plans)
    int rc = build_lattice(p->lattice, p->order, li);
    if (rc != PKR_OK) return rc;
    if (li->dim != p->dim) return PKR_EINVAL;
    int64_t V = 1;
    for (int k = 0; k < 3; ++k) {
        if (p->n[k] < 1) return PKR_EINVAL;
        if (k >= p->dim && p->n[k] != 1) return PKR_EINVAL;
        V *= p->n[k];
        if (V > (int64_t)0x7fffffff) return PKR_EINVAL;  // flat site index is 32-bit
    }
    if (p->max_sweeps < 1) return PKR_EINVAL;
    if (p->variant < -1) return PKR_EINVAL;
    if (p->tol_kind != PKR_TOL_MAX_ABS_DPHI && p->tol_kind != PKR_TOL_REL_L2_DPHI) return PKR_EINVAL;
    if (!(p->epsilon >= 0.0) || !std::isfinite(p->epsilon)) return PKR_EINVAL;
    double t = p->tau_lb;
    if (!(t > 0.0)) {
        if (pkr_tau_from_knudsen(p->lattice, p->knudsen, p->n, &t) != PKR_OK) return PKR_EINVAL;
    }
    if (!(t > 0.5) || !std::isfinite(t)) return PKR_EINVAL;
    *tau = t;
    return PKR_OK;
}

}  // namespace

// Upper bound on a persistent sweep grid (blocks); sizes the partials scratch.
constexpr int kMaxGridBlocks = 152 * 32;

struct pkr_plan {
    pkr_problem prob;
    LatticeInfo lat;
    double tau_lb, omega, scale, rho_mean, last_residual, last_res3[3];
    double soff_next;   // source offset for the next launch (mass correction)
    // > 0: a reduced-precision rung of pkr_solve's ladder, which hands over
    // (pkr_plan_run returns PKR_OK) once the residual, below this cap, stops
    // falling from one check to the next (the storage's rounding floor)
    double stall_cap;
    bool h16pairs;      // binary16 storage: the two-sites-per-lane sweep applies
    bool xpairs;        // other storage: the aligned x-pairs sweep applies
    cudaStream_t stream;
    int device, grid, red_blocks, elem, small, variant, nsm;
    int64_t ntiles;
    int64_t V, launches;
    void* pop[2];
    int cur;
    void* S;
    double* Phi;
    double* partials;
    double* scal;   // [0] source mean, [1..4] residual out, [5] mean of an imported Phi
    int* flag;
    double* host;   // pinned: [0] mean, [1..4] residual, [5] import mean, [6] flag (int),
                    // [7] binary16 overflow flag (int)
    bool stencil;          // omega = 1, binary64: the state is Phi alone (scalar stencil)
    double* Ps[2];         // stencil mode: Phi ping-pong
    double* St;            // stencil mode: sum_i chi_i S(x - v_i)
    Coefs<double> cchi;    // stencil mode: chi_c in the weight slot (builds St)
    float* h16sc;          // binary16 storage: scales of the two arrays
    unsigned int* h16max;  // binary16 storage: max |p| of the current step
    int* h16of;            // binary16 storage: overflow flag
    int* fxF;              // fixed-point storage: exponents of the two arrays
    unsigned long long* fxmax;  // fixed-point storage: OR of |stored| over the current step
                                // (its bit length is that of the largest |stored|)
    long long cfx;         // fixed-point storage: round((1 - omega) 2^62)
    // device-side stopping (binary64 runs that check every step): a captured
    // graph of kGraphSteps check steps, each followed by the stopping rule on
    // the device; steps after a stop return at once (SweepArgs::stop)
    RunCtl* ctl;           // device state of the rule
    RunCtl* hctl;          // pinned host copy
    cudaGraphExec_t gexec; // the captured steps (nullptr: none yet)
    cudaStream_t cap;      // stream the graph is captured on
    int gcur, gkind, gj;   // array parity and tol kind the graph was captured for;
                           // index of the step being captured
    double gtol;           // tolerance it was captured for
    const int* stop_arg;   // &ctl->stop while capturing, else nullptr
    bool loaded;
    Coefs<double> c64;
    Coefs<float> c32;
};

namespace {

// Residual of a check step: plain, or with the device-side stopping rule
// while the steps of a run are being captured.
int finalize_step(pkr_plan* P)
{
    if (P->stop_arg)
        return launch_finalize_check(P->partials, P->grid, P->scal + 1, P->ctl, P->gtol, P->gkind,
                                     P->gj, P->stream);
    return launch_finalize_residual(P->partials, P->grid, P->scal + 1, P->stream);
}

int launch_stencil_step(pkr_plan* P, const double* in, double* out, const double* add,
                        const Coefs<double>& c, int check)
{
    const int64_t* n = P->prob.n;
    const int nx = (int)n[0], ny = (int)n[1], nz = (int)n[2];
    int rc = 0;
#define PKR_ST(LL) launch_stencil<LL>(in, out, add, c, P->V, nx, ny, nz, P->small, check, \
                                      P->partials, P->grid, P->stream, P->stop_arg)
    switch (P->prob.lattice) {
    case PKR_D1Q5: rc = PKR_ST(D1Q5); break;
    case PKR_D1Q9: rc = PKR_ST(D1Q9); break;
    case PKR_D1Q13: rc = PKR_ST(D1Q13); break;
    case PKR_D2Q25: rc = PKR_ST(D2Q25); break;
    case PKR_D2Q81: rc = PKR_ST(D2Q81); break;
    case PKR_D2Q169: rc = PKR_ST(D2Q169); break;
    case PKR_D3Q19: rc = PKR_ST(D3Q19); break;
    case PKR_D3Q111: rc = PKR_ST(D3Q111); break;
    default: return PKR_EINVAL;
    }
#undef PKR_ST
    return rc == 0 ? PKR_OK : PKR_ECUDA;
}

int launch_one(pkr_plan* P, int mode, bool zero_in)
{
    if (P->stencil) {
        // Phi^k = stencil(Phi^(k-1)) + St; a zero-in step keeps Phi^0 = 0
        if (!zero_in) {
            const int check = (mode == kCheck) ? 1 : 0;
            int rc = launch_stencil_step(P, P->Ps[P->cur], P->Ps[P->cur ^ 1], P->St, P->c64,
                                         check);
            if (rc != PKR_OK) return rc;
            if (check && finalize_step(P) != 0) return PKR_ECUDA;
            P->cur ^= 1;
        }
        P->Phi = P->Ps[P->cur];
        P->launches += 1;
        return PKR_OK;
    }
    SweepArgs a{};
    a.A = P->pop[P->cur];
    a.B = P->pop[P->cur ^ 1];
    a.S = P->S;
    a.Phi = P->Phi;
    a.partials = P->partials;
    a.V = P->V;
    a.nx = (int32_t)P->prob.n[0];
    a.ny = (int32_t)P->prob.n[1];
    a.nz = (int32_t)P->prob.n[2];
    a.ntiles = (int32_t)P->ntiles;
    a.mode = mode;
    a.zero_in = zero_in ? 1 : 0;
    a.small = P->small;
    a.soff = P->soff_next;
    P->soff_next = 0.0;
    const void* c = wide_source(P->prob.precision) ? (const void*)&P->c64 : (const void*)&P->c32;
    int rc = 0;
    const int pr = P->prob.precision;
    const int vr = P->variant;
    a.cur = P->cur;
    a.fxF = P->fxF;
    a.fxmax = P->fxmax;
    a.cfx = P->cfx;
    a.sc = P->h16sc;
    a.pmax = P->h16max;
    a.oflow = P->h16of;
    a.stop = P->stop_arg;
    if (pr == PKR_FP16) {
        const int vh = (vr == 1 && P->h16pairs) ? 1 : 0;
        switch (P->prob.lattice) {
        case PKR_D1Q5: rc = launch_sweep_h16<D1Q5>(vh, a, c, P->grid, P->stream); break;
        case PKR_D1Q9: rc = launch_sweep_h16<D1Q9>(vh, a, c, P->grid, P->stream); break;
        case PKR_D1Q13: rc = launch_sweep_h16<D1Q13>(vh, a, c, P->grid, P->stream); break;
        case PKR_D2Q25: rc = launch_sweep_h16<D2Q25>(vh, a, c, P->grid, P->stream); break;
        case PKR_D2Q81: rc = launch_sweep_h16<D2Q81>(vh, a, c, P->grid, P->stream); break;
        case PKR_D2Q169: rc = launch_sweep_h16<D2Q169>(vh, a, c, P->grid, P->stream); break;
        case PKR_D3Q19: rc = launch_sweep_h16<D3Q19>(vh, a, c, P->grid, P->stream); break;
        case PKR_D3Q111: rc = launch_sweep_h16<D3Q111>(vh, a, c, P->grid, P->stream); break;
        default: return PKR_EINVAL;
        }
        if (rc != 0) return PKR_ECUDA;
        // the array this step read is the one the next step writes
        if (launch_h16_rescale(P->h16sc, P->h16max, P->cur, P->stream) != 0) return PKR_ECUDA;
        P->cur ^= 1;
        P->launches += 1;
        if (mode == kCheck &&
            launch_finalize_residual(P->partials, P->grid, P->scal + 1, P->stream) != 0)
            return PKR_ECUDA;
        return PKR_OK;
    }
    // the aligned x-pairs sweep reads whole 64-site x pieces: never on other grids
    if (is_pair_variant(P->prob.lattice, vr) && !P->xpairs) return PKR_EINVAL;
    switch (P->prob.lattice) {
    case PKR_D1Q5: rc = dispatch_launch<D1Q5>(vr, pr, a, c, P->grid, P->stream); break;
    case PKR_D1Q9: rc = dispatch_launch<D1Q9>(vr, pr, a, c, P->grid, P->stream); break;
    case PKR_D1Q13: rc = dispatch_launch<D1Q13>(vr, pr, a, c, P->grid, P->stream); break;
    case PKR_D2Q25: rc = dispatch_launch<D2Q25>(vr, pr, a, c, P->grid, P->stream); break;
    case PKR_D2Q81: rc = dispatch_launch<D2Q81>(vr, pr, a, c, P->grid, P->stream); break;
    case PKR_D2Q169: rc = dispatch_launch<D2Q169>(vr, pr, a, c, P->grid, P->stream); break;
    case PKR_D3Q19: rc = dispatch_launch<D3Q19>(vr, pr, a, c, P->grid, P->stream); break;
    case PKR_D3Q111: rc = dispatch_launch<D3Q111>(vr, pr, a, c, P->grid, P->stream); break;
    default: return PKR_EINVAL;
    }
    if (rc != 0) return PKR_ECUDA;
    // fixed point: the array this step read is the one the next step writes
    if (pr == PKR_FX64 && launch_fx_rescale(P->fxF, P->fxmax, P->cur, P->stream) != 0)
        return PKR_ECUDA;
    P->cur ^= 1;
    P->launches += 1;
    if (mode == kCheck) {
        if (finalize_step(P) != 0) return PKR_ECUDA;
    }
    return PKR_OK;
}

int occupancy(int variant, int lattice, int precision, int* b, int* tpb)
{
    if (precision == PKR_FP16) {
        switch (lattice) {
        case PKR_D1Q5: return occupancy_h16<D1Q5>(variant, b, tpb);
        case PKR_D1Q9: return occupancy_h16<D1Q9>(variant, b, tpb);
        case PKR_D1Q13: return occupancy_h16<D1Q13>(variant, b, tpb);
        case PKR_D2Q25: return occupancy_h16<D2Q25>(variant, b, tpb);
        case PKR_D2Q81: return occupancy_h16<D2Q81>(variant, b, tpb);
        case PKR_D2Q169: return occupancy_h16<D2Q169>(variant, b, tpb);
        case PKR_D3Q19: return occupancy_h16<D3Q19>(variant, b, tpb);
        case PKR_D3Q111: return occupancy_h16<D3Q111>(variant, b, tpb);
        }
        return -1;
    }
    switch (lattice) {
    case PKR_D1Q5: return dispatch_occ<D1Q5>(variant, precision, b, tpb);
    case PKR_D1Q9: return dispatch_occ<D1Q9>(variant, precision, b, tpb);
    case PKR_D1Q13: return dispatch_occ<D1Q13>(variant, precision, b, tpb);
    case PKR_D2Q25: return dispatch_occ<D2Q25>(variant, precision, b, tpb);
    case PKR_D2Q81: return dispatch_occ<D2Q81>(variant, precision, b, tpb);
    case PKR_D2Q169: return dispatch_occ<D2Q169>(variant, precision, b, tpb);
    case PKR_D3Q19: return dispatch_occ<D3Q19>(variant, precision, b, tpb);
    case PKR_D3Q111: return dispatch_occ<D3Q111>(variant, precision, b, tpb);
    }
    return -1;
}

// Select a variant: occupancy, persistent grid size (blocks resident on all
// SMs, capped by the work).  The partials scratch holds 3 doubles per block
// of the largest grid any variant may use (allocated at plan creation).
int set_variant(pkr_plan* P, int variant)
{
    // the aligned x-pairs geometry only where x rows split into 64-site
    // pairs; elsewhere the staged 2 groups x 2 tiles (the same results)
    if (P->prob.precision != PKR_FP16 && is_pair_variant(P->prob.lattice, variant) &&
        !P->xpairs)
        variant = 2;
    int bps = 0, tpb = 1;
    if (occupancy(variant, P->prob.lattice, P->prob.precision, &bps, &tpb) != 0 || bps < 1)
        return PKR_ECUDA;
    const int64_t nbt = (P->ntiles + tpb - 1) / tpb;
    int64_t grid = (int64_t)P->nsm * bps;
    if (grid > nbt) grid = nbt;
    if (grid > kMaxGridBlocks) grid = kMaxGridBlocks;
    P->variant = variant;
    P->grid = (int)grid;
    if (P->gexec) {   // captured with the previous geometry
        cudaGraphExecDestroy(P->gexec);
        P->gexec = nullptr;
    }
    return PKR_OK;
}

// Checks without a new smallest residual after which a reduced-precision rung
// of pkr_solve's ladder is taken to sit at its rounding floor.
constexpr int kStallChecks = 4;

// Steps per captured graph of device-stopped check steps (even, so that the
// arrays are back at the same parity after a full replay).
constexpr int kGraphSteps = 64;

// Capture kGraphSteps check steps, each followed by the stopping rule on the
// device, as one graph for this plan, array parity, tol and tol kind.  The
// host view that launch_one advances (parity, step count, Phi) is restored
// afterwards: capturing runs nothing.  On failure the caller steps on the host.
int capture_steps(pkr_plan* P, double tol, int tol_kind)
{
    if (!P->ctl) {
        if (cudaMalloc((void**)&P->ctl, sizeof(RunCtl)) != cudaSuccess ||
            cudaMallocHost((void**)&P->hctl, sizeof(RunCtl)) != cudaSuccess) {
            cudaGetLastError();
            return PKR_ENOMEM;
        }
    }
    if (!P->cap && cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        P->cap = nullptr;
        return PKR_ECUDA;
    }
    if (P->gexec) {
        cudaGraphExecDestroy(P->gexec);
        P->gexec = nullptr;
    }
    const int cur = P->cur;
    const int64_t launches = P->launches;
    double* const Phi = P->Phi;
    const cudaStream_t stream = P->stream;
    P->stream = P->cap;
    P->stop_arg = &P->ctl->stop;
    P->gtol = tol;
    P->gkind = tol_kind;
    cudaGraph_t g = nullptr;
    int rc = cudaStreamBeginCapture(P->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess
                 ? PKR_OK
                 : PKR_ECUDA;
    if (rc == PKR_OK) {
        for (int j = 0; j < kGraphSteps && rc == PKR_OK; ++j) {
            P->gj = j;
            rc = launch_one(P, kCheck, false);
        }
        if (cudaStreamEndCapture(P->cap, &g) != cudaSuccess) rc = PKR_ECUDA;
    }
    if (rc == PKR_OK && cudaGraphInstantiate(&P->gexec, g, 0) != cudaSuccess) {
        P->gexec = nullptr;
        rc = PKR_ECUDA;
    }
    if (g) cudaGraphDestroy(g);
    P->stream = stream;
    P->stop_arg = nullptr;
    P->cur = cur;
    P->launches = launches;
    P->Phi = Phi;
    if (rc != PKR_OK) {
        cudaGetLastError();
        return rc;
    }
    P->gcur = cur;
    return PKR_OK;
}

size_t plan_bytes(const pkr_problem* p, const LatticeInfo& li, int64_t V, int grid_max)
{
    const size_t e = (size_t)elem_bytes(p->precision);
    size_t b = 2 * ((size_t)li.Q * (size_t)V * e + 16);   // ping-pong populations
    b += (size_t)V * source_bytes(p->precision);           // S
    b += (size_t)V * 8;                             // Phi
    b += (size_t)(4 * grid_max + 4096) * 8 + 64;    // partials + scalars + flag
    return b;
}

}  // namespace

extern "C" {

const char* pkr_status_str(int s)
{
    switch (s) {
    case PKR_OK: return "ok";
    case PKR_EINVAL: return "invalid argument";
    case PKR_ENOMEM: return "out of device memory";
    case PKR_EUNSTABLE: return "relaxation time in the unstable range of this lattice";
    case PKR_ENOCONV: return "not converged within max_sweeps";
    case PKR_EDIVERGED: return "iteration diverged";
    case PKR_ECUDA: return "CUDA runtime error";
    case PKR_EBUSY: return "not finished";
    default: return "unknown status";
    }
}

const char* pkr_version(void) { return "pkr 0.1 sm_103a"; }

int pkr_lattice_info(int lattice, int order, int32_t* Q, int32_t* dim, int32_t* vel, double* w,
                     double* phi, double* chi, double* cs2)
{
    LatticeInfo li;
    int rc = build_lattice(lattice, order, &li);
    if (rc != PKR_OK) return rc;
    if (Q) *Q = li.Q;
    if (dim) *dim = li.dim;
    for (int i = 0; i < li.Q; ++i) {
        if (vel) {
            vel[3 * i + 0] = li.vel[3 * i + 0];
            vel[3 * i + 1] = li.vel[3 * i + 1];
            vel[3 * i + 2] = li.vel[3 * i + 2];
        }
        if (w) w[i] = li.w[i];
        if (phi) phi[i] = li.phi[i];
        if (chi) chi[i] = li.chi[i];
    }
    if (cs2) *cs2 = li.cs2;
    return PKR_OK;
}

int pkr_tau_from_knudsen(int lattice, double knudsen, const int64_t n[3], double* tau_lb)
{
    if (!n || !tau_lb || !(knudsen > 0.0) || !std::isfinite(knudsen)) return PKR_EINVAL;
    int32_t order = 1;
    LatticeInfo li;
    int rc = build_lattice(lattice, order, &li);
    if (rc != PKR_OK) return rc;
    int64_t L = 0;
    for (int k = 0; k < 3; ++k)
        if (n[k] > 1 && (L == 0 || n[k] < L)) L = n[k];
    if (L == 0) L = 1;
    *tau_lb = 0.5 + knudsen * (double)L / std::sqrt(li.cs2);
    return PKR_OK;
}

int pkr_plan_bytes(const pkr_problem* p, size_t* bytes)
{
    LatticeInfo li;
    double tau;
    int rc = validate(p, &li, &tau);
    if (rc != PKR_OK) return rc;
    if (!bytes) return PKR_EINVAL;
    const int64_t V = p->n[0] * p->n[1] * p->n[2];
    *bytes = plan_bytes(p, li, V, kMaxGridBlocks);
    return PKR_OK;
}

namespace {

// pkr_plan_create, with the second population array optional (spare =
// false: only pop[0] is allocated, for a ladder rung that receives a
// converted state in pop[0] and gets pop[1] once the previous rung is gone).
int plan_create(const pkr_problem* p, void* stream, pkr_plan** out, bool spare)
{
    if (!out) return PKR_EINVAL;
    *out = nullptr;
    LatticeInfo li;
    double tau;
    int rc = validate(p, &li, &tau);
    if (rc != PKR_OK) return rc;
    const double omega = 1.0 / tau;
    if (unstable(li, omega)) return PKR_EUNSTABLE;

    pkr_plan* P = new (std::nothrow) pkr_plan();
    if (!P) return PKR_ENOMEM;
    P->prob = *p;
    P->stencil = (p->precision == PKR_FP64 && omega == 1.0 && p->variant == -1);
    if (P->prob.epsilon == 0.0) P->prob.epsilon = 1.0;
    if (P->prob.check_every <= 0) P->prob.check_every = 32;
    P->lat = li;
    P->tau_lb = tau;
    P->omega = omega;
    P->scale = li.cs2 * (tau - 0.5) / P->prob.epsilon;
    P->stream = (cudaStream_t)stream;
    P->V = p->n[0] * p->n[1] * p->n[2];
    P->elem = elem_bytes(p->precision);
    P->small = 0;
    for (int k = 0; k < li.dim; ++k)
        if (p->n[k] < li.reach) P->small = 1;
    P->last_residual = -1.0;
    // collision coefficients per symmetry class
    P->c64.om1 = 1.0 - omega;
    P->c32.om1 = (float)(1.0 - omega);
    P->cchi.om1 = 0.0;
    P->cfx = std::llround(std::ldexp(1.0 - omega, 62));
    for (int c = 0; c < li.ncls; ++c) {
        P->c64.wphi[c] = omega * li.cls_phi[c];
        P->c64.chi[c] = li.cls_chi[c];
        P->c32.wphi[c] = (float)(omega * li.cls_phi[c]);
        P->c32.chi[c] = (float)li.cls_chi[c];
        P->cchi.wphi[c] = li.cls_chi[c];
    }

    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        delete P;
        return PKR_ECUDA;
    }
    P->device = dev;
    P->nsm = nsm;
    P->ntiles = tiles_of(p->n);
    const int nvar = variant_count(p->lattice);
    // binary16 storage: two sites per lane where every x row splits into
    // 64-site tiles (and no edge is below the reach), unless variant 0 (one
    // site per lane) is asked for; else one
    P->h16pairs = p->precision == PKR_FP16 && x_pairs(p, li);
    P->xpairs = p->precision != PKR_FP16 && x_pairs(p, li);
    int var = (p->variant >= 0) ? p->variant
                                : default_variant(p->lattice, p->precision, P->V, nsm, P->xpairs);
    if (p->precision == PKR_FP16) var = (P->h16pairs && p->variant != 0) ? 1 : 0;
    if (var >= nvar) {
        delete P;
        return PKR_EINVAL;
    }
    if (P->stencil) {
        const int tb = stencil_block(P->V, nsm);
        int64_t g = (P->V + tb - 1) / tb;
        if (g > (int64_t)nsm * 8) g = (int64_t)nsm * 8;
        P->grid = (int)g;
        P->variant = 0;
    } else if (set_variant(P, var) != PKR_OK) {
        delete P;
        return PKR_ECUDA;
    }
    P->red_blocks = nsm * 4;

    // (+16 bytes: binary16 steps read the aligned 4-byte word around a value)
    const size_t popb = (size_t)li.Q * (size_t)P->V * (size_t)P->elem + 16;
    size_t freeb = 0, totb = 0;
    if (cudaMemGetInfo(&freeb, &totb) != cudaSuccess) {
        delete P;
        return PKR_ECUDA;
    }
    const size_t need = P->stencil ? (size_t)P->V * 8 * 5 + (size_t)4 * kMaxGridBlocks * 8
                                   : plan_bytes(p, li, P->V, kMaxGridBlocks) - (spare ? 0 : popb);
    if (need > freeb) {
        delete P;
        return PKR_ENOMEM;
    }
    const size_t nscratch = (size_t)4 * kMaxGridBlocks;
    bool ok = (P->stencil
                   ? (cudaMalloc((void**)&P->Ps[0], (size_t)P->V * 8) == cudaSuccess &&
                      cudaMalloc((void**)&P->Ps[1], (size_t)P->V * 8) == cudaSuccess &&
                      cudaMalloc((void**)&P->St, (size_t)P->V * 8) == cudaSuccess)
                   : (cudaMalloc(&P->pop[0], popb) == cudaSuccess &&
                      (!spare || cudaMalloc(&P->pop[1], popb) == cudaSuccess))) &&
              cudaMalloc(&P->S, (size_t)P->V * source_bytes(p->precision)) == cudaSuccess &&
              cudaMalloc((void**)&P->h16sc, 2 * sizeof(float)) == cudaSuccess &&
              cudaMalloc((void**)&P->h16max, sizeof(unsigned int)) == cudaSuccess &&
              cudaMalloc((void**)&P->h16of, sizeof(int)) == cudaSuccess &&
              cudaMalloc((void**)&P->fxF, 2 * sizeof(int)) == cudaSuccess &&
              cudaMalloc((void**)&P->fxmax, sizeof(unsigned long long)) == cudaSuccess &&
              (P->stencil || cudaMalloc((void**)&P->Phi, (size_t)P->V * 8) == cudaSuccess) &&
              cudaMalloc((void**)&P->partials, nscratch * 8) == cudaSuccess &&
              cudaMalloc((void**)&P->scal, 8 * 8) == cudaSuccess &&
              cudaMalloc((void**)&P->flag, sizeof(int)) == cudaSuccess &&
              cudaMallocHost((void**)&P->host, 8 * 8) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        pkr_plan_destroy(P);
        return PKR_ENOMEM;
    }
    if (P->stencil) P->Phi = P->Ps[0];
    *out = P;
    return PKR_OK;
}

size_t pop_bytes(const pkr_plan* P)
{
    return (size_t)P->lat.Q * (size_t)P->V * (size_t)P->elem + 16;
}

// Free the population array a plan does not read next (its state stays in
// pop[cur], Phi and S; it cannot step again until plan_alloc_spare).
void plan_free_spare(pkr_plan* P)
{
    if (P->stencil || !P->pop[P->cur ^ 1]) return;
    cudaStreamSynchronize(P->stream);
    cudaFree(P->pop[P->cur ^ 1]);
    P->pop[P->cur ^ 1] = nullptr;
}

int plan_alloc_spare(pkr_plan* P)
{
    if (P->stencil || P->pop[P->cur ^ 1]) return PKR_OK;
    if (cudaMalloc(&P->pop[P->cur ^ 1], pop_bytes(P)) != cudaSuccess) {
        cudaGetLastError();
        return PKR_ENOMEM;
    }
    return PKR_OK;
}

}  // namespace

int pkr_plan_create(const pkr_problem* p, void* stream, pkr_plan** out)
{
    return plan_create(p, stream, out, true);
}

int pkr_plan_destroy(pkr_plan* P)
{
    if (!P) return PKR_OK;
    if (P->stream || P->pop[0] || P->Ps[0]) cudaStreamSynchronize(P->stream);
    cudaFree(P->pop[0]);
    cudaFree(P->pop[1]);
    cudaFree(P->Ps[0]);
    cudaFree(P->Ps[1]);
    cudaFree(P->St);
    cudaFree(P->S);
    if (!P->stencil) cudaFree(P->Phi);
    cudaFree(P->partials);
    cudaFree(P->scal);
    cudaFree(P->flag);
    cudaFree(P->h16sc);
    cudaFree(P->h16max);
    cudaFree(P->h16of);
    cudaFree(P->fxF);
    cudaFree(P->fxmax);
    if (P->host) cudaFreeHost(P->host);
    if (P->gexec) cudaGraphExecDestroy(P->gexec);
    cudaFree(P->ctl);
    if (P->hctl) cudaFreeHost(P->hctl);
    if (P->cap) cudaStreamDestroy(P->cap);
    delete P;
    return PKR_OK;
}

namespace {

// pkr_plan_load_source; first_step = false leaves out the first step (from
// zero populations), for a plan that pkr_plan_import fills next: it touches
// pop[0] only.
int load_source(pkr_plan* P, const double* rho, int rho_on_host, bool first_step)
{
    if (!P || !rho) return PKR_EINVAL;
    const double* rd = rho;
    if (rho_on_host) {
        // stage rho through the Phi buffer (V doubles), which is reset below
        PKR_CK(cudaMemcpyAsync(P->Phi, rho, (size_t)P->V * 8, cudaMemcpyHostToDevice, P->stream));
        rd = P->Phi;
    }
    PKR_CK(cudaMemsetAsync(P->flag, 0, sizeof(int), P->stream));
    if (launch_rho_partials(rd, P->V, P->partials, P->red_blocks, P->flag, P->stream) != 0 ||
        launch_finalize_mean(P->partials, P->red_blocks, P->V, P->scal, P->stream) != 0 ||
        launch_make_source(rd, P->scal, P->scale, P->V, P->S,
                           wide_source(P->prob.precision) ? PKR_FP64 : PKR_FP32, P->stream) != 0)
        return PKR_ECUDA;
    if (P->prob.precision == PKR_FX64) {
        PKR_CK(cudaMemsetAsync(P->fxmax, 0, sizeof(unsigned long long), P->stream));
        if (launch_absmax_f64(static_cast<const double*>(P->S), P->V, P->fxmax, P->stream) != 0)
            return PKR_ECUDA;
    }
    if (P->prob.precision == PKR_FP16) {
        PKR_CK(cudaMemsetAsync(P->h16max, 0, sizeof(unsigned int), P->stream));
        PKR_CK(cudaMemsetAsync(P->h16of, 0, sizeof(int), P->stream));
        if (launch_absmax_f32(static_cast<const float*>(P->S), P->V, P->h16max, P->stream) != 0)
            return PKR_ECUDA;
    }
    PKR_CK(cudaMemcpyAsync(P->host, P->scal, 8, cudaMemcpyDeviceToHost, P->stream));
    PKR_CK(cudaMemcpyAsync(P->host + 6, P->flag, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
    PKR_CK(cudaStreamSynchronize(P->stream));
    int bad = 0;
    std::memcpy(&bad, P->host + 6, sizeof(int));
    if (bad) {
        P->loaded = false;
        return PKR_EINVAL;
    }
    P->rho_mean = P->host[0];
    if (P->prob.precision == PKR_FX64) {
        // exponent of the first write (the step from zero stores chi_i S):
        // its largest value lands near 2^52, leaving room to grow before the
        // device-side rescaling shifts the scale
        unsigned long long mb = 0;
        PKR_CK(cudaMemcpy(&mb, P->fxmax, sizeof(mb), cudaMemcpyDeviceToHost));
        double ms = 0.0;
        std::memcpy(&ms, &mb, sizeof(ms));
        double mchi = 0.0;
        for (int i = 0; i < P->lat.Q; ++i) mchi = std::fmax(mchi, std::fabs(P->lat.chi[i]));
        const double m = ms * mchi;
        int F = 0;
        if (m > 0.0 && std::isfinite(m)) F = 52 - (std::ilogb(m) + 1);
        const int F2[2] = {F, F};
        PKR_CK(cudaMemcpyAsync(P->fxF, F2, sizeof(F2), cudaMemcpyHostToDevice, P->stream));
        PKR_CK(cudaMemsetAsync(P->fxmax, 0, sizeof(unsigned long long), P->stream));
    }
    if (P->prob.precision == PKR_FP16) {
        // scale of the first write: the step from zero stores chi_i S
        unsigned int mb = 0;
        PKR_CK(cudaMemcpy(&mb, P->h16max, sizeof(mb), cudaMemcpyDeviceToHost));
        float ms = 0.f;
        std::memcpy(&ms, &mb, sizeof(ms));
        double mchi = 0.0;
        for (int i = 0; i < P->lat.Q; ++i) mchi = std::fmax(mchi, std::fabs(P->lat.chi[i]));
        const double m = (double)ms * mchi;
        float sc = 1.0f;
        if (m > 0.0 && std::isfinite(m)) sc = std::ldexp(1.0f, std::ilogb(4.0 * m / 65504.0) + 1);
        const float sc2[2] = {sc, sc};
        PKR_CK(cudaMemcpyAsync(P->h16sc, sc2, sizeof(sc2), cudaMemcpyHostToDevice, P->stream));
        PKR_CK(cudaMemsetAsync(P->h16max, 0, sizeof(unsigned int), P->stream));
    }
    if (P->stencil) {
        // St = sum_i chi_i S(x - v_i); Phi^0 = 0 in both buffers
        int rc0 = launch_stencil_step(P, static_cast<const double*>(P->S), P->St, nullptr,
                                      P->cchi, 0);
        if (rc0 != PKR_OK) return rc0;
        PKR_CK(cudaMemsetAsync(P->Ps[0], 0, (size_t)P->V * 8, P->stream));
        PKR_CK(cudaMemsetAsync(P->Ps[1], 0, (size_t)P->V * 8, P->stream));
        P->Phi = P->Ps[0];
    }
    // Phi^0 = 0; the first step starts from zero populations
    PKR_CK(cudaMemsetAsync(P->Phi, 0, (size_t)P->V * 8, P->stream));
    P->launches = 0;
    P->cur = 0;
    P->last_residual = -1.0;
    P->soff_next = 0.0;
    if (first_step) {
        int rc = launch_one(P, kWritePhi, true);
        if (rc != PKR_OK) return rc;
    } else {
        PKR_CK(cudaStreamSynchronize(P->stream));
    }
    P->loaded = true;
    return PKR_OK;
}

}  // namespace

int pkr_plan_load_source(pkr_plan* P, const double* rho, int rho_on_host)
{
    return load_source(P, rho, rho_on_host, true);
}

int pkr_variant_count(int lattice) { return variant_count(lattice); }

int pkr_plan_autotune(pkr_plan* P, int steps_per_variant, int32_t* best_variant,
                      double* best_ms_per_step)
{
    if (!P || !P->loaded || steps_per_variant < 1) return PKR_EINVAL;
    const int n = P->stencil ? 1
                  : P->prob.precision == PKR_FP16 ? (P->h16pairs ? 2 : 1)
                                                   : variant_count(P->prob.lattice);
    cudaEvent_t e0, e1;
    PKR_CK(cudaEventCreate(&e0));
    PKR_CK(cudaEventCreate(&e1));
    int best = P->variant;
    float best_ms = 1e30f;
    int rc = PKR_OK;
    for (int v = 0; v < n && rc == PKR_OK; ++v) {
        if (P->prob.precision != PKR_FP16 && is_pair_variant(P->prob.lattice, v) && !P->xpairs)
            continue;   // the aligned x pairs need rows of whole 64-site pairs
        if (!P->stencil && (rc = set_variant(P, v)) != PKR_OK) break;
        if ((rc = launch_one(P, kPlain, false)) != PKR_OK) break;   // warm-up
        cudaEventRecord(e0, P->stream);
        for (int k = 0; k < steps_per_variant && rc == PKR_OK; ++k)
            rc = launch_one(P, kPlain, false);
        cudaEventRecord(e1, P->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = PKR_ECUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= (float)steps_per_variant;
        if (ms < best_ms) {
            best_ms = ms;
            best = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != PKR_OK) return rc;
    if (!P->stencil && (rc = set_variant(P, best)) != PKR_OK) return rc;
    // keep the invariant that the latest Phi is written
    if ((rc = launch_one(P, kWritePhi, false)) != PKR_OK) return rc;
    PKR_CK(cudaStreamSynchronize(P->stream));
    if (best_variant) *best_variant = P->stencil ? best : P->variant;
    if (best_ms_per_step) *best_ms_per_step = best_ms;
    return PKR_OK;
}

int pkr_plan_import(pkr_plan* P, const pkr_plan* F)
{
    if (!P || !F || !F->loaded || !P->loaded) return PKR_EINVAL;
    if (F->stencil) return PKR_EINVAL;   // a stencil plan holds no populations to hand on
    if (P->stencil && F->omega != 1.0) return PKR_EINVAL;
    if (P->prob.lattice != F->prob.lattice || P->prob.order != F->prob.order ||
        P->prob.n[0] != F->prob.n[0] || P->prob.n[1] != F->prob.n[1] ||
        P->prob.n[2] != F->prob.n[2])
        return PKR_EINVAL;
    PKR_CK(cudaStreamSynchronize(F->stream));
    // Project the imported state onto the zero-mass gauge: with c the mean of
    // its latest Phi, subtract c phi_i from every population (the k = 0
    // equilibrium mode, sum_i phi_i = 1) and c from Phi.  This removes the
    // mass drift a binary32 run accumulates before it is continued in binary64.
    PKR_CK(cudaMemcpyAsync(P->Phi, F->Phi, (size_t)P->V * 8, cudaMemcpyDeviceToDevice,
                           P->stream));
    if (launch_rho_partials(P->Phi, P->V, P->partials, P->red_blocks, P->flag, P->stream) != 0 ||
        launch_finalize_mean(P->partials, P->red_blocks, P->V, P->scal + 5, P->stream) != 0)
        return PKR_ECUDA;
    PKR_CK(cudaMemcpyAsync(P->host + 5, P->scal + 5, 8, cudaMemcpyDeviceToHost, P->stream));
    PKR_CK(cudaStreamSynchronize(P->stream));
    const double c = std::isfinite(P->host[5]) ? P->host[5] : 0.0;
    std::vector<double> shift(P->lat.Q);
    for (int i = 0; i < P->lat.Q; ++i) shift[i] = c * P->lat.phi[i];
    PKR_CK(cudaMemcpyAsync(P->partials, shift.data(), shift.size() * 8, cudaMemcpyHostToDevice,
                           P->stream));
    if (P->stencil) {
        // omega = 1 on both sides: the state is Phi (populations are phi Phi + chi S)
        if (F->omega != 1.0) return PKR_EINVAL;
        if (launch_make_source(P->Phi, P->scal + 5, 1.0, P->V, P->Ps[P->cur], PKR_FP64,
                               P->stream) != 0)
            return PKR_ECUDA;
        PKR_CK(cudaStreamSynchronize(P->stream));
        P->Phi = P->Ps[P->cur];
        P->launches = F->launches;
        P->last_residual = F->last_residual;
        P->soff_next = 0.0;
        return PKR_OK;
    }
    if (P->prob.precision == PKR_FP16 || F->prob.precision == PKR_FX64)
        return PKR_EINVAL;   // imports into binary16, or from fixed point: no
    const float* in_scale = F->prob.precision == PKR_FP16 ? F->h16sc + F->cur : nullptr;
    if (P->prob.precision == PKR_FX64) {
        // into fixed point: the exponent from the largest converted magnitude
        // (both arrays start at it; the device rescale lowers it as needed)
        unsigned long long mb = 0;
        PKR_CK(cudaMemsetAsync(P->fxmax, 0, sizeof(unsigned long long), P->stream));
        if (launch_absmax_shift(F->pop[F->cur], F->prob.precision, P->lat.Q, P->V, P->partials,
                                in_scale, P->fxmax, P->stream) != 0)
            return PKR_ECUDA;
        PKR_CK(cudaMemcpyAsync(&mb, P->fxmax, sizeof(mb), cudaMemcpyDeviceToHost, P->stream));
        PKR_CK(cudaStreamSynchronize(P->stream));
        double m = 0.0;
        std::memcpy(&m, &mb, sizeof(m));
        const int Fx = fx_exponent(m);
        const int F2[2] = {Fx, Fx};
        PKR_CK(cudaMemcpyAsync(P->fxF, F2, sizeof(F2), cudaMemcpyHostToDevice, P->stream));
        PKR_CK(cudaMemsetAsync(P->fxmax, 0, sizeof(unsigned long long), P->stream));
        if (launch_convert_fx(F->pop[F->cur], F->prob.precision,
                              static_cast<long long*>(P->pop[P->cur]), P->lat.Q, P->V,
                              P->partials, in_scale, Fx, P->stream) != 0 ||
            launch_make_source(P->Phi, P->scal + 5, 1.0, P->V, P->Phi, PKR_FP64, P->stream) != 0)
            return PKR_ECUDA;
        PKR_CK(cudaStreamSynchronize(P->stream));
        P->launches = F->launches;
        P->last_residual = F->last_residual;
        P->soff_next = 0.0;
        return PKR_OK;
    }
    if (launch_convert_shift(F->pop[F->cur], F->prob.precision, P->pop[P->cur], P->prob.precision,
                             P->lat.Q, P->V, P->partials, P->stream, F->h16sc + F->cur) != 0 ||
        launch_make_source(P->Phi, P->scal + 5, 1.0, P->V, P->Phi, PKR_FP64, P->stream) != 0)
        return PKR_ECUDA;
    PKR_CK(cudaStreamSynchronize(P->stream));
    P->launches = F->launches;
    P->last_residual = F->last_residual;
    P->soff_next = 0.0;
    return PKR_OK;
}

int pkr_plan_sweeps(pkr_plan* P, int64_t count)
{
    if (!P || !P->loaded || count < 0) return PKR_EINVAL;
    for (int64_t j = 0; j < count; ++j) {
        int rc = launch_one(P, j == count - 1 ? kWritePhi : kPlain, false);
        if (rc != PKR_OK) return rc;
    }
    return PKR_OK;
}

int pkr_plan_run(pkr_plan* P, int64_t steps, double tol, int tol_kind, int check_every,
                 pkr_stats* st)
{
    if (!P || !P->loaded || steps < 0) return PKR_EINVAL;
    if (tol_kind != PKR_TOL_MAX_ABS_DPHI && tol_kind != PKR_TOL_REL_L2_DPHI) return PKR_EINVAL;
    const int64_t K = check_every > 0 ? check_every : P->prob.check_every;
    const double t0 = now_ms();
    int status = PKR_OK;
    double min_res = INFINITY;
    int nchecks = 0, since_min = 0;   // checks since the last new minimum
    int64_t done = 0;
    bool stopped = false;
    // Binary64 runs that check every step (the per-step stopping rules of
    // small problems): steps go in captured graphs of kGraphSteps, the rule is
    // applied on the device after each check, and the host reads the outcome
    // once per graph instead of once per step.  Same steps, same stopping step.
    if (K == 1 && tol > 0.0 && P->prob.precision == PKR_FP64 && steps >= kGraphSteps) {
        bool ok = true;
        if (!P->gexec || P->gcur != P->cur || P->gtol != tol || P->gkind != tol_kind)
            ok = capture_steps(P, tol, tol_kind) == PKR_OK;
        if (ok) {
            *P->hctl = RunCtl{0, PKR_OK, -1, 0, INFINITY, P->last_residual};
            PKR_CK(cudaMemcpyAsync(P->ctl, P->hctl, sizeof(RunCtl), cudaMemcpyHostToDevice,
                                   P->stream));
            while (steps - done >= kGraphSteps) {
                PKR_CK(cudaGraphLaunch(P->gexec, P->stream));
                PKR_CK(cudaMemcpyAsync(P->hctl, P->ctl, sizeof(RunCtl), cudaMemcpyDeviceToHost,
                                       P->stream));
                PKR_CK(cudaStreamSynchronize(P->stream));
                const RunCtl c = *P->hctl;
                const int64_t ran = c.stop ? (int64_t)c.done_at + 1 : (int64_t)kGraphSteps;
                P->launches += ran;
                done += ran;
                if (ran & 1) P->cur ^= 1;
                if (P->stencil) P->Phi = P->Ps[P->cur];
                P->last_residual = c.last_res;
                nchecks = c.nchecks;
                min_res = c.min_res;
                if (c.stop) {
                    status = c.status;
                    stopped = true;
                    break;
                }
            }
        }
    }
    for (int64_t j = stopped ? steps : done; j < steps; ++j) {
        const int64_t k = P->launches;  // this launch computes Phi^k
        int mode = kPlain;
        if (k % K == 0) mode = kCheck;
        else if ((k + 1) % K == 0 || j == steps - 1) mode = kWritePhi;
        int rc = launch_one(P, mode, false);
        if (rc != PKR_OK) return rc;
        ++done;
        if (mode == kCheck) {
            PKR_CK(cudaMemcpyAsync(P->host + 1, P->scal + 1, 4 * 8, cudaMemcpyDeviceToHost,
                                   P->stream));
            PKR_CK(cudaStreamSynchronize(P->stream));
            const double r = P->host[1 + (tol_kind == PKR_TOL_MAX_ABS_DPHI ? 0 : 1)];
            P->last_residual = r;
            // binary32 rounding does not conserve the mass sum_x Phi, and the
            // k = 0 mode never decays, so the mass random-walks away from its
            // exact value 0 (the source has zero mean).  Remove it in the next
            // step through the source: sum_i chi_i = 1, so adding -M/V to S at
            // every site removes exactly M.
            if ((P->prob.precision == PKR_FP32 || P->prob.precision == PKR_FP16) &&
                std::isfinite(P->host[4]))
                P->soff_next = -P->host[4] / (double)P->V;
            if (P->prob.precision == PKR_FP16) {
                int of = 0;
                PKR_CK(cudaMemcpy(&of, P->h16of, sizeof(int), cudaMemcpyDeviceToHost));
                if (of) {
                    status = PKR_EDIVERGED;
                    break;
                }
            }
            ++nchecks;
            if (!std::isfinite(P->host[1]) || !std::isfinite(P->host[3]) ||
                (nchecks > 2 && r > 1e6 * min_res && r > 1e-300)) {
                status = PKR_EDIVERGED;
                break;
            }
            since_min = r < min_res ? 0 : since_min + 1;
            if (r < min_res) min_res = r;
            if (tol > 0.0 && r < tol) break;
            // a reduced-precision rung at its rounding floor: no new minimum
            // for kStallChecks checks in a row (the residual of a converging
            // run may rise for a check or two on its way down)
            if (P->stall_cap > 0.0 && since_min >= kStallChecks && r < P->stall_cap) break;
        }
    }
    PKR_CK(cudaStreamSynchronize(P->stream));
    const double ms = now_ms() - t0;
    if (st) {
        st->sweeps = P->launches - 1;
        st->launches = P->launches;
        st->residual = P->last_residual;
        st->rho_mean_removed = P->rho_mean;
        st->tau_lb = P->tau_lb;
        st->cs2 = P->lat.cs2;
        st->wall_ms = ms;
        const double upd = (double)done * (double)P->V;
        st->glups = ms > 0 ? upd / (ms * 1e6) : 0.0;
        const double bytes_site = 2.0 * P->lat.Q * P->elem + source_bytes(P->prob.precision);
        st->hbm_gbs = ms > 0 ? upd * bytes_site / (ms * 1e6) : 0.0;
        st->variant = P->stencil ? -1 : P->variant;
    }
    return status;
}

int pkr_plan_phi(pkr_plan* P, double* phi, int phi_on_host)
{
    if (!P || !phi || !P->loaded) return PKR_EINVAL;
    PKR_CK(cudaMemcpyAsync(phi, P->Phi, (size_t)P->V * 8,
                           phi_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                           P->stream));
    PKR_CK(cudaStreamSynchronize(P->stream));
    return PKR_OK;
}

int64_t pkr_plan_steps(const pkr_plan* P) { return P && P->launches > 0 ? P->launches - 1 : 0; }

void* pkr_plan_populations(pkr_plan* P) { return (P && !P->stencil) ? P->pop[P->cur] : nullptr; }

int pkr_solve(const pkr_problem* p, const double* rho, double* phi, int host_buffers,
              pkr_stats* st, void* stream)
{
    if (!p || !rho || !phi) return PKR_EINVAL;
    const double t0 = now_ms();
    // Precision ladder: each stage runs to its switch tolerance (or tol, if
    // looser), then the next, wider stage continues from the converted state.
    // A reduced-precision rung also hands over when its residual stops
    // falling below a cap (binary16: 0.1, binary32: 1e-3), as batch contexts
    // do: its rounding floor may lie above the switch tolerance.  (Tests can
    // lower both switch tolerances with the environment variable
    // PKR_TEST_SWITCH_TOL, so that the rungs end at their floor.)
    double sw16 = PKR_MIXED16_SWITCH_TOL, sw32 = PKR_MIXED_SWITCH_TOL;
    if (const char* e = std::getenv("PKR_TEST_SWITCH_TOL")) sw16 = sw32 = std::atof(e);
    int stages[3];
    double switch_tol[3];
    int nst = 0;
    if (p->precision == PKR_MIXED16) {
        stages[nst] = PKR_FP16, switch_tol[nst++] = sw16;
        stages[nst] = PKR_FP32, switch_tol[nst++] = sw32;
        stages[nst] = PKR_FP64, switch_tol[nst++] = p->tol;
    } else if (p->precision == PKR_MIXED || p->precision == PKR_MIXED_FX64) {
        stages[nst] = PKR_FP32, switch_tol[nst++] = sw32;
        stages[nst] = p->precision == PKR_MIXED ? PKR_FP64 : PKR_FX64, switch_tol[nst++] = p->tol;
    } else {
        stages[nst] = p->precision, switch_tol[nst++] = p->tol;
    }
    pkr_problem p1 = *p;
    p1.precision = stages[0];
    pkr_plan* P = nullptr;
    int rc = pkr_plan_create(&p1, stream, &P);
    if (rc != PKR_OK) return rc;
    rc = pkr_plan_load_source(P, rho, host_buffers);
    if (rc != PKR_OK) {
        pkr_plan_destroy(P);
        return rc;
    }
    pkr_stats s{};
    double upd_bytes = 0.0;
    int64_t prev_launches = 0;
    for (int k = 0; k < nst; ++k) {
        if (k > 0) {
            // Hand the state on with little memory: the rung's second array
            // goes first, the next rung is built with one array, receives
            // the converted state in it, and gets its second array once the
            // previous rung is gone.  Peak: the rung's state + one array of
            // the next (binary32 to binary64 at 512^3: 60 + 119 GB; then the
            // two binary64 arrays, 238 GB).
            pkr_problem pk = *p;
            pk.precision = stages[k];
            plan_free_spare(P);
            pkr_plan* P2 = nullptr;
            rc = plan_create(&pk, stream, &P2, false);
            if (rc == PKR_OK) rc = load_source(P2, rho, host_buffers, false);
            if (rc == PKR_OK) rc = pkr_plan_import(P2, P);
            if (rc != PKR_OK) {
                if (P2) pkr_plan_destroy(P2);
                break;
            }
            pkr_plan_destroy(P);
            P = P2;
            rc = plan_alloc_spare(P);
            if (rc != PKR_OK) break;
        }
        const bool last = (k == nst - 1);
        if (!last) P->stall_cap = stages[k] == PKR_FP16 ? 0.1 : 1e-3;
        double t = switch_tol[k];
        if (!last && p->tol > t) t = p->tol;
        if (p->tol <= 0.0) t = 0.0;
        const int64_t left = p->max_sweeps - (P->launches - 1);
        if (left > 0) rc = pkr_plan_run(P, left, t, p->tol_kind, p->check_every, &s);
        upd_bytes += (double)(P->launches - prev_launches) * (double)P->V *
                     (2.0 * P->lat.Q * P->elem + source_bytes(P->prob.precision));
        prev_launches = P->launches;
        if (rc != PKR_OK) break;
        if (p->tol <= 0.0) break;    // fixed step count: first stage only
        if (s.residual >= 0.0 && s.residual < p->tol) break;
    }
    const int64_t launches_total = P->launches;
    if (rc == PKR_OK && p->tol > 0.0 && !(s.residual >= 0.0 && s.residual < p->tol))
        rc = PKR_ENOCONV;
    if (rc == PKR_OK || rc == PKR_ENOCONV) {
        int rc2 = pkr_plan_phi(P, phi, host_buffers);
        if (rc2 != PKR_OK) rc = rc2;
    }
    const double ms = now_ms() - t0;
    if (st) {
        *st = s;
        st->sweeps = P->launches - 1;
        st->launches = launches_total;
        st->wall_ms = ms;
        st->glups = ms > 0 ? (double)launches_total * (double)P->V / (ms * 1e6) : 0.0;
        st->hbm_gbs = ms > 0 ? upd_bytes / (ms * 1e6) : 0.0;
    }
    pkr_plan_destroy(P);
    return rc;
}

}  // extern "C"
