// pkr_internal.h -- declarations shared by the library's translation units.
#pragma once
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <vector>

#include "../../include/pkr.h"
#include "pkr_lattices.h"

namespace pkr {

constexpr int kMaxQ = 169;

struct LatticeInfo {
    int lattice, order, Q, dim, reach, ncls;
    int vel[3 * kMaxQ];
    int cls[kMaxQ];
    int key[kMaxQ];
    long double wl[kMaxQ];
    double w[kMaxQ], phi[kMaxQ], chi[kMaxQ];
    double cls_phi[kMaxClasses], cls_chi[kMaxClasses];
    long double cs2l;
    double cs2;
};

int build_lattice(int lattice, int order, LatticeInfo* out);
bool unstable(const LatticeInfo& li, double omega);

// Per-class coefficients handed to the sweep kernels by value (kernel
// parameter space, so concurrent plans never share state).
template <typename R>
struct Coefs {
    R om1;                     // 1 - omega
    R wphi[kMaxClasses];       // omega * phi_c
    R chi[kMaxClasses];        // chi_c
};

enum SweepMode { kPlain = 0, kWritePhi = 1, kCheck = 2 };
enum SweepVariant { kStaged = 0 };

// Storage precision code of binary16 populations (include/pkr.h: PKR_FP16).
constexpr int kFP16 = 3;
// Storage precision code of 64-bit fixed-point populations (PKR_FX64).
constexpr int kFX64 = 5;

// One grid of a batch (device-resident descriptor, see pkr_batch.cpp).
template <typename R>
struct BatchGrid {
    void* pop[2];          // ping-pong populations
    const void* S;         // source
    double* Phi;           // density
    int64_t V;
    int nx, ny, nz, small;
    int tile_begin;        // first batch-wide tile of this grid
    int pad;
    long long join;        // batch step at which the grid starts from zero
    // 64-bit fixed-point storage only (device memory of the grid): exponents
    // of the two arrays, OR of |stored| over the current step, and
    // round((1 - omega) 2^62)
    int* fxF;
    unsigned long long* fxmax;
    long long cfx;
    // binary32 storage only (device memory of the grid): source offset that
    // removes the measured mass, written at a check, used by the next step
    double* soff;
    Coefs<R> c;
};

// Device-resident state read by every batch launch, so that a captured graph
// stays valid while grids join and retire.
struct BatchState {
    const void* grids;     // BatchGrid<R>[ngrids], sorted by tile_begin
    double* tile_partials; // 4 doubles per batch-wide tile (check steps)
    double* grid_res;      // 4 doubles per grid (after the per-grid reduction)
    long long step;        // batch step counter (launch index)
    int ngrids;
    int ntiles;
};

struct SweepArgs {
    const void* A;        // populations in (pulled), Q planes of V
    void* B;              // populations out
    const void* S;        // source, V values of the storage type
    double* Phi;          // density buffer (binary64)
    double* partials;     // residual partials: 4 doubles per block
    int64_t V;            // sites
    int32_t nx, ny, nz;
    int32_t ntiles;       // flat tiles of 32 sites
    int32_t mode;         // SweepMode
    int32_t zero_in;      // populations in are all zero (first step)
    int32_t small;        // some edge shorter than the lattice reach
    int32_t cur;          // index (0/1) of the population array read (binary16 scales)
    double soff;          // constant added to S in this step (mass correction)
    // binary16 storage only: per-array scales sc[2] (a value v is stored as
    // v / sc[k]), the running max |p| of this step (float bits) and an
    // overflow flag
    float* sc;
    unsigned int* pmax;
    int* oflow;
    // 64-bit fixed-point storage only: exponents fxF[2] (a value v is stored
    // as round(v 2^fxF[k]) in array k), the OR of |stored| over this step
    // (bit length of the largest |stored|), and
    // 1 - omega as round((1 - omega) 2^62)
    int* fxF;
    unsigned long long* fxmax;
    long long cfx;
    // device flag: when it is set the launch returns at once (steps queued in
    // a captured graph after the solve has stopped); nullptr: never
    const int* stop;
};

// State of a device-side stopping rule (a captured run of check steps):
// after each check the rule of pkr_plan_run is applied on the device and the
// remaining steps of the graph see stop != 0 and do nothing.
struct RunCtl {
    int stop;         // 1 once converged or diverged
    int status;       // PKR_OK or PKR_EDIVERGED
    int done_at;      // index (in the graph) of the step that stopped
    int nchecks;      // checks so far in this run
    double min_res;   // smallest residual so far in this run
    double last_res;  // last checked residual
};


// Source preparation and reductions (pkr_kernels.cu).
int launch_rho_partials(const double* rho, int64_t V, double* partials, int nblocks,
                        int* nonfinite, void* stream);
int launch_finalize_mean(const double* partials, int nblocks, int64_t V, double* mean,
                         void* stream);
int launch_make_source(const double* rho, const double* mean, double scale, int64_t V,
                       void* S, int precision, void* stream);
// Threads per block of the scalar stencil: 64 on grids too small to give
// every SM a 256-thread block, else 256.  A launch of `grid` blocks over V
// sites used 64 exactly when grid * 64 >= V.
inline int stencil_block(int64_t V, int nsm) { return V < (int64_t)nsm * 256 ? 64 : 256; }

int launch_finalize_residual(const double* partials, int nblocks, double* out4, void* stream);
// finalize_residual, then the stopping rule on the device for check step j
// of a captured run (does nothing once ctl->stop is set).
int launch_finalize_check(const double* partials, int nblocks, double* out4, RunCtl* ctl,
                          double tol, int tol_kind, int j, void* stream);

// Batch engine kernels (sweep_*.cu / pkr_kernels.cu).
int launch_batch_step(int lattice, int precision, int variant, BatchState* state, int check_every,
                      int grid, void* stream);
int batch_occupancy(int lattice, int precision, int variant, int* blocks_per_sm);
int launch_batch_reduce(BatchState* state, int max_grids, int grid_stride_bytes, void* stream);
int launch_batch_increment(BatchState* state, void* stream);
// 64-bit fixed-point batches: after a step, each grid's rescale (as
// launch_fx_rescale does for a plan), for the array its next step writes.
int launch_batch_fx_rescale(BatchState* state, int max_grids, void* stream);
int launch_convert(const void* in, int in_precision, void* out, int out_precision, int64_t n,
                   void* stream);
// out[i*V + x] = in[i*V + x] - shift[i] (storage conversion with a per-plane
// shift; shift: Q doubles in device memory).
int launch_convert_shift(const void* in, int in_precision, void* out, int out_precision, int Q,
                         int64_t V, const double* shift, void* stream, const float* in_scale = nullptr);
// Into 64-bit fixed point: max |in * in_scale - shift_i| over Q planes (as
// binary64 bits, atomicMax into *out), and out = round((in * in_scale -
// shift_i) 2^F).  in_scale: binary16 inputs only (device pointer).
int launch_absmax_shift(const void* in, int in_precision, int Q, int64_t V, const double* shift,
                        const float* in_scale, unsigned long long* out, void* stream);
int launch_convert_fx(const void* in, int in_precision, long long* out, int Q, int64_t V,
                      const double* shift, const float* in_scale, int F, void* stream);
// Exponent of a fixed-point array whose largest magnitude is m: the largest
// stored value lands in [2^51, 2^52).
inline int fx_exponent(double m)
{
    int e = 0;
    if (m > 0.0 && m < 1.0e300) {
        std::frexp(m, &e);   // m in [2^(e-1), 2^e)
        return 52 - e;
    }
    return 0;
}
// binary16 storage: after a step, set the scale of the array the next step
// writes (sc[next]) from this step's max |p| (4x headroom), reset the max.
int launch_h16_rescale(float* sc, unsigned int* pmax, int next, void* stream);
// 64-bit fixed-point storage: after a step, set the exponent of the array the
// next step writes from the bit length of this step's largest |stored| (the
// OR of all of them; keep it below 2^54), reset.
int launch_fx_rescale(int* F, unsigned long long* fmax, int next, void* stream);
// max |S| of a binary64 source as bits (atomicMax into *out).
int launch_absmax_f64(const double* S, int64_t V, unsigned long long* out, void* stream);
// max |S| of a binary32 source as float bits (atomicMax into *out).
int launch_absmax_f32(const float* S, int64_t V, unsigned int* out, void* stream);

}  // namespace pkr
