/*
 * pkr.h -- C ABI of the GB300 high-order kinetic relaxation Poisson solver.
 *
 * The library solves the periodic Poisson problem
 *     lap Phi = -(rho - <rho>) / eps
 * (the paper's Eq. poisson1, Sec. "Numerical Results") as the steady state of
 * a lattice-Boltzmann diffusion scheme whose equilibrium and source weights
 * are Hermite expansions truncated at order N so that the unwanted high-order
 * moments vanish (Sec. "Kinetic approach to the Poisson equation", Eqs. CON,
 * equilibrium2, omega:eq, chi:eq, omega:eq3, chi:eq3).  One time step at every
 * site x, for all discrete velocities v_i:
 *     g_i(x)     = f_i(x - v_i)                       streaming (periodic)
 *     Phi(x)     = sum_i g_i(x)                       zeroth moment
 *     f'_i(x)    = g_i(x) - (g_i(x) - phi_i Phi(x))/tau_lb + chi_i S(x)
 * with S = (rho - <rho>) c_s^2 (tau_lb - 1/2) / eps (text after Eq. poisson1)
 * and populations starting at zero.  Steps repeat until the change of Phi
 * over one step drops below a tolerance.  Everything runs in this library's
 * CUDA kernels on one GPU.
 *
 * Conventions for every entry point:
 *   - Return value: a pkr_status (0 = PKR_OK, negative = error).  No call
 *     throws or aborts; on an error no output buffer is written unless the
 *     entry point says otherwise.
 *   - Grids are given as n[3] = {nx, ny, nz}; unused dimensions are 1.  Site
 *     arrays (rho, Phi) are dense, x fastest: index (z*ny + y)*nx + x.
 *   - "Device pointer" means memory of the GPU that is current when the call
 *     is made; "host pointer" means ordinary (pageable or pinned) host memory.
 *   - The caller owns every buffer it passes in; the library owns what a plan
 *     allocates and frees it in pkr_plan_destroy.
 *   - stream: a cudaStream_t passed as void*; NULL means the legacy default
 *     stream.  Calls that return results synchronise that stream.
 *   - A NULL handle, or a NULL pointer where one is required, is refused
 *     with PKR_EINVAL before any device work; pkr_plan_destroy(NULL) and
 *     pkr_ctx_destroy(NULL) are no-ops returning PKR_OK.  Pointers an entry
 *     point marks "may be NULL" are optional outputs.
 */
#ifndef PKR_H
#define PKR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pkr_status {
    PKR_OK = 0,
    PKR_EINVAL = -1,     /* bad argument: sizes, lattice/order, tau, NaN in rho */
    PKR_ENOMEM = -2,     /* device allocation failed or over the budget */
    PKR_EUNSTABLE = -3,  /* tau_lb below the lattice's stability bound */
    PKR_ENOCONV = -4,    /* max_sweeps reached before tol (Phi still written) */
    PKR_EDIVERGED = -5,  /* residual became non-finite or grew without bound */
    PKR_ECUDA = -6,      /* a CUDA runtime call failed */
    PKR_EBUSY = -7       /* a ticket has not finished yet */
} pkr_status;

/* Velocity sets.  1D sets: the paper's Appendix (N=3 set {0,+-1,+-3}, N=5 set
 * {0,+-1,+-2,+-3,+-5}, N=7 set {0,..,+-6}); 2D sets: their tensor products;
 * D3Q19: standard first-order LB; D3Q111: Appendix Table "vector2". */
typedef enum pkr_lattice {
    PKR_D1Q5 = 0, PKR_D1Q9 = 1, PKR_D1Q13 = 2,
    PKR_D2Q25 = 3, PKR_D2Q81 = 4, PKR_D2Q169 = 5,
    PKR_D3Q19 = 6, PKR_D3Q111 = 7
} pkr_lattice;

/* Storage of the populations.  FP64: stored and updated in binary64.
 * FP32: stored and updated in binary32 (Phi, residual norms and the source
 * mean stay binary64); the per-step change of Phi bottoms out near 1e-7 of
 * Phi, so binary32 alone cannot meet tighter tolerances.  binary32 rounding
 * does not conserve the mass sum_x Phi; plans remove the drift at every
 * residual check (through the source of the next step).
 * MIXED (pkr_solve and contexts): binary32 steps until the per-step change falls
 * below PKR_MIXED_SWITCH_TOL (or tol, if looser), then the state is
 * converted to binary64 and binary64 steps continue to tol.  The binary64
 * iteration converges to the binary64 fixed point from any start, so the
 * result meets tol as a pure binary64 solve would, at binary32 cost for the
 * early decades.
 * FP16: populations stored in binary16 with a power-of-two scale per array
 * (set before each step so that the step's largest value has 4x headroom),
 * arithmetic in binary32, source in binary32; accurate to ~1e-4 of Phi.
 * Where nx is a multiple of 64 and no edge is below the lattice's reach, the
 * sweep gives each lane two adjacent sites (variant 1, the default there;
 * variant 0 keeps one site per lane); both give the same Phi bit for bit
 * between residual checks.
 * MIXED16 (pkr_solve only): binary16 to PKR_MIXED16_SWITCH_TOL, binary32 to
 * PKR_MIXED_SWITCH_TOL, then binary64 to tol.
 * A reduced-precision rung also hands over at its rounding floor, which can
 * lie above the switch tolerance: in pkr_solve's ladders when four checks in
 * a row bring no new smallest per-step change (below 0.1 for binary16, 1e-3
 * for binary32); in contexts when the change stops falling from one check to
 * the next (below 1e-3).  (Tests can set both switch tolerances of pkr_solve
 * with the environment variable PKR_TEST_SWITCH_TOL.)
 * FX64: populations stored as 64-bit integers v 2^F with a power-of-two scale
 * per array (F lowered on the device whenever the largest stored value
 * passes 2^54).  The density is an exact integer sum and the relaxation a
 * 64 x 64-bit fixed-point product by (1 - omega) (rounded to nearest) plus
 * the per-class equilibrium-and-source term; only that term and the density
 * conversion use binary64.  The largest stored value stays in [2^51, 2^54],
 * so every value is resolved to 2^-51 or finer relative to the largest one:
 * about binary64's accuracy for the field as a whole (not for values many
 * orders below the largest).  On GPUs with little binary64 throughput it runs
 * the sweep on the integer units.
 * MIXED_FX64 (pkr_solve and contexts): as MIXED, with the continuation in
 * 64-bit fixed point (FX64) instead of binary64 storage: the converted state's
 * exponent is set from its largest magnitude.  */
typedef enum pkr_precision {
    PKR_FP64 = 0, PKR_FP32 = 1, PKR_MIXED = 2, PKR_FP16 = 3, PKR_MIXED16 = 4, PKR_FX64 = 5,
    PKR_MIXED_FX64 = 6
} pkr_precision;
#define PKR_MIXED_SWITCH_TOL 1e-6
#define PKR_MIXED16_SWITCH_TOL 1e-3

/* Stopping rule: change of Phi over one step, checked every check_every
 * steps.  MAX_ABS: max_x |Phi^t - Phi^(t-1)|.  REL_L2: ||dPhi||_2/||Phi^t||_2. */
typedef enum pkr_tol_kind { PKR_TOL_MAX_ABS_DPHI = 0, PKR_TOL_REL_L2_DPHI = 1 } pkr_tol_kind;

typedef struct pkr_problem {
    int32_t dim;          /* 1, 2 or 3; must match the lattice */
    int32_t lattice;      /* pkr_lattice */
    int64_t n[3];         /* periodic grid {nx, ny, nz}, each >= 1, n[k]=1 for k>=dim */
    int32_t order;        /* expansion order N in {1,3,5,7}; <= the lattice's maximum */
    int32_t precision;    /* pkr_precision */
    double tau_lb;        /* relaxation time; > 0.5 used as is, <= 0 => from knudsen */
    double knudsen;       /* Kn = c_s (tau_lb - 1/2) / min(n): used if tau_lb <= 0 */
    double epsilon;       /* permittivity eps > 0 (0 means 1) */
    double tol;           /* stop when the residual < tol; <= 0: run max_sweeps steps */
    int32_t tol_kind;     /* pkr_tol_kind */
    int32_t check_every;  /* steps between residual checks (<= 0: 32) */
    int64_t max_sweeps;   /* upper bound on the steps taken (>= 1) */
    int32_t variant;      /* sweep kernel geometry: -1 = library default, 0 .. count-1 =
                             a compiled variant (pkr_variant_count); in binary64 and
                             fixed point all variants give identical results (binary32
                             ones differ in rounding), they differ in speed.  -1 picks
                             a geometry by grid size: the early-refill x-pairs sweep
                             for sets of more than 64 velocities on grids of whole
                             64-site x pairs with a few pairs per block (not D2Q169
                             in fixed point), else 2 velocity groups x 2 tiles, or
                             4 x 1 on grids of a few tiles per SM.  With -1, a
                             binary64 problem at tau_lb == 1 (omega = 1, the paper's
                             setting) runs as the scalar stencil Phi' = sum_i phi_i
                             Phi(x - v_i) + sum_i chi_i S(x - v_i): at omega = 1 the
                             collision forgets the populations, so this is the same
                             iteration with 24 instead of 2Q*8+8 bytes per site */
} pkr_problem;

typedef struct pkr_stats {
    int64_t sweeps;          /* steps t such that the returned Phi is Phi^t */
    int64_t launches;        /* sweep kernels launched */
    double residual;         /* last checked change of Phi (-1 if none) */
    double rho_mean_removed; /* <rho> subtracted before solving */
    double tau_lb;           /* relaxation time used */
    double cs2;              /* lattice c_s^2 */
    double wall_ms;          /* host wall time of the call */
    double glups;            /* site updates / wall time, 1e9 / s */
    double hbm_gbs;          /* algorithmic bytes / wall time, GB/s */
    int32_t variant;         /* sweep geometry that ran (its last plan, for a precision
                                ladder): an index into the list pkr_variant_count counts
                                (pkr_batch_variant_count for a context's request; binary16:
                                0 one site per lane, 1 two); -1 when no population sweep
                                ran (scalar stencil, pkr_fixed_point_fft) */
} pkr_stats;

/* Human-readable name of a status code (static string). */
const char *pkr_status_str(int status);

/* Library version string, e.g. "pkr 0.1 sm_103a". */
const char *pkr_version(void);

/*
 * Velocity set and weights of a lattice at expansion order N (host only; no
 * GPU needed).  Velocities are in the library's order (grouped by symmetry
 * class).  Any output pointer may be NULL.  vel: 3*Q int32 (x,y,z per
 * velocity); w, phi, chi: Q doubles.  phi_i, chi_i follow the isotropic
 * Hermite expansions of order N (Eqs. omega:eq, chi:eq for D=1, N=7 and
 * omega:eq3, chi:eq3 for D=3, N=5).  Errors: PKR_EINVAL for an unknown
 * lattice or an order the lattice cannot carry.
 */
int pkr_lattice_info(int lattice, int order, int32_t *Q, int32_t *dim, int32_t *vel,
                     double *w, double *phi, double *chi, double *cs2);

/* tau_lb = 1/2 + Kn * min_k(n_k > 1) / c_s (Kn = lambda / L with the mean free
 * path lambda = c_s (tau_lb - 1/2); Sec. "From Boltzmann kinetic theory to
 * diffusion equation").  Host only. */
int pkr_tau_from_knudsen(int lattice, double knudsen, const int64_t n[3], double *tau_lb);

/* Number of compiled sweep-kernel geometries of a plan for a lattice: the
 * staged ones (velocity groups per 32-site tile x tiles per block) first,
 * then, for sets of more than 64 velocities, the warp-specialised one (loader
 * warps filling a ring of tile slots, groups of compute warps draining it)
 * and the two aligned x-pairs ones (64-site x pairs copied from aligned runs;
 * the second refills each symmetry class's rows for the block's next pair as
 * soon as that class is relaxed).  The x-pairs variants apply to grids whose
 * x edge is a multiple of 64 and whose every edge is at least the reach;
 * asked for on other grids, a plan takes the staged 2 x 2 geometry instead.
 * Host only; < 0 for an unknown lattice. */
int pkr_variant_count(int lattice);

/* Number of compiled geometries of the batch sweep (pkr_ctx_config.variant
 * ranges over 0 .. count - 1): the staged ones only.  Host only; < 0 for an
 * unknown lattice. */
int pkr_batch_variant_count(int lattice);

/* Device bytes a plan for this problem allocates (populations, source, Phi,
 * scratch).  Host only. */
int pkr_plan_bytes(const pkr_problem *problem, size_t *bytes);

/* ---------------------------------------------------------------------
 * Plans: device-resident state of one solve.  A plan owns two population
 * arrays (Q planes of V sites each, ping-pong), the source S, Phi and a small
 * scratch area.  All work is queued on the plan's stream.
 * --------------------------------------------------------------------- */
typedef struct pkr_plan pkr_plan;

/* Validate the problem, build the lattice tables and allocate device memory
 * on the current device.  Errors: PKR_EINVAL, PKR_EUNSTABLE (tau_lb at or
 * below the lattice's stability bound), PKR_ENOMEM, PKR_ECUDA. */
int pkr_plan_create(const pkr_problem *problem, void *stream, pkr_plan **out);

/* Free everything the plan owns (after synchronising its stream). */
int pkr_plan_destroy(pkr_plan *plan);

/* Step a0: S = (rho - <rho>) c_s^2 (tau_lb - 1/2) / eps with the mean taken in
 * binary64 in a fixed order, and reset the populations to zero (t = 0).
 * rho: V doubles, device pointer (rho_on_host = 0) or host pointer (1).
 * Synchronises.  Errors: PKR_EINVAL if rho holds NaN or Inf. */
int pkr_plan_load_source(pkr_plan *plan, const double *rho, int rho_on_host);

/* Advance until Phi^(t + steps) is known, checking the residual every
 * check_every steps (<= 0: the problem's value) and stopping early once it
 * drops below tol (tol <= 0: never).  stats may be NULL.  Returns PKR_OK,
 * PKR_EDIVERGED or PKR_ECUDA.  Synchronises once per check; except that a
 * binary64 run that checks every step (check_every = 1, tol > 0, steps >= 64)
 * runs its steps as a CUDA graph of 64 steps captured on a stream of the plan
 * and launched on the plan's stream, with the stopping rule applied on the
 * device after each check: same steps and stopping step, one synchronisation
 * per 64 steps. */
int pkr_plan_run(pkr_plan *plan, int64_t steps, double tol, int tol_kind, int check_every,
                 pkr_stats *stats);

/* Autotuner: time every compiled sweep variant that applies to the plan's
 * grid (the x-pairs variants only on grids of whole 64-site x pairs; see
 * pkr_variant_count) on the plan's own buffers (one warm-up step, then
 * `steps_per_variant` timed steps each, CUDA events on the plan's stream)
 * and keep the fastest.  The steps are real steps of the solve: the plan
 * advances by (1 + steps_per_variant) x (variants timed) steps.  Must
 * follow pkr_plan_load_source.  best_variant / best_ms_per_step may be NULL.
 * Synchronises. */
int pkr_plan_autotune(pkr_plan *plan, int steps_per_variant, int32_t *best_variant,
                      double *best_ms_per_step);

/* Continue from another plan's state: copy (converting the storage type) the
 * populations and Phi of `from`, which must have the same lattice, order and
 * grid, and take over its step count.  Both plans must have loaded the same
 * source (the receiving plan keeps its own S).  The copied state is projected
 * onto the zero-mass gauge (mean of Phi removed through the k = 0
 * equilibrium mode), which the exact iteration from zero keeps to rounding.
 * Into PKR_FX64 the exponent is set from the largest converted magnitude.
 * Not into PKR_FP16, nor from PKR_FX64 (PKR_EINVAL).  Synchronises. */
int pkr_plan_import(pkr_plan *plan, const pkr_plan *from);

/* Queue `count` plain steps (no residual, no synchronisation).  For timing. */
int pkr_plan_sweeps(pkr_plan *plan, int64_t count);

/* Copy the most recent Phi^t (binary64, V values) into phi: a device pointer
 * (phi_on_host = 0) or host pointer (1).  Computes it first if the last step
 * did not.  Synchronises. */
int pkr_plan_phi(pkr_plan *plan, double *phi, int phi_on_host);

/* Steps t completed so far (Phi^t is the latest density). */
int64_t pkr_plan_steps(const pkr_plan *plan);

/* Raw access for tests: device pointer of the current population array
 * (Q*V elements of the storage type, plane i at offset i*V) and of Phi. */
void *pkr_plan_populations(pkr_plan *plan);

/* ---------------------------------------------------------------------
 * One-shot solve: create a plan, load rho, run to tol (or max_sweeps), write
 * Phi, destroy the plan.  rho and phi are device pointers, or host pointers
 * when host_buffers != 0 (copies then happen inside the call).  Phi is written
 * on PKR_OK and on PKR_ENOCONV (best effort, stats filled); untouched on
 * every other error.  With tol <= 0 exactly max_sweeps steps run and the call
 * returns PKR_OK.
 * --------------------------------------------------------------------- */
int pkr_solve(const pkr_problem *problem, const double *rho, double *phi, int host_buffers,
              pkr_stats *stats, void *stream);

/* ---------------------------------------------------------------------
 * Direct comparator: the exact fixed point of the scheme by FFT.
 *
 * The time step above (streaming, BGK relaxation to phi_i Phi, source
 * chi_i S; Sec. "Kinetic approach to the Poisson equation") is linear and
 * translation invariant on the periodic grid, so its steady state is diagonal
 * in Fourier space: Phi(k) = T(k) S(k) with
 *     T(k) = sum_i chi_i q_i / sum_i phi_i (1 - e_i) / (1 - (1 - w) e_i),
 *     q_i = e_i / (1 - (1 - w) e_i),  e_i = exp(-i k.v_i),  w = 1 / tau_lb,
 * and Phi(0) = 0.  This is the limit the iteration (pkr_solve with tol -> 0)
 * converges to -- same lattice, order, tau_lb and source, including the
 * O(Kn^2) kinetic correction -- so it serves as a direct solver for the
 * scheme and as an exact reference for its residual.  It is not the Poisson
 * solution: that is the tau_lb -> 1/2 limit.
 *
 * problem: lattice, n, order, tau_lb (or knudsen), epsilon are used; tol,
 * check_every, max_sweeps, precision and variant are ignored (binary64
 * throughout).  rho, phi: as pkr_solve (device, or host with host_buffers).
 * Device memory: V doubles + (nx/2+1) ny nz complex doubles + nx+ny+nz
 * complex phase-table entries + cuFFT's plan work area, allocated and freed
 * inside the call.  Synchronises the stream.
 * stats: rho_mean_removed, tau_lb, cs2, wall_ms (others 0).
 * Errors (phi untouched on each): PKR_EINVAL (bad problem, V > 2^31 - 1,
 * tau_lb <= 1/2, non-finite rho), PKR_EUNSTABLE (tau_lb outside the stable
 * range of the lattice, as pkr_solve), PKR_ENOMEM, PKR_ECUDA (a CUDA or cuFFT
 * call failed).
 * --------------------------------------------------------------------- */
int pkr_fixed_point_fft(const pkr_problem *problem, const double *rho, double *phi,
                        int host_buffers, pkr_stats *stats, void *stream);

/* ---------------------------------------------------------------------
 * Batches and serving: a context advances many independent periodic solves
 * (same lattice, order and storage) together, one persistent kernel launch
 * per step over all live grids, K steps per captured CUDA graph.  Requests
 * are admitted first-fit while their device bytes fit the HBM budget, join at
 * the next K-step boundary, and retire when their own residual check (every
 * K steps of their own age) passes; the freed memory admits the next ones.
 * A grid's result does not depend on what else is in the batch.
 * A PKR_MIXED context keeps two batches, binary32 and binary64: a request
 * starts in binary32 and, at the check where its residual falls below
 * PKR_MIXED_SWITCH_TOL (or stops falling, at the binary32 rounding floor),
 * its state is converted to binary64 (projected onto the zero-mass gauge)
 * and it continues in the binary64 batch to its tolerance, with its step
 * count and check schedule unchanged.  Requests with tol >= the switch
 * tolerance finish in binary32.  Its budget reservation per request is the
 * binary32 state + the binary64 state + Phi (both states exist while it is
 * converted); the binary32 share is released at the switch.
 * A PKR_FX64 context stores every grid in 64-bit fixed point, each grid with
 * its own pair of array exponents, rescaled on the device after every step.
 * A PKR_MIXED_FX64 context is a MIXED one whose second batch is PKR_FX64.
 * --------------------------------------------------------------------- */
typedef struct pkr_ctx pkr_ctx;

typedef struct pkr_ctx_config {
    int32_t lattice;          /* pkr_lattice of every request */
    int32_t order;            /* expansion order N of every request */
    int32_t precision;        /* PKR_FP64, PKR_FP32, PKR_FX64, PKR_MIXED or
                                 PKR_MIXED_FX64, for every request */
    int32_t check_every;      /* K: steps per graph replay and per residual check (>= 1) */
    size_t hbm_budget_bytes;  /* device bytes the live requests may hold */
    int32_t variant;          /* 0 .. pkr_batch_variant_count - 1: kernel geometry;
                                 -1: library default; -2: autotune on a probe grid
                                 of edge probe_edge */
    int32_t probe_edge;       /* edge of the cubic probe grid for variant = -2 */
    int32_t threaded;         /* 1: a worker thread drives the batch; 0: pkr_ctx_run does */
    int32_t max_grids;        /* most requests live at once (<= 0: 4096) */
} pkr_ctx_config;

/* Create a context on the current device.  stream: the stream all its work
 * is queued on.  Errors: PKR_EINVAL, PKR_ENOMEM, PKR_ECUDA. */
int pkr_ctx_create(const pkr_ctx_config *config, void *stream, pkr_ctx **out);

/* Queue a request.  problem: its grid, tau/Kn, eps, tol, tol_kind and
 * max_sweeps (lattice, order and precision must match the context).  rho: V
 * doubles; phi: V doubles written when the request finishes (device pointers,
 * or host pointers when host_buffers != 0); both must stay valid until then.
 * ticket: the request's id.  Errors: PKR_EINVAL, PKR_ENOMEM (the request alone
 * exceeds the budget). */
int pkr_submit(pkr_ctx *ctx, const pkr_problem *problem, const double *rho, double *phi,
               int host_buffers, uint64_t *ticket);

/* State of a request: PKR_EBUSY while queued or running, otherwise its final
 * status (PKR_OK, PKR_ENOCONV, PKR_EDIVERGED, PKR_EINVAL for a source with
 * NaN/Inf, PKR_ECUDA); stats (may be NULL) is filled once it has finished:
 * sweeps, residual, rho_mean_removed, tau_lb, cs2, and wall_ms = completion
 * minus submission. */
int pkr_poll(pkr_ctx *ctx, uint64_t ticket, pkr_stats *stats);

/* Drive a non-threaded context from the caller's thread: admit what fits and
 * run K-step windows until nothing is queued or live, or max_windows windows
 * have run (max_windows <= 0: no limit).  Several threads may call it (and
 * pkr_ctx_wait) on one context: one at a time runs a round, the others wait
 * for that round to end.  Returns PKR_OK or PKR_ECUDA; after PKR_ECUDA every
 * request that was queued or running has finished with PKR_ECUDA and has
 * given its device memory back.  (Tests can make the n-th round, counted
 * from 0 per context, report PKR_ECUDA without launching anything by setting
 * the environment variable PKR_TEST_FAIL_ROUND=n before pkr_ctx_create.) */
int pkr_ctx_run(pkr_ctx *ctx, int64_t max_windows);

/* Block until a request has finished and return as pkr_poll does.  In a
 * threaded context the worker drives; in a non-threaded one the caller runs
 * rounds until the request finishes (PKR_EINVAL if nothing is left to run
 * and it has not). */
int pkr_ctx_wait(pkr_ctx *ctx, uint64_t ticket, pkr_stats *stats);

/* Forget a finished request: its ticket becomes invalid and the context's
 * record of it (status and stats) is freed.  Long-running contexts call this
 * once a request's result has been read, so that their bookkeeping stays
 * bounded.  Errors: PKR_EINVAL (NULL context or unknown ticket), PKR_EBUSY
 * (the request is still queued or running, or another thread is waiting on
 * it in pkr_ctx_wait). */
int pkr_ctx_release(pkr_ctx *ctx, uint64_t ticket);

/* Counters: requests finished, site updates performed, windows run, bytes
 * currently held, kernel variant in use.  Any pointer may be NULL. */
int pkr_ctx_info(pkr_ctx *ctx, int64_t *finished, double *site_updates, int64_t *windows,
                 size_t *bytes_in_use, int32_t *variant);

/* Stop the worker (if any), drop queued and running requests (their phi is
 * not written), free everything.  The context and its tickets are invalid
 * afterwards.  No other thread may be inside a call on this context. */
int pkr_ctx_destroy(pkr_ctx *ctx);

/* ---------------------------------------------------------------------
 * Memory ceiling of the sweep's access pattern (a diagnostic for the
 * roofline; the paper has no counterpart).
 *
 * Moves the bytes of one sweep without arithmetic: Q planes of V values of
 * elem_bytes (8: binary64 or fixed point, 4: binary32) read through the
 * sweep's per-lane asynchronous copies of 32-site tiles into shared memory
 * and written back with streaming stores, in the staged sweep's default
 * geometry (2 velocity groups x 2 tiles per block of 4 warps), as many
 * blocks as fit.  shift_axes selects which components of the pull offsets
 * -v_i are kept: 0 none (a plain copy of Q planes), 1 x only, 2 y and z only,
 * 3 all (the staged sweep's pull); 7 all, with the x offsets served from
 * aligned runs (the block's two tiles x-adjacent, nx a multiple of 64: each
 * velocity's two aligned 32-site blocks plus one aligned 4-site halo, per
 * lane, read back shifted); 8 all, through the aligned x-pairs sweep's own
 * staging (halo = the reach, values written shifted by v_x; nx a multiple
 * of 64).  Runs one untimed and `reps` timed copies on `stream`
 * and returns, in *gbs, the bytes read and written per second (1e9 B/s).
 * It allocates 2 x Q x V x elem_bytes of device memory for the call.
 * lattice: PKR_D3Q19 or PKR_D3Q111; every edge at least the lattice's reach.
 * Errors: PKR_EINVAL (other lattices or element sizes, an edge below the
 * reach, V outside [1, 2^31 - 1], reps < 1, shift_axes not in 0..3, 7 or 8,
 * nx not a multiple of 64 for 7 and 8), PKR_ENOMEM, PKR_ECUDA.
 */
int pkr_pull_copy_ceiling(int lattice, const int64_t n[3], int elem_bytes, int shift_axes,
                          int reps, double *gbs, void *stream);

/* ---------------------------------------------------------------------
 * Allocation-free residual (the paper has no counterpart: this is a service
 * for callers that cannot allocate device memory -- runtimes whose device
 * memory all belongs to their own pool and that forbid side allocations, and
 * loops that must not enter the allocator, where cudaMalloc and cudaFree can
 * synchronise the device).
 *
 * Computes, in binary64 with a fixed reduction order, the same change of Phi
 * that the solver's stopping rule uses:
 *     out[0] = max_x |phi_new - phi_old|
 *     out[1] = ||phi_new - phi_old||_2 / ||phi_new||_2   (0 if both vanish,
 *              +inf if only phi_new does)
 *     out[2] = ||phi_new||_2
 * For finite inputs whose squares and sums stay finite these are finite
 * (out[1] may be +inf as stated).  If an input holds NaN, out[0] and out[1]
 * are NaN.  If an input holds +-inf, or a square or a sum overflows, the
 * binary64 arithmetic decides: out[1] can then be NaN (inf / inf) although
 * no input is NaN, so a NaN in out[1] means "not finite", not "NaN input".
 * phi_new, phi_old: device pointers to V doubles each.  out: host pointer to
 * 3 doubles.  The call queues two kernels on `stream`, copies out[] back and
 * synchronises the stream before it returns.
 *
 * Memory: no cudaMalloc, cudaFree or allocating library routine is called.
 * The scratch (at most 1024 block partials of 3 doubles and the three
 * results, 24.6 KB) is a static device array of the library, held on every
 * GPU that loads the library until the process exits.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) with
 * the device current; make that first call before any stream capture.  All
 * calls on a device share the
 * array and it keeps the last call's contents, so calls that overlap on the
 * GPU (different streams, no ordering between them) race: order them.
 *
 * Errors: PKR_EINVAL for NULL pointers or V outside [1, PKR_NOALLOC_MAX_SITES];
 * PKR_ECUDA if a CUDA call fails.
 */
#define PKR_NOALLOC_MAX_SITES 2147483647LL
int pkr_residual_noalloc(const double *phi_new, const double *phi_old, int64_t V, double out[3],
                         void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PKR_H */
