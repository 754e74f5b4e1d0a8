/*
 * pkr_oracle.c -- serial FP64 oracle of the high-order kinetic relaxation
 * Poisson solver (Mendoza, Succi, Herrmann, "High-Order Kinetic Relaxation
 * Schemes as High-Accuracy Poisson Solvers").
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously correct
 * statement of the scheme that the CUDA path is checked against.  Only the
 * tests, __graft_entry__.smoke() and the CPU-baseline leg of the benchmark may
 * load it.  It shares no code, header or table with the product library:
 * the lattice tables (v_i, phi_i, chi_i) are handed in by the caller.
 *
 * The scheme, in the order the paper states it:
 *   - BGK kinetic equation with source, Eq. (boltzmann):
 *       df/dt + v.grad f = -(f - f_eq)/tau + Src
 *   - separable equilibrium and source, Eq. (equilibrium2) and the line after:
 *       f_eq_i = phi_i Phi,   Src_i = chi_i S
 *   - Phi is the zeroth moment, Phi = sum_i f_i (Sec. "From Boltzmann kinetic
 *     theory to diffusion equation"); it is taken from the populations as
 *     they arrive at a site, before they collide.
 *   - Poisson application (Sec. "Numerical Results", Eq. poisson1 and the
 *     text after it): S = rho c_s^2 tau / eps with tau = tau_lb - 1/2; the
 *     mean of rho is removed first so that the periodic problem is solvable.
 *   - periodic domain, populations start at zero.
 * One time step of the discrete scheme at every site x:
 *       Phi(x)      = sum_i g_i(x)
 *       p_i(x)      = g_i(x) - omega (g_i(x) - phi_i Phi(x)) + chi_i S(x),
 *                     omega = 1/tau_lb
 *       g_i(x+v_i)  = p_i(x)                      (streaming, periodic)
 *
 * Layout: g[i*V + (z*ny + y)*nx + x], V = nx*ny*nz.
 *
 * The same file also builds, with -fopenmp, the multi-core CPU baseline: the
 * site loop of a step is shared among threads by z-plane.  Every site's
 * arithmetic and every written address are unchanged (each (i, x) pushes to
 * its own destination), so the result is bitwise the serial one.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads used by oracle_step: sets the count when n > 0 (OpenMP build
 * only) and returns the count in effect (1 for the serial build). */
int oracle_threads(int n)
{
#ifdef _OPENMP
    if (n > 0)
        omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

static int64_t wrap(int64_t a, int64_t n)
{
    int64_t r = a % n;
    return r < 0 ? r + n : r;
}

/* a0: remove the mean of rho (FP64, plain left-to-right sum) and scale by
 * c_s^2 (tau_lb - 1/2) / eps.  Returns the removed mean. */
double oracle_source(int64_t V, const double *rho, double cs2, double tau_lb,
                     double eps, double *S)
{
    double sum = 0.0;
    for (int64_t x = 0; x < V; ++x)
        sum += rho[x];
    double mean = sum / (double)V;
    double scale = cs2 * (tau_lb - 0.5) / eps;
    for (int64_t x = 0; x < V; ++x)
        S[x] = (rho[x] - mean) * scale;
    return mean;
}

/* Phi(x) = sum_i g_i(x), summed in velocity order i = 0..Q-1. */
void oracle_density(int Q, int64_t V, const double *g, double *Phi)
{
    for (int64_t x = 0; x < V; ++x) {
        double s = 0.0;
        for (int i = 0; i < Q; ++i)
            s += g[(int64_t)i * V + x];
        Phi[x] = s;
    }
}

/* One time step: collide every site, then push each p_i(x) to x + v_i. */
void oracle_step(const int64_t n[3], int Q, const int32_t *vel,
                 const double *phi, const double *chi, double omega,
                 const double *S, const double *g, double *gnew)
{
    const int64_t nx = n[0], ny = n[1], nz = n[2];
    const int64_t V = nx * ny * nz;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                const int64_t s = (z * ny + y) * nx + x;
                double Phi = 0.0;
                for (int i = 0; i < Q; ++i)
                    Phi += g[(int64_t)i * V + s];
                for (int i = 0; i < Q; ++i) {
                    double gi = g[(int64_t)i * V + s];
                    double p = gi - omega * (gi - phi[i] * Phi) + chi[i] * S[s];
                    int64_t xd = wrap(x + vel[3 * i + 0], nx);
                    int64_t yd = wrap(y + vel[3 * i + 1], ny);
                    int64_t zd = wrap(z + vel[3 * i + 2], nz);
                    gnew[(int64_t)i * V + (zd * ny + yd) * nx + xd] = p;
                }
            }
}

/* Change of Phi between two steps.  kind 0: max |dPhi|;
 * kind 1: ||dPhi||_2 / ||Phi_new||_2 (0 when both vanish). */
double oracle_residual(int64_t V, const double *Phi_new, const double *Phi_old,
                       int kind)
{
    double mx = 0.0, d2 = 0.0, n2 = 0.0;
    for (int64_t x = 0; x < V; ++x) {
        double d = Phi_new[x] - Phi_old[x];
        if (fabs(d) > mx)
            mx = fabs(d);
        d2 += d * d;
        n2 += Phi_new[x] * Phi_new[x];
    }
    if (kind == 0)
        return mx;
    if (n2 == 0.0)
        return d2 == 0.0 ? 0.0 : INFINITY;
    return sqrt(d2) / sqrt(n2);
}

/*
 * Run steps from the state g (Q*V, updated in place) until the change of Phi
 * over one step, checked after every check_every-th step, drops below tol,
 * or max_steps steps have run.  tol <= 0 runs exactly max_steps steps.
 * On return Phi holds sum_i g_i of the final state.  Returns the number of
 * steps taken; *residual gets the last checked change (or -1 if none).
 * Returns -1 on allocation failure.
 */
int64_t oracle_solve(const int64_t n[3], int Q, const int32_t *vel,
                     const double *phi, const double *chi, double omega,
                     const double *S, double tol, int tol_kind,
                     int64_t check_every, int64_t max_steps, double *g,
                     double *Phi, double *residual)
{
    const int64_t V = n[0] * n[1] * n[2];
    double *tmp = malloc(sizeof(double) * (size_t)Q * (size_t)V);
    double *prev = malloc(sizeof(double) * (size_t)V);
    if (!tmp || !prev) {
        free(tmp);
        free(prev);
        return -1;
    }
    if (check_every < 1)
        check_every = 1;
    *residual = -1.0;
    oracle_density(Q, V, g, prev);
    int64_t t = 0;
    while (t < max_steps) {
        oracle_step(n, Q, vel, phi, chi, omega, S, g, tmp);
        memcpy(g, tmp, sizeof(double) * (size_t)Q * (size_t)V);
        ++t;
        oracle_density(Q, V, g, Phi);
        if (tol > 0.0 && t % check_every == 0) {
            *residual = oracle_residual(V, Phi, prev, tol_kind);
            if (*residual < tol)
                break;
        }
        memcpy(prev, Phi, sizeof(double) * (size_t)V);
    }
    oracle_density(Q, V, g, Phi);
    free(tmp);
    free(prev);
    return t;
}
