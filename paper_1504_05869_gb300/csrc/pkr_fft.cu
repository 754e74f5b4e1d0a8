// pkr_fft.cu -- the scheme's exact fixed point by FFT (a direct comparator).
//
// The kinetic relaxation scheme is linear and translation invariant on the
// periodic grid, so each Fourier mode k of the populations evolves on its own:
//     g(k) <- E(k) [ (1 - w) g(k) + w phi (1^T g(k)) + chi S(k) ],
// E(k) = diag(e_i), e_i = exp(-i k.v_i).  At the fixed point, with
// q_i = e_i / (1 - (1 - w) e_i) (Sherman-Morrison on the rank-one collision),
//     Phi(k) = T(k) S(k),  T(k) = sum_i chi_i q_i / (1 - w sum_i phi_i q_i),
// and Phi(0) = 0 (the gauge the iteration from zero keeps).  The velocity sets
// are symmetric (v and -v with equal weights), so q(-v) = conj(q(v)) and both
// sums are real: 2 Re over one velocity of each pair (the rest velocity once).
// The denominator is small near k = 0 (it vanishes like |k|^2); since the phi_i
// sum to one it is written as sum_i phi_i Re[(1 - e_i) / (1 - (1 - w) e_i)]
// with 1 - cos(theta) = 2 sin^2(theta / 2), so no term cancels.  The phase
// theta = k.v_i is reduced exactly on the integers (m v mod n) and its half
// angle built from per-axis tables of exp(-i pi j / n).
// The transforms are cuFFT's; the transfer function T(k) is this file's kernel.
#include <cuda_runtime.h>
#include <cufft.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "pkr_internal.h"

namespace pkr {
namespace {

constexpr int kMaxPairs = 96;   // one representative per +-v pair (D2Q169: 84 + rest)

struct FftCoefs {
    int npairs;               // representatives (rest velocity first if present)
    int vx[kMaxPairs], vy[kMaxPairs], vz[kMaxPairs];
    double phi[kMaxPairs], chi[kMaxPairs], mult[kMaxPairs];   // mult: 1 (rest) or 2 (pair)
    double omega;
};

// H[j] = exp(-i pi j / n), j < n: the half-angle phase of one axis.
__global__ void half_phase_kernel(double2* __restrict__ H, int n)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        double sn, cs;
        sincospi((double)j / n, &sn, &cs);
        H[j] = make_double2(cs, -sn);
    }
}

// Multiply the half spectrum S(k) (nx/2 + 1 modes along x) by T(k).  For a
// velocity v, theta = k.v = 2 pi sum_a (m_a v_a mod n_a) / n_a; the indices
// are reduced exactly on the integers and the half-angle phase
// h = exp(-i theta / 2) is the product of three table entries.  Then
// e = h^2 and 1 - cos(theta) = 2 Im(h)^2 (no cancellation near k = 0).
__global__ void transfer_kernel(cufftDoubleComplex* __restrict__ sk, int nx, int ny, int nz,
                                const FftCoefs c, const double2* __restrict__ Hx,
                                const double2* __restrict__ Hy, const double2* __restrict__ Hz)
{
    const int nxh = nx / 2 + 1;
    const int64_t total = (int64_t)nxh * ny * nz;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const double cw = 1.0 - c.omega;
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < total; m += stride) {
        const int mx = (int)(m % nxh);
        const int my = (int)((m / nxh) % ny);
        const int mz = (int)(m / ((int64_t)nxh * ny));
        if (mx == 0 && my == 0 && mz == 0) {
            sk[m].x = 0.0;
            sk[m].y = 0.0;
            continue;
        }
        double num = 0.0, den = 0.0;
        for (int p = 0; p < c.npairs; ++p) {
            const int jx = (int)((((int64_t)mx * c.vx[p]) % nx + nx) % nx);
            const int jy = (int)((((int64_t)my * c.vy[p]) % ny + ny) % ny);
            const int jz = (int)((((int64_t)mz * c.vz[p]) % nz + nz) % nz);
            const double2 a = __ldg(Hx + jx), b = __ldg(Hy + jy), d = __ldg(Hz + jz);
            const double tr = a.x * b.x - a.y * b.y, ti = a.x * b.y + a.y * b.x;
            const double hr = tr * d.x - ti * d.y, hi = tr * d.y + ti * d.x;   // h
            const double cs = hr * hr - hi * hi;      // e = h^2 = cs - i sn
            const double sn = -2.0 * hr * hi;
            const double omc = 2.0 * hi * hi;         // 1 - cos(theta)
            // d = 1 - (1 - w) e;  Re q = Re[e conj(d)] / |d|^2;
            // Re[(1 - e) / d] = Re[(1 - e) conj(d)] / |d|^2
            const double dr = 1.0 - cw * cs, di = cw * sn;
            const double inv = 1.0 / (dr * dr + di * di);
            num += c.mult[p] * c.chi[p] * ((cs * dr - sn * di) * inv);
            den += c.mult[p] * c.phi[p] * ((omc * dr + sn * di) * inv);
        }
        const double T = num / den;
        sk[m].x *= T;
        sk[m].y *= T;
    }
}

__global__ void scale_kernel(double* __restrict__ x, int64_t n, double s)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) x[i] *= s;
}

}  // namespace
}  // namespace pkr

using namespace pkr;

extern "C" int pkr_fixed_point_fft(const pkr_problem* p, const double* rho, double* phi,
                                   int host_buffers, pkr_stats* st, void* stream)
{
    if (!p || !rho || !phi) return PKR_EINVAL;
    LatticeInfo li;
    int rc = build_lattice(p->lattice, p->order, &li);
    if (rc != PKR_OK) return rc;
    if (li.dim != p->dim) return PKR_EINVAL;
    int64_t V = 1;
    for (int k = 0; k < 3; ++k) {
        if (p->n[k] < 1 || (k >= p->dim && p->n[k] != 1)) return PKR_EINVAL;
        V *= p->n[k];
    }
    if (V > (int64_t)0x7fffffff) return PKR_EINVAL;
    double tau = p->tau_lb;
    if (!(tau > 0.0) && pkr_tau_from_knudsen(p->lattice, p->knudsen, p->n, &tau) != PKR_OK)
        return PKR_EINVAL;
    if (!(tau > 0.5) || !std::isfinite(tau)) return PKR_EINVAL;
    if (unstable(li, 1.0 / tau)) return PKR_EUNSTABLE;
    const double eps = p->epsilon == 0.0 ? 1.0 : p->epsilon;
    const int nx = (int)p->n[0], ny = (int)p->n[1], nz = (int)p->n[2];
    cudaStream_t s = (cudaStream_t)stream;

    // one representative per +-v pair
    FftCoefs c{};
    c.omega = 1.0 / tau;
    std::vector<bool> used(li.Q, false);
    for (int i = 0; i < li.Q; ++i) {
        if (used[i]) continue;
        const int* v = &li.vel[3 * i];
        int partner = -1;
        for (int j = 0; j < li.Q; ++j)
            if (li.vel[3 * j] == -v[0] && li.vel[3 * j + 1] == -v[1] && li.vel[3 * j + 2] == -v[2])
                partner = j;
        if (partner < 0 || c.npairs >= kMaxPairs) return PKR_EINVAL;
        used[i] = used[partner] = true;
        c.vx[c.npairs] = v[0];
        c.vy[c.npairs] = v[1];
        c.vz[c.npairs] = v[2];
        c.phi[c.npairs] = li.phi[i];
        c.chi[c.npairs] = li.chi[i];
        c.mult[c.npairs] = (partner == i) ? 1.0 : 2.0;
        c.npairs += 1;
    }

    const int nxh = nx / 2 + 1;
    const size_t nspec = (size_t)nxh * ny * nz;
    double* d_r = nullptr;              // source, then Phi
    cufftDoubleComplex* d_k = nullptr;  // half spectrum (first holds host rho: 16 nspec >= 8 V)
    double* d_mean = nullptr;
    double* d_part = nullptr;
    int* d_flag = nullptr;
    double2* d_h = nullptr;             // half-angle phase tables of x, y, z
    const int red_blocks = 152 * 4;
    if (cudaMalloc((void**)&d_r, (size_t)V * 8) != cudaSuccess ||
        cudaMalloc((void**)&d_k, nspec * sizeof(cufftDoubleComplex)) != cudaSuccess ||
        cudaMalloc((void**)&d_mean, 8) != cudaSuccess ||
        cudaMalloc((void**)&d_part, red_blocks * 8) != cudaSuccess ||
        cudaMalloc((void**)&d_flag, sizeof(int)) != cudaSuccess ||
        cudaMalloc((void**)&d_h, (size_t)(nx + ny + nz) * sizeof(double2)) != cudaSuccess) {
        cudaFree(d_h);
        cudaFree(d_r);
        cudaFree(d_k);
        cudaFree(d_mean);
        cudaFree(d_part);
        cudaFree(d_flag);
        cudaGetLastError();
        return PKR_ENOMEM;
    }
    cufftHandle fwd = 0, inv = 0;
    bool ok = true;
    int flag = 0;
    double mean = 0.0;
    const auto t0 = std::chrono::steady_clock::now();
    {
        const double* rd = rho;
        if (host_buffers) {
            ok = cudaMemcpyAsync(d_k, rho, (size_t)V * 8, cudaMemcpyHostToDevice, s) == cudaSuccess;
            rd = reinterpret_cast<const double*>(d_k);
        }
        // S = (rho - <rho>) c_s^2 (tau_lb - 1/2) / eps, into d_r
        ok = ok && cudaMemsetAsync(d_flag, 0, sizeof(int), s) == cudaSuccess &&
             launch_rho_partials(rd, V, d_part, red_blocks, d_flag, s) == 0 &&
             launch_finalize_mean(d_part, red_blocks, V, d_mean, s) == 0 &&
             launch_make_source(rd, d_mean, li.cs2 * (tau - 0.5) / eps, V, d_r, PKR_FP64, s) == 0 &&
             cudaMemcpyAsync(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
             cudaMemcpyAsync(&mean, d_mean, sizeof(double), cudaMemcpyDeviceToHost, s) ==
                 cudaSuccess &&
             cudaStreamSynchronize(s) == cudaSuccess;
        ok = ok && !flag;   // a non-finite rho stops here, before phi is written
        if (ok) {
            int n3[3] = {nz, ny, nx};
            const int rank = p->dim;
            int* dims = n3 + (3 - rank);
            ok = cufftPlanMany(&fwd, rank, dims, nullptr, 1, 0, nullptr, 1, 0, CUFFT_D2Z, 1) ==
                     CUFFT_SUCCESS &&
                 cufftPlanMany(&inv, rank, dims, nullptr, 1, 0, nullptr, 1, 0, CUFFT_Z2D, 1) ==
                     CUFFT_SUCCESS &&
                 cufftSetStream(fwd, s) == CUFFT_SUCCESS && cufftSetStream(inv, s) == CUFFT_SUCCESS;
        }
        ok = ok && cufftExecD2Z(fwd, d_r, d_k) == CUFFT_SUCCESS;
        if (ok) {
            int blocks = (int)((nspec + 255) / 256);
            if (blocks > 152 * 16) blocks = 152 * 16;
            half_phase_kernel<<<(nx + 255) / 256, 256, 0, s>>>(d_h, nx);
            half_phase_kernel<<<(ny + 255) / 256, 256, 0, s>>>(d_h + nx, ny);
            half_phase_kernel<<<(nz + 255) / 256, 256, 0, s>>>(d_h + nx + ny, nz);
            transfer_kernel<<<blocks, 256, 0, s>>>(d_k, nx, ny, nz, c, d_h, d_h + nx,
                                                  d_h + nx + ny);
            ok = cudaGetLastError() == cudaSuccess;
        }
        ok = ok && cufftExecZ2D(inv, d_k, d_r) == CUFFT_SUCCESS;
        if (ok) {
            scale_kernel<<<152 * 16, 256, 0, s>>>(d_r, V, 1.0 / (double)V);
            ok = cudaGetLastError() == cudaSuccess;
        }
        ok = ok && cudaMemcpyAsync(phi, d_r, (size_t)V * 8,
                                   host_buffers ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                                   s) == cudaSuccess &&
             cudaStreamSynchronize(s) == cudaSuccess;
    }
    const double ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (fwd) cufftDestroy(fwd);
    if (inv) cufftDestroy(inv);
    cudaFree(d_r);
    cudaFree(d_k);
    cudaFree(d_mean);
    cudaFree(d_part);
    cudaFree(d_flag);
    cudaFree(d_h);
    if (flag) return PKR_EINVAL;
    if (!ok) return PKR_ECUDA;
    if (st) {
        std::memset(st, 0, sizeof(*st));
        st->rho_mean_removed = mean;
        st->tau_lb = tau;
        st->cs2 = li.cs2;
        st->wall_ms = ms;
        st->residual = 0.0;
        st->variant = -1;
    }
    return PKR_OK;
}
