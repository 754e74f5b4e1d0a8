// pkr_lattice.cpp -- host-side lattice tables of the product library:
// quadrature weights, c_s^2, the order-N equilibrium and source weights
// phi_i, chi_i, a moment self-check and the small-tau stability pre-check.
#include "pkr_internal.h"

#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

namespace pkr {
namespace {

// Weights of the paper's 1D quadratures by |v| (Appendix): N = 3 set, N = 5
// set and N = 7 set, as printed.
const long double kW5[4] = {0.6366469031260781628443461L, 0.18141458774368577505004149L, 0.0L,
                            0.0002619606932751435277854615L};
const long double kW9[6] = {0.45813515550767658573L, 0.23734280857794043891L,
                            0.032324653788654934092L, 0.0012640621515365148385L, 0.0L,
                            8.977280298192933351e-7L};
const long double kW13[7] = {0.3455934552621565L,    0.2374599218260301L,
                             0.07705730993964580L,   0.011801423732312036L,
                             0.0008552466009513439L, 0.00002884934614927074L,
                             5.209238332209471e-7L};

// D3Q111 (Table "vector2"): the printed weights carry 8-9 digits, so the
// library uses the exact solution of the 3D quadrature condition (Eq. quad3)
// through degree 8 -- 11 cubic-invariant moment equations for the 10 shell
// weights and c_s^2 -- evaluated to 25 digits.  The self-check below
// verifies the moment equations at start-up.
struct Shell {
    int key;
    long double w;
};
const Shell kShellW111[10] = {
    {0x000, 0.1501440521132679892807733L},   {0x100, 0.0250039884070412273298494L},
    {0x110, 0.04505812049781918143471641L},  {0x333, 7.817069506635642121453264e-7L},
    {0x330, 9.792909088441142878716089e-6L}, {0x310, 1.812073460862837756734646e-4L},
    {0x220, 6.031099650419177085026658e-4L}, {0x211, 3.494179755520203150182236e-3L},
    {0x200, 1.054903046257696824624415e-2L}, {0x300, 4.500168524455984920966311e-5L},
};
const long double kCs2_111 = 0.697953322019683088238409055389L;

long double w1d(int lat, int a)
{
    a = a < 0 ? -a : a;
    switch (lat) {
    case PKR_D1Q5: case PKR_D2Q25: return a <= 3 ? kW5[a] : 0.0L;
    case PKR_D1Q9: case PKR_D2Q81: return a <= 5 ? kW9[a] : 0.0L;
    default: return a <= 6 ? kW13[a] : 0.0L;
    }
}

template <class L>
void copy_vel(LatticeInfo& li)
{
    li.Q = L::Q;
    li.dim = L::DIM;
    li.reach = L::T.reach;
    li.ncls = L::T.ncls;
    for (int i = 0; i < L::Q; ++i) {
        li.vel[3 * i + 0] = L::T.v[i].x;
        li.vel[3 * i + 1] = L::T.v[i].y;
        li.vel[3 * i + 2] = L::T.v[i].z;
        li.cls[i] = L::T.cls[i];
        li.key[i] = L::T.key[i];
    }
}

int max_order(int lat)
{
    switch (lat) {
    case PKR_D1Q5: case PKR_D2Q25: case PKR_D3Q19: return 3;
    case PKR_D1Q9: case PKR_D2Q81: case PKR_D3Q111: return 5;
    case PKR_D1Q13: case PKR_D2Q169: return 7;
    default: return 0;
    }
}

// Gaussian moment <x^a y^b z^c> with variance cs2 per axis.
long double gmom(int a, int b, int c, long double cs2)
{
    long double r = 1.0L;
    const int e[3] = {a, b, c};
    for (int k = 0; k < 3; ++k) {
        if (e[k] & 1) return 0.0L;
        for (int j = e[k] - 1; j > 1; j -= 2) r *= j;
        for (int j = 0; j < e[k] / 2; ++j) r *= cs2;
    }
    return r;
}

// Moment self-check: the weights reproduce the Gaussian moments through the
// degree the Hermite terms of the highest order need (4 for the D3Q19 set).
bool self_check(const LatticeInfo& li)
{
    const int deg = (li.lattice == PKR_D3Q19) ? 4 : (li.lattice == PKR_D1Q5 || li.lattice == PKR_D2Q25) ? 6 : 8;
    for (int a = 0; a <= deg; a += 2)
        for (int b = 0; a + b <= deg; b += 2)
            for (int c = 0; a + b + c <= deg; c += 2) {
                if (li.dim < 2 && b) continue;
                if (li.dim < 3 && c) continue;
                long double s = 0, mag = 0;
                for (int i = 0; i < li.Q; ++i) {
                    long double t = li.wl[i];
                    for (int k = 0; k < a; ++k) t *= li.vel[3 * i];
                    for (int k = 0; k < b; ++k) t *= li.vel[3 * i + 1];
                    for (int k = 0; k < c; ++k) t *= li.vel[3 * i + 2];
                    s += t;
                    mag += fabsl(t);
                }
                long double want = gmom(a, b, c, li.cs2l);
                if (fabsl(s - want) > 1e-14L * (mag > 1 ? mag : 1)) return false;
            }
    return true;
}

std::mutex g_mu;
std::map<std::pair<int, int>, LatticeInfo> g_cache;

}  // namespace

int build_lattice(int lat, int order, LatticeInfo* out)
{
    if (lat < PKR_D1Q5 || lat > PKR_D3Q111) return PKR_EINVAL;
    if (!(order == 1 || order == 3 || order == 5 || order == 7) || order > max_order(lat))
        return PKR_EINVAL;
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_cache.find({lat, order});
    if (it != g_cache.end()) {
        *out = it->second;
        return PKR_OK;
    }
    LatticeInfo li{};
    li.lattice = lat;
    li.order = order;
    switch (lat) {
    case PKR_D1Q5: copy_vel<D1Q5>(li); break;
    case PKR_D1Q9: copy_vel<D1Q9>(li); break;
    case PKR_D1Q13: copy_vel<D1Q13>(li); break;
    case PKR_D2Q25: copy_vel<D2Q25>(li); break;
    case PKR_D2Q81: copy_vel<D2Q81>(li); break;
    case PKR_D2Q169: copy_vel<D2Q169>(li); break;
    case PKR_D3Q19: copy_vel<D3Q19>(li); break;
    case PKR_D3Q111: copy_vel<D3Q111>(li); break;
    }
    // quadrature weights
    for (int i = 0; i < li.Q; ++i) {
        const int* v = &li.vel[3 * i];
        long double w = 0;
        if (lat <= PKR_D1Q13) {
            w = w1d(lat, v[0]);
        } else if (lat <= PKR_D2Q169) {
            w = w1d(lat, v[0]) * w1d(lat, v[1]);
        } else if (lat == PKR_D3Q19) {
            int k = li.key[i];
            w = (k == 0) ? 1.0L / 3 : (k == 0x100) ? 1.0L / 18 : 1.0L / 36;
        } else {
            for (const Shell& s : kShellW111)
                if (s.key == li.key[i]) w = s.w;
        }
        li.wl[i] = w;
        li.w[i] = (double)w;
    }
    // c_s^2 = sum_i w_i v_ix^2 (Appendix); fixed for the 3D sets
    if (lat == PKR_D3Q19) {
        li.cs2l = 1.0L / 3;
    } else if (lat == PKR_D3Q111) {
        li.cs2l = kCs2_111;
    } else {
        long double s = 0;
        for (int i = 0; i < li.Q; ++i) s += li.wl[i] * li.vel[3 * i] * li.vel[3 * i];
        li.cs2l = s;
    }
    li.cs2 = (double)li.cs2l;
    if (!self_check(li)) return PKR_EINVAL;
    // equilibrium and source weights: isotropic Hermite expansion, dimension D
    const long double D = li.dim;
    for (int i = 0; i < li.Q; ++i) {
        const int* v = &li.vel[3 * i];
        long double xi2 = (long double)(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) / li.cs2l;
        long double H2 = xi2 - D;
        long double H4 = xi2 * xi2 - 2 * (D + 2) * xi2 + D * (D + 2);
        long double H6 = xi2 * xi2 * xi2 - 3 * (D + 4) * xi2 * xi2 + 3 * (D + 2) * (D + 4) * xi2 -
                         D * (D + 2) * (D + 4);
        long double ph = 1, ch = 1;
        if (order >= 5) ph -= H4 / 8;
        if (order >= 7) ph += H6 / 24;
        if (order >= 3) ch -= H2 / 2;
        if (order >= 5) ch += H4 / 8;
        if (order >= 7) ch -= H6 / 48;
        li.phi[i] = (double)(li.wl[i] * ph);
        li.chi[i] = (double)(li.wl[i] * ch);
        li.cls_phi[li.cls[i]] = li.phi[i];
        li.cls_chi[li.cls[i]] = li.chi[i];
    }
    g_cache[{lat, order}] = li;
    *out = li;
    return PKR_OK;
}

// Stability pre-check for over-relaxation (omega > 1).  Each Fourier mode k
// evolves by M(k) = E(k) [(1-omega) I + omega phi 1^T], E = diag(exp(-i k.v)).
// Its eigenvalues off the circle |lambda| = |1-omega| solve
//     F(lambda) = 1 - omega sum_i phi_i e_i / (lambda - (1-omega) e_i) = 0,
// and F is analytic outside |lambda| = |1-omega| < 1 with F(inf) = 1, so the
// number of eigenvalues with |lambda| > 1 is minus the winding number of
// F(exp(i theta)) about 0.  The check scans k on a (13)^D grid of [0, pi]^D
// (13 points per axis, including every multiple of pi/12).  For omega <= 1 the
// solver relies on the run-time divergence monitor instead.
bool unstable(const LatticeInfo& li, double omega)
{
    if (!(omega > 1.0)) return false;
    const int m = 13;
    const int nth = 1024;
    const int nk = li.dim == 1 ? m : li.dim == 2 ? m * m : m * m * m;
    std::vector<std::complex<double>> e(li.Q);
    for (int kk = 0; kk < nk; ++kk) {
        int a = kk % m, b = (kk / m) % m, c = kk / (m * m);
        if (li.dim >= 2 && b > a) continue;
        if (li.dim >= 3 && c > b) continue;
        if (kk == 0) continue;
        double k[3] = {M_PI * a / (m - 1), M_PI * b / (m - 1), M_PI * c / (m - 1)};
        for (int i = 0; i < li.Q; ++i) {
            double ph = -(k[0] * li.vel[3 * i] + k[1] * li.vel[3 * i + 1] + k[2] * li.vel[3 * i + 2]);
            e[i] = std::complex<double>(cos(ph), sin(ph));
        }
        double total = 0.0;
        std::complex<double> prev;
        for (int t = 0; t <= nth; ++t) {
            double th = 2 * M_PI * t / nth;
            std::complex<double> lam(cos(th), sin(th));
            std::complex<double> s = 0;
            for (int i = 0; i < li.Q; ++i) s += li.phi[i] * e[i] / (lam - (1 - omega) * e[i]);
            std::complex<double> F = 1.0 - omega * s;
            if (t > 0) total += std::arg(F / prev);
            prev = F;
        }
        if (fabs(total) > M_PI) return true;  // non-zero winding number
    }
    return false;
}

}  // namespace pkr
