"""Oracle lattice tables: velocity sets, quadrature weights, c_s^2 and the
higher-order equilibrium / source weights phi_i, chi_i.

TEST INFRASTRUCTURE ONLY.  This module belongs to the oracle: a plain, slow,
obviously correct statement of the method used to check the CUDA path.  Only
the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of the
benchmark may import it.  It shares no code with the product library.

Everything here is computed in 60-digit ``decimal`` arithmetic and only rounded
to binary64 at the very end, so the tables are correctly rounded.

Sources (Mendoza, Succi, Herrmann, "High-Order Kinetic Relaxation Schemes as
High-Accuracy Poisson Solvers"):
  * 1D velocity sets and weights: Appendix "Quadrature of the Boltzmann
    Equation", N=3 set (D1Q5), N=5 set (D1Q9), N=7 set (D1Q13).  c_s^2 is
    defined there as sum_i w_i v_i^2; it is computed from the printed weights
    (the printed "c_s^2" of the N=5 and N=7 sets equals c_s, not c_s^2).
  * 3D velocity set D3Q111: Appendix, Table "vector2" (10 shells, 111
    vectors).  The printed weights carry only 8-9 digits, so they are
    re-derived here from the 3D quadrature condition (Eq. quad3): the
    degree <= 8 cubic-invariant moments of the discrete set must equal those
    of the Gaussian weight w(v) with variance c_s^2.  11 equations, 10 shell
    weights + c_s^2 as unknowns, Newton's method started from the printed
    digits.
  * 2D sets: the paper says the extension is straightforward (Sec. "Kinetic
    approach to the Poisson equation") but prints none; a 2D set is the
    tensor product of a 1D set with itself (w_ab = w_a w_b, same c_s^2).
  * D3Q19: the standard first-order lattice-Boltzmann set (weights 1/3, 1/18,
    1/36, c_s^2 = 1/3), the comparator the paper calls standard LB.
  * phi_i and chi_i: the truncated Hermite expansions of Sec. "Kinetic
    approach to the Poisson equation" -- Eqs. omega:eq / chi:eq (1D, N=7) and
    Eqs. omega:eq3 / chi:eq3 (3D, N=5) -- written with the isotropic
    contracted Hermite polynomials of dimension D so that one formula covers
    every lattice and order N in {1, 3, 5, 7}.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass
from decimal import Decimal, getcontext

import numpy as np

getcontext().prec = 60

# --------------------------------------------------------------------------
# 1D quadratures as printed in the Appendix.  Tuples of (velocity, weight
# string); the weight strings are the paper's digits.
# --------------------------------------------------------------------------
_D1Q5 = [
    (0, "0.6366469031260781628443461"),
    (1, "0.18141458774368577505004149"),
    (-1, "0.18141458774368577505004149"),
    (3, "0.0002619606932751435277854615"),
    (-3, "0.0002619606932751435277854615"),
]
_D1Q9 = [
    (0, "0.45813515550767658573"),
    (1, "0.23734280857794043891"),
    (-1, "0.23734280857794043891"),
    (2, "0.032324653788654934092"),
    (-2, "0.032324653788654934092"),
    (3, "0.0012640621515365148385"),
    (-3, "0.0012640621515365148385"),
    (5, "8.977280298192933351E-7"),
    (-5, "8.977280298192933351E-7"),
]
_D1Q13 = [
    (0, "0.3455934552621565"),
    (1, "0.2374599218260301"),
    (-1, "0.2374599218260301"),
    (2, "0.07705730993964580"),
    (-2, "0.07705730993964580"),
    (3, "0.011801423732312036"),
    (-3, "0.011801423732312036"),
    (4, "0.0008552466009513439"),
    (-4, "0.0008552466009513439"),
    (5, "0.00002884934614927074"),
    (-5, "0.00002884934614927074"),
    (6, "5.209238332209471E-7"),
    (-6, "5.209238332209471E-7"),
]

# D3Q111 shells (Table vector2): representative vector and the weight printed
# in the paper (8-9 digits; used as Newton start and as a test pin).
D3Q111_SHELLS = [
    ((0, 0, 0), "0.15014405"),
    ((1, 0, 0), "0.02500399"),
    ((1, 1, 0), "0.04505812"),
    ((3, 3, 3), "7.81706951E-7"),
    ((3, 3, 0), "9.79290909E-6"),
    ((3, 1, 0), "1.81207346E-4"),
    ((2, 2, 0), "6.03109965E-4"),
    ((2, 1, 1), "3.49417975E-3"),
    ((2, 0, 0), "1.05490305E-2"),
    ((3, 0, 0), "4.50016852E-5"),
]

# Degree <= 8 monomials x^a y^b z^c (a >= b >= c, all even) that span the
# cubic-invariant moments a 3D set must reproduce (Eq. quad3 up to order 8).
_CUBIC_MONOMIALS = [
    (0, 0, 0), (2, 0, 0), (4, 0, 0), (2, 2, 0), (6, 0, 0), (4, 2, 0),
    (2, 2, 2), (8, 0, 0), (6, 2, 0), (4, 4, 0), (4, 2, 2),
]


def _double_factorial(n: int) -> int:
    r = 1
    while n > 1:
        r *= n
        n -= 2
    return r


def gaussian_moment(exponents, cs2):
    """<v_x^a v_y^b ...> of the Gaussian w(v) with variance cs2 per axis."""
    out = Decimal(1) if isinstance(cs2, Decimal) else 1.0
    for a in exponents:
        if a % 2:
            return 0 * out
        out = out * _double_factorial(a - 1) * cs2 ** (a // 2)
    return out


def shell_vectors(rep):
    """All sign changes and permutations of a representative vector."""
    out = set()
    for p in itertools.permutations(rep):
        for s in itertools.product((1, -1), repeat=len(rep)):
            out.add(tuple(a * b for a, b in zip(p, s)))
    return sorted(out)


def _solve_dense(M, b):
    """Gaussian elimination with partial pivoting in Decimal."""
    n = len(M)
    A = [list(row) + [bb] for row, bb in zip(M, b)]
    for c in range(n):
        p = max(range(c, n), key=lambda r: abs(A[r][c]))
        A[c], A[p] = A[p], A[c]
        if A[c][c] == 0:
            raise ZeroDivisionError("singular system")
        for r in range(c + 1, n):
            f = A[r][c] / A[c][c]
            if f:
                A[r] = [x - f * y for x, y in zip(A[r], A[c])]
    x = [Decimal(0)] * n
    for r in range(n - 1, -1, -1):
        s = A[r][n] - sum(A[r][j] * x[j] for j in range(r + 1, n))
        x[r] = s / A[r][r]
    return x


def derive_d3q111():
    """Solve Eq. quad3 (orders <= 8) for the D3Q111 shell weights and c_s^2.

    Unknowns u = (w_1..w_10, c_s^2).  Residuals
        F_m(u) = sum_s w_s M_{s,m} - <x^a y^b z^c>_Gauss(c_s^2)
    for the 11 monomials m.  Newton's method from the printed digits and
    c_s^2 = 0.7 converges quadratically.  Returns (weights, cs2) as Decimals.
    """
    shells = [shell_vectors(rep) for rep, _ in D3Q111_SHELLS]
    Msm = [[sum(v[0] ** a * v[1] ** b * v[2] ** c for v in sh) for sh in shells]
           for (a, b, c) in _CUBIC_MONOMIALS]
    u = [Decimal(ws) for _, ws in D3Q111_SHELLS] + [Decimal("0.7")]
    for _ in range(100):
        w, t = u[:10], u[10]
        F = [sum(Decimal(Msm[m][s]) * w[s] for s in range(10))
             - gaussian_moment(mon, t) for m, mon in enumerate(_CUBIC_MONOMIALS)]
        # d/dt of the Gaussian moment t^k * C is k t^(k-1) C
        J = []
        for m, mon in enumerate(_CUBIC_MONOMIALS):
            k = sum(mon) // 2
            dg = k * gaussian_moment(mon, t) / t if k else Decimal(0)
            J.append([Decimal(Msm[m][s]) for s in range(10)] + [-dg])
        du = _solve_dense(J, [-f for f in F])
        u = [a + d for a, d in zip(u, du)]
        if max(abs(d) for d in du) < Decimal("1e-55"):
            break
    else:  # pragma: no cover - would mean the system has no nearby root
        raise RuntimeError("D3Q111 Newton iteration did not converge")
    return u[:10], u[10]


@dataclass
class Lattice:
    """A discrete velocity set with its equilibrium and source weights."""

    name: str
    dim: int
    order: int
    vel: np.ndarray          # (Q, 3) int
    w: np.ndarray            # (Q,) float64 quadrature weights
    cs2: float               # c_s^2 = sum_i w_i v_ix^2
    phi: np.ndarray          # (Q,) float64 equilibrium weights phi_i
    chi: np.ndarray          # (Q,) float64 source weights chi_i
    w_dec: list              # Decimal weights (for moment tests)
    cs2_dec: Decimal

    @property
    def Q(self) -> int:
        return len(self.w)

    @property
    def reach(self) -> int:
        return int(np.abs(self.vel).max())


MAX_ORDER = {"D1Q5": 3, "D1Q9": 5, "D1Q13": 7, "D2Q25": 3, "D2Q81": 5,
             "D2Q169": 7, "D3Q19": 3, "D3Q111": 5}
LATTICES = list(MAX_ORDER)


def _raw_set(name):
    """(velocities as 3-tuples, Decimal weights, Decimal cs2, dim)."""
    if name in ("D1Q5", "D1Q9", "D1Q13", "D2Q25", "D2Q81", "D2Q169"):
        base = {"D1Q5": _D1Q5, "D2Q25": _D1Q5, "D1Q9": _D1Q9, "D2Q81": _D1Q9,
                "D1Q13": _D1Q13, "D2Q169": _D1Q13}[name]
        vs = [v for v, _ in base]
        ws = [Decimal(s) for _, s in base]
        cs2 = sum(w * v * v for v, w in zip(vs, ws))  # Appendix: c_s^2 = sum w v^2
        if name.startswith("D1"):
            return [(v, 0, 0) for v in vs], ws, cs2, 1
        vel, wt = [], []
        for (va, wa), (vb, wb) in itertools.product(zip(vs, ws), zip(vs, ws)):
            vel.append((va, vb, 0))
            wt.append(wa * wb)
        return vel, wt, cs2, 2
    if name == "D3Q19":
        vel, wt = [], []
        for rep, w in (((0, 0, 0), Decimal(1) / 3), ((1, 0, 0), Decimal(1) / 18),
                       ((1, 1, 0), Decimal(1) / 36)):
            for v in shell_vectors(rep):
                vel.append(v)
                wt.append(w)
        return vel, wt, Decimal(1) / 3, 3
    if name == "D3Q111":
        wsh, cs2 = derive_d3q111()
        vel, wt = [], []
        for (rep, _), w in zip(D3Q111_SHELLS, wsh):
            for v in shell_vectors(rep):
                vel.append(v)
                wt.append(w)
        return vel, wt, cs2, 3
    raise KeyError(name)


def hermite_weights(xi2, dim, order):
    """phi_i/w_i and chi_i/w_i for squared reduced speed xi2 = |v|^2/c_s^2.

    Isotropic contracted Hermite polynomials in dimension D:
        H2 = xi^2 - D
        H4 = xi^4 - 2(D+2) xi^2 + D(D+2)
        H6 = xi^6 - 3(D+4) xi^4 + 3(D+2)(D+4) xi^2 - D(D+2)(D+4)
    Equilibrium (Eq. omega:eq for D=1, N=7; Eq. omega:eq3 for D=3, N=5):
        phi/w = 1                          (N <= 3)
              = 1 - H4/8                   (N = 5)
              = 1 - H4/8 + H6/24           (N = 7)
    Source (Eq. chi:eq for D=1, N=7; Eq. chi:eq3 for D=3, N=5):
        chi/w = 1                          (N = 1)
              = 1 - H2/2                   (N = 3)
              = 1 - H2/2 + H4/8            (N = 5)
              = 1 - H2/2 + H4/8 - H6/48    (N = 7)
    """
    D = dim
    H2 = xi2 - D
    H4 = xi2 * xi2 - 2 * (D + 2) * xi2 + D * (D + 2)
    H6 = (xi2 ** 3 - 3 * (D + 4) * xi2 * xi2 + 3 * (D + 2) * (D + 4) * xi2
          - D * (D + 2) * (D + 4))
    one = xi2 * 0 + 1
    phi = one
    if order >= 5:
        phi = phi - H4 / 8
    if order >= 7:
        phi = phi + H6 / 24
    chi = one
    if order >= 3:
        chi = chi - H2 / 2
    if order >= 5:
        chi = chi + H4 / 8
    if order >= 7:
        chi = chi - H6 / 48
    return phi, chi


_CACHE: dict = {}


def lattice(name: str, order: int) -> Lattice:
    """Build (and cache) a lattice with its phi_i, chi_i for expansion order N."""
    if name not in MAX_ORDER:
        raise KeyError(f"unknown lattice {name}")
    if order not in (1, 3, 5, 7) or order > MAX_ORDER[name]:
        raise ValueError(f"order {order} not supported on {name}")
    key = (name, order)
    if key in _CACHE:
        return _CACHE[key]
    vel, wdec, cs2, dim = _raw_set(name)
    phi, chi = [], []
    for v, w in zip(vel, wdec):
        xi2 = Decimal(v[0] ** 2 + v[1] ** 2 + v[2] ** 2) / cs2
        a, b = hermite_weights(xi2, dim, order)
        phi.append(float(w * a))
        chi.append(float(w * b))
    lat = Lattice(name=name, dim=dim, order=order,
                  vel=np.array(vel, dtype=np.int64),
                  w=np.array([float(w) for w in wdec]),
                  cs2=float(cs2), phi=np.array(phi), chi=np.array(chi),
                  w_dec=wdec, cs2_dec=cs2)
    _CACHE[key] = lat
    return lat
