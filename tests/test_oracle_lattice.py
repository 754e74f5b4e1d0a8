"""Pins for the oracle's lattice tables (quadratures, c_s^2, phi_i, chi_i).

Every check here compares the oracle's tables with something the paper or the
mathematics fixes: exact Gaussian moments, the paper's printed digits, and the
moment conditions (Eq. CON) that the equilibrium and source weights exist to
satisfy.  A wrong weight, a transposed velocity component, a wrong Hermite
coefficient or the wrong c_s^2 reading fails one of them.
"""
import itertools
from decimal import Decimal
from math import sqrt

import numpy as np
import pytest

from conftest import golden
from oracle import lattice
from oracle.lattice import LATTICES, MAX_ORDER, gaussian_moment

# Degree to which each set integrates the Gaussian weight exactly (the
# Appendix's orthogonality conditions, Eqs. quadrature / quad3).
EXACT_DEGREE = {"D1Q5": 7, "D1Q9": 11, "D1Q13": 13, "D2Q25": 7, "D2Q81": 11,
                "D2Q169": 13, "D3Q19": 5, "D3Q111": 9}


def _moment(lat, exps, wts=None):
    v = lat.vel.astype(float)
    w = lat.w if wts is None else wts
    m = np.ones(len(w))
    for ax, e in enumerate(exps):
        m = m * v[:, ax] ** e
    return float(np.sum(w * m))


def _scale(lat, exps, wts=None):
    """sum |w_i v_i^e|: the size of the terms a moment sums (rounding scale)."""
    v = np.abs(lat.vel.astype(float))
    w = np.abs(lat.w if wts is None else wts)
    m = np.ones(len(w))
    for ax, e in enumerate(exps):
        m = m * v[:, ax] ** e
    return max(1.0, float(np.sum(w * m)))


@pytest.mark.parametrize("name", LATTICES)
def test_quadrature_exact_to_degree(name):
    lat = lattice(name, 1)
    deg = EXACT_DEGREE[name]
    for exps in itertools.product(range(deg + 1), repeat=lat.dim):
        if sum(exps) > deg:
            continue
        e3 = tuple(exps) + (0,) * (3 - lat.dim)
        want = float(gaussian_moment(e3, Decimal(repr(lat.cs2))))
        got = _moment(lat, e3)
        assert abs(got - want) <= 4e-15 * _scale(lat, e3), (name, e3, got, want)


def test_d3q111_not_exact_at_degree_10():
    """The set is a degree-9 rule, not better (x^10 misses by ~3e-2)."""
    lat = lattice("D3Q111", 1)
    want = float(gaussian_moment((10, 0, 0), Decimal(repr(lat.cs2))))
    assert abs(_moment(lat, (10, 0, 0)) - want) > 1e-3


def test_d3q111_counts_and_printed_weights():
    lat = lattice("D3Q111", 5)
    assert lat.Q == 111
    rows = golden("d3q111_table_vector2.txt")
    norms = np.sort(np.abs(lat.vel), axis=1)[:, ::-1]
    for r in rows:
        rep = tuple(int(c) for c in r[:3])
        count, printed = int(r[3]), float(r[4])
        ulp = float(Decimal(1).scaleb(Decimal(r[4]).as_tuple().exponent))
        sel = np.all(norms == rep, axis=1)
        assert sel.sum() == count, rep
        ws = lat.w[sel]
        assert np.all(ws == ws[0])
        # the printed digits agree with the derived weight to their last place
        # (some entries are truncated rather than rounded, e.g. the (2,1,1)
        # shell prints 3.49417975e-3 for 3.4941797555e-3)
        assert abs(ws[0] - printed) <= ulp, (rep, ws[0], printed)


def test_d3q111_cs2_and_moment_residuals_high_precision():
    lat = lattice("D3Q111", 5)
    w = lat.w_dec
    t = lat.cs2_dec
    for exps in [(0, 0, 0), (2, 0, 0), (4, 0, 0), (2, 2, 0), (6, 0, 0),
                 (4, 2, 0), (2, 2, 2), (8, 0, 0), (6, 2, 0), (4, 4, 0),
                 (4, 2, 2)]:
        s = sum(wi * Decimal(int(v[0]) ** exps[0] * int(v[1]) ** exps[1]
                             * int(v[2]) ** exps[2]) for wi, v in zip(w, lat.vel))
        assert abs(s - gaussian_moment(exps, t)) < Decimal("1e-45")
    assert 0.69795332 < lat.cs2 < 0.69795333
    assert all(x > 0 for x in w)


def test_printed_sound_speeds_reading():
    """Appendix: c_s^2 = sum w v^2.  The N=3 line prints c_s^2 itself; the
    N=5 and N=7 lines print a number that is c_s (its square matches)."""
    for name, printed, kind in golden("appendix_sound_speeds.txt"):
        lat = lattice(name, 1)
        val = 1 - sqrt(2 / 5) if printed == "1-sqrt(2/5)" else float(printed)
        if kind == "cs2":
            assert abs(lat.cs2 - val) < 1e-15
        else:
            assert abs(lat.cs2 - val * val) < 1e-15
            # and it is not c_s^2 itself
            assert abs(lat.cs2 - val) > 0.05


def test_step_counts_match_slowest_mode_decay():
    """The paper's L=100 step counts (Sec. "Computational performance")
    correspond to the same number of e-folds of the slowest Fourier mode
    for every N when the tables use c_s^2 = sum w v^2: the higher sound speed
    of the N=5/7 sets is what shortens the run."""
    efolds = []
    for N, name, steps in ((int(r[0]), r[1], int(r[2])) for r in golden("steps_L100.txt")):
        lat = lattice(name, N)
        k = 2 * np.pi / 100
        e = np.exp(-1j * k * lat.vel[:, 0])
        M = np.diag(e) @ np.outer(lat.phi, np.ones(lat.Q))   # tau_lb = 1
        lam = np.abs(np.linalg.eigvals(M)).max()
        efolds.append(steps * -np.log(lam))
    efolds = np.array(efolds)
    assert efolds.max() / efolds.min() < 1.15, efolds
    assert 40 < efolds.mean() < 60


@pytest.mark.parametrize("name", LATTICES)
def test_weights_positive_and_symmetric(name):
    lat = lattice(name, 1)
    assert np.all(lat.w > 0)
    assert abs(lat.w.sum() - 1) < 1e-15
    # every velocity has its opposite with the same weight
    d = {tuple(v): w for v, w in zip(lat.vel, lat.w)}
    for v, w in d.items():
        assert d[tuple(-a for a in v)] == w
    assert len(d) == lat.Q


def _orders(name):
    return [N for N in (1, 3, 5, 7) if N <= MAX_ORDER[name]]


@pytest.mark.parametrize("name,N", [(n, N) for n in LATTICES for N in _orders(n)])
def test_equilibrium_and_source_moments(name, N):
    """Eq. CON: Pi_eq(0) = Phi, Pi_eq(1) = 0, Pi_eq(2) = c_s^2 Phi,
    Pi_eq(n>2) = 0 and S(0) = S, S(n>0) = 0, as far as order N asks
    (the N=7 1D statement after Eq. chi:eq; the N=5 3D statement after
    Eq. chi:eq3).  N = 1 is standard LB: phi = chi = w."""
    lat = lattice(name, N)
    cs2 = lat.cs2
    D = lat.dim
    assert abs(lat.phi.sum() - 1) < 1e-14
    assert abs(lat.chi.sum() - 1) < 1e-14
    if N == 1:
        assert np.array_equal(lat.phi, lat.w) and np.array_equal(lat.chi, lat.w)
    # tensor moments of phi and chi up to degree N + 1 where the condition holds
    for deg in range(1, N + 1 if N > 1 else 3):
        for exps in itertools.product(range(deg + 1), repeat=D):
            if sum(exps) != deg:
                continue
            e3 = tuple(exps) + (0,) * (3 - D)
            mphi = _moment(lat, e3, lat.phi)
            mchi = _moment(lat, e3, lat.chi)
            if deg == 2:
                want = cs2 if max(e3) == 2 else 0.0
                assert abs(mphi - want) < 4e-15 * _scale(lat, e3, lat.phi), (e3, mphi)
            elif deg % 2 == 1 or N >= deg:
                assert abs(mphi) < 4e-15 * _scale(lat, e3, lat.phi), (e3, mphi)
            if N >= 3:
                assert abs(mchi) < 4e-15 * _scale(lat, e3, lat.chi), (e3, mchi)


def test_n1_source_has_second_moment():
    """Standard LB (N=1) keeps the source's second moment: the error term
    the higher-order chi removes."""
    lat = lattice("D1Q5", 1)
    assert abs(_moment(lat, (2, 0, 0), lat.chi) - lat.cs2) < 1e-15
    lat3 = lattice("D1Q5", 3)
    assert abs(_moment(lat3, (2, 0, 0), lat3.chi)) < 1e-15


def test_paper_formulas_1d_n7_and_3d_n5():
    """phi/chi agree with Eqs. omega:eq / chi:eq (1D N=7) and omega:eq3 /
    chi:eq3 (3D N=5) written out in the paper's own variables."""
    lat = lattice("D1Q13", 7)
    c2 = lat.cs2
    for v, w, p, c in zip(lat.vel[:, 0].astype(float), lat.w, lat.phi, lat.chi):
        t4 = (3 * c2 * c2 - 6 * c2 * v * v + v ** 4) / (8 * c2 * c2)
        t6 = (15 * c2 ** 3 - 45 * c2 * c2 * v * v + 15 * c2 * v ** 4 - v ** 6) / (24 * c2 ** 3)
        assert abs(p - w * (1 - t4 - t6)) < 1e-15
        assert abs(c - w * (1 + 0.5 * (1 - v * v / c2) + t4 + t6 / 2)) < 1e-15
    lat = lattice("D3Q111", 5)
    c2 = lat.cs2
    for v, w, p, c in zip(lat.vel.astype(float), lat.w, lat.phi, lat.chi):
        v2 = float(v @ v)
        t4 = (15 * c2 * c2 - 10 * c2 * v2 + v2 * v2) / (8 * c2 * c2)
        assert abs(p - w * (1 - t4)) < 1e-15
        assert abs(c - w * (1 + 0.5 * (3 - v2 / c2) + t4)) < 1e-15


def test_negative_equilibrium_weights():
    """The higher-order phi_i go negative (the source of the small-tau
    instability)."""
    assert lattice("D3Q111", 5).phi.min() < -0.13
    assert lattice("D2Q169", 7).phi.min() < -0.23
    assert lattice("D3Q19", 1).phi.min() > 0
