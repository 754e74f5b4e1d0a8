"""Pins for the oracle's sweep, source preparation and steady state.

The oracle iterates the scheme in real space with plain loops.  These tests
hold it to results obtained by other routes (``pins.py``): per-Fourier-mode
evolution, the closed-form fixed point, a direct sparse solve, the omega = 1
scalar stencil, conservation, the continuum Poisson solution and the paper's
Table 2 errors and convergence orders.
"""
import numpy as np
import pytest

import pins
from conftest import golden
from oracle import lattice, solve, source, step, tau_from_knudsen


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def _rand_source(shape, seed):
    r = np.random.default_rng(seed).standard_normal(shape)
    return r - r.mean()


CASES = [
    ("D1Q5", 3, (23,), 0.9),
    ("D1Q9", 5, (17,), 1.7),
    ("D1Q13", 7, (29,), 1.0),
    ("D2Q25", 1, (7, 9), 0.8),
    ("D2Q81", 5, (6, 11), 1.2),
    ("D2Q169", 7, (9, 10), 6.04398),
    ("D3Q19", 1, (5, 6, 7), 0.75),
    ("D3Q19", 3, (4, 5, 6), 1.1),
    ("D3Q111", 5, (5, 4, 7), 1.0),
    ("D3Q111", 5, (6, 6, 6), 2.5),
]


@pytest.mark.parametrize("name,N,shape,tau", CASES)
def test_steps_match_fourier_evolution(name, N, shape, tau):
    lat = lattice(name, N)
    rho = _rand_source(shape, 1)
    S, _ = source(rho, lat, tau)
    T = 9
    got = solve(rho, name, N, tau_lb=tau, max_steps=T).phi
    want = pins.fourier_steps(S, lat.vel, lat.phi, lat.chi, 1 / tau, T)
    assert _rel(got, want) < 1e-13


def test_single_step_matches_fourier_from_random_state():
    """One step from an arbitrary (non-zero) state, raw source."""
    lat = lattice("D3Q111", 5)
    rng = np.random.default_rng(5)
    shape = (4, 6, 5)
    g = rng.standard_normal((lat.Q,) + shape)
    S = rng.standard_normal(shape)
    omega = 0.7
    g1 = step(g, S, lat, omega)
    # the same step written with numpy rolls (push: g'_i(x + v_i) = p_i(x))
    Phi = g.sum(axis=0)
    want = np.empty_like(g)
    for i, v in enumerate(lat.vel):
        p = (1 - omega) * g[i] + omega * lat.phi[i] * Phi + lat.chi[i] * S
        want[i] = np.roll(p, shift=(v[2], v[1], v[0]), axis=(0, 1, 2))
    assert np.max(np.abs(g1 - want)) < 1e-14


@pytest.mark.parametrize("name,N,shape,tau", [
    ("D1Q13", 7, (24,), 1.0),
    ("D2Q169", 7, (12, 12), 1.0),
    ("D2Q81", 5, (10, 8), 3.0),
    ("D3Q19", 1, (8, 8, 8), 1.0),
    ("D3Q111", 5, (8, 6, 8), 1.3),
])
def test_converged_state_is_closed_form_fixed_point(name, N, shape, tau):
    lat = lattice(name, N)
    rho = _rand_source(shape, 2)
    S, _ = source(rho, lat, tau)
    r = solve(rho, name, N, tau_lb=tau, tol=1e-15, tol_kind=0, max_steps=200000)
    want = pins.fixed_point(S, lat.vel, lat.phi, lat.chi, 1 / tau)
    assert _rel(r.phi, want) < 1e-10
    assert abs(r.phi.mean()) < 1e-13 * np.abs(r.phi).max()


@pytest.mark.parametrize("name,N,shape,tau", [
    ("D2Q25", 3, (6, 5), 1.0),
    ("D3Q19", 1, (4, 4, 5), 0.9),
    ("D2Q81", 5, (5, 6), 1.4),
])
def test_dense_solve_matches_closed_form_and_oracle(name, N, shape, tau):
    lat = lattice(name, N)
    rho = _rand_source(shape, 3)
    S, _ = source(rho, lat, tau)
    dense = pins.dense_fixed_point(S, lat.vel, lat.phi, lat.chi, 1 / tau)
    closed = pins.fixed_point(S, lat.vel, lat.phi, lat.chi, 1 / tau)
    assert _rel(closed, dense) < 1e-11
    r = solve(rho, name, N, tau_lb=tau, tol=1e-15, tol_kind=0, max_steps=200000)
    assert _rel(r.phi, dense) < 1e-10


@pytest.mark.slow
def test_dense_solve_d3q111_4cubed():
    lat = lattice("D3Q111", 5)
    rho = _rand_source((4, 4, 4), 4)
    S, _ = source(rho, lat, 1.0)
    dense = pins.dense_fixed_point(S, lat.vel, lat.phi, lat.chi, 1.0)
    r = solve(rho, "D3Q111", 5, tau_lb=1.0, tol=1e-15, tol_kind=0, max_steps=100000)
    assert _rel(r.phi, dense) < 1e-10


def test_conservation_with_non_neutral_source():
    """sum_phi = sum_chi = 1, so every step adds sum_x S to sum_x Phi."""
    lat = lattice("D2Q81", 5)
    rng = np.random.default_rng(6)
    shape = (7, 9)
    S = rng.random(shape) + 0.5  # not mean-free, used as the raw source
    for T in (1, 5, 12):
        r = solve(S, "D2Q81", 5, tau_lb=1.3, max_steps=T, S=S)
        assert abs(r.phi.sum() - T * S.sum()) < 1e-12 * T * S.sum()


def test_omega_one_is_scalar_stencil():
    lat = lattice("D3Q111", 5)
    rho = _rand_source((6, 5, 7), 7)
    S, _ = source(rho, lat, 1.0)
    T = 6
    got = solve(rho, "D3Q111", 5, tau_lb=1.0, max_steps=T).phi
    want = pins.stencil_omega1(S, lat.vel, lat.phi, lat.chi, T)
    assert _rel(got, want) < 1e-13


def test_source_prep():
    lat = lattice("D3Q111", 5)
    rho = np.random.default_rng(8).random((5, 6, 7)) + 3.0
    S, mean = source(rho, lat, 2.0, eps=0.5)
    assert abs(mean - rho.mean()) < 1e-14
    want = (rho - rho.mean()) * lat.cs2 * 1.5 / 0.5
    assert np.max(np.abs(S - want)) < 1e-14


def _table2_error(name, N, L):
    x = np.arange(L)
    k = 2 * np.pi / L
    rho = np.sin(k * x)
    r = solve(rho, name, N, tau_lb=1.0, tol=1e-15, tol_kind=1, max_steps=10 ** 7)
    exact = rho / k ** 2
    return float(np.abs(r.phi - exact).max() / np.abs(exact).max())


LAT_FOR_N = {1: "D1Q5", 3: "D1Q5", 5: "D1Q9", 7: "D1Q13"}


def test_table2_per_node_errors():
    """Errors of the converged 1D solution (tau_lb = 1, l = 1) against the
    analytic Poisson solution agree with the paper's Table 2 (printed to one
    digit) within a factor 1.45."""
    for L, N, printed in golden("table2_per_node_error.txt"):
        L, N, printed = int(L), int(N), float(printed)
        err = _table2_error(LAT_FOR_N[N], N, L)
        assert 0.7 < err / printed < 1.45, (L, N, err, printed)


def test_convergence_orders():
    """Per-node error falls as L^-2, L^-4, L^-6 for N = 3, 5, 7 (one more
    than Table 1's alpha_N, see the discussion of Table 2)."""
    for N, order in ((3, 2), (5, 4), (7, 6)):
        e16 = _table2_error(LAT_FOR_N[N], N, 16)
        e32 = _table2_error(LAT_FOR_N[N], N, 32)
        e64 = _table2_error(LAT_FOR_N[N], N, 64)
        assert abs(np.log2(e32 / e64) - order) < 0.15, N
        assert abs(np.log2(e16 / e32) - order) < 0.6, N


def test_fig1_errors_at_L128():
    """Sec. "Numerical Results", Fig. 1 (L = 128, l = 1): about 0.02 % for
    N = 1, 3 and below 1e-3 % for N = 5, 7."""
    e1 = _table2_error("D1Q5", 1, 128)
    e3 = _table2_error("D1Q5", 3, 128)
    assert 1e-4 < e1 < 3e-4 and 1e-4 < e3 < 3e-4
    assert _table2_error("D1Q9", 5, 128) < 1e-5
    assert _table2_error("D1Q13", 7, 128) < 1e-5


def test_closed_form_error_single_mode_2d():
    """Config geometry 64x64, rho = sin(2 pi x/64) sin(2 pi y/64), D2Q169 N=7:
    the fixed point is T(k) times the source mode, so its error against the
    analytic rho / (2 k^2) follows from T(k) alone; the oracle reaches it."""
    lat = lattice("D2Q169", 7)
    n = 32
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    k = 2 * np.pi / n
    rho = np.sin(k * x) * np.sin(k * y)
    tau = 1.0
    S, _ = source(rho, lat, tau)
    r = solve(rho, "D2Q169", 7, tau_lb=tau, tol=1e-14, tol_kind=0, max_steps=100000)
    exact = rho / (2 * k * k)
    T = pins.transfer([k, k, 0], lat.vel, lat.phi, lat.chi, 1 / tau)
    # S = rho cs2 (tau_lb - 1/2); analytic amplitude 1/(2k^2)
    amp = np.real(T) * lat.cs2 * (tau - 0.5)
    # sixth-order accurate: 1.6e-5 at n = 32 (2.6e-7 at n = 64)
    assert 1e-5 < abs(amp * 2 * k * k - 1) < 2e-5
    assert _rel(r.phi, amp * rho) < 1e-9
    assert abs(_rel(r.phi, exact) - abs(amp * 2 * k * k - 1)) < 1e-8


def test_gaussian_sources_against_continuum_poisson():
    """Stiff localised sources: the converged N=5 D3Q111 potential is close
    to the continuum periodic Poisson solution, and closer than the N=1
    (standard LB) equilibrium on the same lattice."""
    n = 16
    z, y, x = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    rho = np.zeros((n, n, n))
    for c, q in (((4.0, 5.0, 6.0), 1.0), ((11.0, 10.0, 9.5), -1.0)):
        d2 = sum(np.minimum(np.abs(a - ca), n - np.abs(a - ca)) ** 2
                 for a, ca in zip((x, y, z), c))
        rho += q * np.exp(-d2 / (2 * 2.0 ** 2)) / (2 * np.pi * 4.0) ** 1.5
    ref = pins.spectral_poisson(rho)
    errs = {}
    for N in (1, 5):
        r = solve(rho, "D3Q111", N, tau_lb=1.0, tol=1e-13, tol_kind=1,
                  check_every=10, max_steps=100000)
        errs[N] = _rel(r.phi, ref)
    assert errs[5] < 5e-3          # 3.3e-3 on this 16^3 grid
    assert errs[5] < errs[1] / 5   # N=1: 3.8e-2


def test_knudsen_reading():
    """Kn = lambda / L with lambda = c_s (tau_lb - 1/2) and L the shortest
    edge: 64x64 at Kn 0.1 on the N=7 set gives tau_lb = 6.04398."""
    lat = lattice("D2Q169", 7)
    t = tau_from_knudsen(0.1, (64, 64, 1), lat.cs2)
    assert abs(t - 6.043980) < 1e-5
    assert abs((t - 0.5) * np.sqrt(lat.cs2) / 64 - 0.1) < 1e-15


def test_small_tau_instability():
    """Contrary to the paper's expectation of stability, the N=5 set with
    tau_lb = 0.6 has Fourier modes with spectral radius > 1 (the worst of
    this scan is k = (5, 3, 1) pi/6); the oracle's iteration on a 12^3 grid,
    which carries that mode, grows without bound there and stays bounded at
    tau_lb = 1, where every k != 0 mode decays."""
    lat = lattice("D3Q111", 5)
    axis = np.linspace(0, np.pi, 7)
    ks = [(a, b, c) for a in axis for b in axis for c in axis
          if a >= b >= c and a > 0]

    def radius(tau):
        om = 1 / tau
        C = (1 - om) * np.eye(lat.Q) + om * np.outer(lat.phi, np.ones(lat.Q))
        best = 0.0
        for k in ks:
            e = np.exp(-1j * (lat.vel @ np.array(k)))
            best = max(best, np.abs(np.linalg.eigvals(np.diag(e) @ C)).max())
        return best

    assert radius(0.6) > 1.1
    assert radius(1.0) < 1.0
    rho = _rand_source((12, 12, 12), 9)
    bad = solve(rho, "D3Q111", 5, tau_lb=0.6, max_steps=300)
    good = solve(rho, "D3Q111", 5, tau_lb=1.0, max_steps=300)
    assert np.abs(bad.phi).max() > 1e6 * np.abs(good.phi).max()


def test_openmp_build_is_bitwise_serial():
    """The multi-core baseline build (same source, -fopenmp) gives exactly the
    serial oracle's result: each site's arithmetic is unchanged and every
    push goes to its own address."""
    import oracle
    try:
        n = oracle.threads(3)
    except Exception as e:      # compiler without OpenMP support
        pytest.skip(f"OpenMP build unavailable: {e}")
    assert n == 3
    lat = lattice("D3Q111", 5)
    rho = _rand_source((7, 9, 10), 8)
    S, _ = source(rho, lat, 1.3)
    g = np.random.default_rng(9).standard_normal((lat.Q,) + rho.shape)
    a = step(g, S, lat, 1 / 1.3)
    b = step(g, S, lat, 1 / 1.3, openmp=True)
    assert np.array_equal(a, b)
    r1 = solve(rho, "D3Q111", 5, tau_lb=1.3, max_steps=5)
    r2 = solve(rho, "D3Q111", 5, tau_lb=1.3, max_steps=5, openmp=True)
    assert np.array_equal(r1.phi, r2.phi)


@pytest.mark.parametrize("name,N,shape,tau,kind,every", [
    ("D2Q81", 5, (10, 8), 1.3, 1, 5),
    ("D2Q81", 5, (10, 8), 1.3, 0, 3),
    ("D3Q111", 5, (6, 5, 7), 1.6, 1, 4),
    ("D1Q13", 7, (24,), 0.9, 0, 1),
])
def test_stopping_step_and_residual(name, N, shape, tau, kind, every):
    """The oracle stops at the first check (every ``every`` steps) whose
    change of Phi over one step is below tol, and reports that change:
    max|Phi^t - Phi^(t-1)| (kind 0) or ||Phi^t - Phi^(t-1)||_2 / ||Phi^t||_2
    (kind 1), with Phi^t from the mode-by-mode evolution.  tol is placed
    halfway (geometrically) between two consecutive checks, away from
    rounding; tol <= 0 runs exactly max_steps steps and reports no check."""
    lat = lattice(name, N)
    rho = _rand_source(shape, 9)
    S, _ = source(rho, lat, tau)
    T = 240
    seq = pins.fourier_phi_sequence(S, lat.vel, lat.phi, lat.chi, 1 / tau, T)

    def change(t):                       # change over step t (t >= 2), Phi^1 from 0
        d = seq[t - 1] - seq[t - 2]
        if kind == 0:
            return np.max(np.abs(d))
        return np.linalg.norm(d) / np.linalg.norm(seq[t - 1])

    checks = [t for t in range(every, T + 1, every) if t >= 2]
    r = {t: change(t) for t in checks}
    # the first check three decades below the first one (far above rounding)
    # whose change is below every earlier check's
    t_star = next(t for t in checks[1:]
                  if r[t] < 1e-3 * r[checks[0]] and r[t] < 0.999 * min(r[u] for u in checks
                                                                       if u < t))
    tol = np.sqrt(r[t_star] * min(r[u] for u in checks if u < t_star))
    want_t = next(t for t in checks if r[t] < tol)
    res = solve(rho, name, N, tau_lb=tau, tol=tol, tol_kind=kind, check_every=every,
                max_steps=T)
    assert res.steps == want_t
    assert abs(res.residual - r[want_t]) <= 1e-9 * r[want_t]
    assert _rel(res.phi, seq[want_t - 1]) < 1e-12
    free = solve(rho, name, N, tau_lb=tau, tol=0.0, max_steps=17)
    assert free.steps == 17 and free.residual == -1.0
