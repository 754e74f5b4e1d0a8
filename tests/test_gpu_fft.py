"""GPU tests of the FFT comparator (pkr_fixed_point_fft), through the C ABI.

The comparator returns the scheme's exact steady state.  It is checked
against
* the closed-form Sherman-Morrison fixed point of the test pins (numpy FFT,
  itself pinned to the oracle's converged iteration and to a dense direct
  solve on the CPU), element by element, on every lattice, ragged and odd
  sizes, sizes below the lattice reach, 1D/2D/3D;
* a single Fourier mode at the full 256^3 workload geometry, where the
  answer is T(k) S with T(k) evaluated by the pins for that one k;
* the CUDA iteration itself run to a tight tolerance (same kernels as the
  solver; the two must meet at the fixed point).
"""
import numpy as np
import pytest

import oracle
import pins
from paper_1504_05869_gb300.workloads import sinusoid, stiff_source

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1504_05869_gb300 as pk
    return pk


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _rand(shape, seed):
    r = np.random.default_rng(seed).standard_normal(shape)
    return r - r.mean()


def _fft(pk, rho, lattice, order, tau, host=False, epsilon=1.0):
    import torch
    prob = pk.problem(lattice, rho.shape, order, tau_lb=tau, epsilon=epsilon)
    if host:
        out = np.empty_like(rho)
        st = pk.fixed_point_fft(np.ascontiguousarray(rho), out, prob)
        return out, st
    r = torch.from_numpy(np.ascontiguousarray(rho)).cuda()
    phi = torch.empty_like(r)
    st = pk.fixed_point_fft(r, phi, prob)
    return phi.cpu().numpy(), st


CASES = [
    ("D1Q5", 3, (45,), 0.9),
    ("D1Q9", 5, (77,), 1.7),
    ("D1Q13", 7, (100,), 1.0),
    ("D1Q13", 7, (5,), 1.2),
    ("D2Q25", 1, (9, 13), 0.8),
    ("D2Q81", 5, (17, 23), 1.2),
    ("D2Q169", 7, (21, 19), 6.04398),
    ("D2Q169", 7, (4, 7), 1.0),
    ("D3Q19", 1, (7, 9, 11), 0.75),
    ("D3Q19", 3, (6, 5, 8), 1.1),
    ("D3Q111", 5, (9, 7, 13), 1.0),
    ("D3Q111", 5, (16, 16, 16), 2.5),
    ("D3Q111", 5, (2, 3, 5), 1.4),
    ("D3Q111", 5, (33, 40, 31), 0.8),
]


@pytest.mark.parametrize("lattice,order,shape,tau", CASES)
def test_fft_matches_closed_form(pk, lattice, order, shape, tau):
    rho = _rand(shape, 5) + 0.25          # a non-zero mean, removed on both sides
    lat = oracle.lattice(lattice, order)
    S, mean = oracle.source(rho, lat, tau, 2.0)
    want = pins.fixed_point(S, lat.vel, lat.phi, lat.chi, 1.0 / tau)
    got, st = _fft(pk, rho, lattice, order, tau, epsilon=2.0)
    assert _rel(got, want) <= 1e-12, _rel(got, want)
    assert abs(st["rho_mean_removed"] - rho.mean()) < 1e-15
    assert abs(got.mean()) <= 1e-13 * np.abs(got).max()


def test_fft_host_and_device_buffers_agree(pk):
    rho, _ = stiff_source((24, 20, 28), count=4, sigma=1.5, seed=9)
    a, _ = _fft(pk, rho, "D3Q111", 5, 1.3)
    b, _ = _fft(pk, rho, "D3Q111", 5, 1.3, host=True)
    assert np.array_equal(a, b)


def test_fft_single_mode_full_size(pk):
    """256^3, the 3D N=5 set at the Kn = 0.2 relaxation time: a product of
    sines (modes 1, 2, 3) holds the eight wave vectors (+-k1, +-k2, +-k3),
    on which T takes one value (the set is symmetric under each axis
    reflection), so Phi = T(k) S exactly."""
    shape = (256, 256, 256)
    lat = oracle.lattice("D3Q111", 5)
    tau = oracle.tau_from_knudsen(0.2, (256, 256, 256), lat.cs2)
    rho = sinusoid(shape, modes=(1, 2, 3))     # l_x, l_y, l_z
    got, st = _fft(pk, rho, "D3Q111", 5, tau)
    k = 2 * np.pi * np.array([1.0, 2.0, 3.0]) / 256
    T = pins.transfer(k, lat.vel, lat.phi, lat.chi, 1.0 / tau)
    assert abs(T.imag) < 1e-12 * abs(T.real)
    S = (rho - rho.mean()) * lat.cs2 * (tau - 0.5)
    assert _rel(got, T.real * S) <= 1e-11
    assert st["tau_lb"] == tau


@pytest.mark.parametrize("lattice,order,shape,tau", [
    ("D3Q111", 5, (20, 18, 22), 1.0),
    ("D2Q169", 7, (40, 36), 1.0),
    ("D3Q19", 1, (24, 24, 24), 0.9),
])
def test_iteration_converges_to_fft(pk, lattice, order, shape, tau):
    """The CUDA iteration run until the per-step change is at rounding level
    lands on the comparator's fixed point."""
    import torch
    rho, _ = stiff_source(shape, count=4, sigma=1.5, seed=6)
    fx, _ = _fft(pk, rho, lattice, order, tau)
    prob = pk.problem(lattice, shape, order, tau_lb=tau, tol=1e-14, tol_kind="rel_l2",
                      check_every=16, max_sweeps=60000)
    r = torch.from_numpy(rho).cuda()
    phi = torch.empty_like(r)
    rc, st = pk.solve(r, phi, prob)
    assert rc in (0, -4)
    assert _rel(phi.cpu().numpy(), fx) <= 1e-10, (_rel(phi.cpu().numpy(), fx), st)


def test_fft_rejects_nonfinite_rho(pk):
    rho = _rand((8, 8, 8), 2)
    rho[3, 4, 5] = np.inf
    phi = np.full_like(rho, 7.0)
    with pytest.raises(pk.PkrError) as e:
        pk.fixed_point_fft(rho, phi, pk.problem("D3Q111", rho.shape, 5, tau_lb=1.0))
    assert e.value.status == -1
    assert (phi == 7.0).all()
