"""binary16 storage of the populations against binary16 storage of their
deviations from equilibrium, emulated on the host.

The binary16 mode stores each post-collision population p_i with one
power-of-two scale per array.  The alternative the precision workload names
stores the deviation d_i = p_i - phi_i Phi - chi_i S = (1 - omega)(g_i - phi_i
Phi), again with one power-of-two scale, together with Phi (binary32), and
rebuilds p_i = d_i + phi_i Phi + chi_i S before streaming (the equilibrium of
Eq. equilibrium2 plus the source term).  Both are emulated here with numpy on
a 16^3 grid with stiff Gaussian sources, D3Q111 N=5, for 300 steps from zero,
and compared with binary64 storage of the same steps.

At the relaxation time of the benchmark's Kn 0.2 on 256^3 (tau_lb = 61.8,
omega = 0.016) the deviations are as large as the populations (the iterate
is far from local equilibrium), and the two forms give the same error.
Close to the paper's tau_lb = 1 the deviation is a small fraction of p and
the deviation form is about 4x more accurate.  This is why the library's
binary16 mode stores scaled populations; see the bounds below.
"""
import numpy as np
import pytest

import oracle
from paper_1504_05869_gb300.workloads import stiff_source

TAU_BENCH = 61.78536424412542   # Kn 0.2 on 256^3 (Kn = c_s (tau_lb - 1/2) / L)


def _emulate(tau, mode, shape=(16, 16, 16), steps=300):
    lat = oracle.lattice("D3Q111", 5)
    rho, _ = stiff_source(shape, count=8, sigma=1.5, seed=7)
    S = oracle.source(rho, lat, tau)[0].ravel()
    nz, ny, nx = shape
    V = S.size
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    vel = np.asarray(lat.vel)
    Q = lat.Q
    # pull: g_i(x) = A_i(x - v_i), periodic
    src = np.concatenate([(((z - v[2]) % nz) * ny + (y - v[1]) % ny) * nx + (x - v[0]) % nx
                          for v in vel], axis=None) + np.repeat(np.arange(Q) * V, V)
    ph = np.asarray(lat.phi)[:, None]
    ch = np.asarray(lat.chi)[:, None]
    om = 1.0 / tau

    def stored(a):
        # binary16 with one power-of-two scale per array, 4x headroom
        s = 2.0 ** np.ceil(np.log2(max(4.0 * np.abs(a).max() / 65504.0, 1e-300)))
        return (a / s).astype(np.float16).astype(np.float64) * s

    A = np.zeros((Q, V))
    dmax = pmax = 0.0
    for _ in range(steps):
        g = A.ravel()[src].reshape(Q, V)
        Phi = g.sum(0)
        p = (1.0 - om) * g + om * ph * Phi + ch * S
        d = p - ph * Phi - ch * S
        pmax, dmax = np.abs(p).max(), np.abs(d).max()
        if mode == "fp64":
            A = p
        elif mode == "pop16":
            A = stored(p)
        else:
            A = stored(d) + ph * Phi.astype(np.float32).astype(np.float64) + ch * S
    g = A.ravel()[src].reshape(Q, V)
    return g.sum(0), dmax / pmax


@pytest.mark.parametrize("tau,lo,hi", [(TAU_BENCH, 0.5, 2.0), (1.3, 0.0, 0.5)])
def test_deviation_form_against_population_form(tau, lo, hi):
    ref, ratio = _emulate(tau, "fp64")
    e = {}
    for mode in ("pop16", "dev16"):
        got, _ = _emulate(tau, mode)
        e[mode] = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    gain = e["dev16"] / e["pop16"]
    assert lo <= gain <= hi, (tau, e, ratio)
    if tau == TAU_BENCH:
        assert ratio > 0.9          # deviations as large as the populations
    else:
        assert ratio < 0.5
