"""The allocation-free residual entry point (pkr_residual_noalloc).

Callers that cannot allocate device memory -- runtimes whose device memory
all belongs to their own pool, loops that must not enter the allocator -- use
this entry point, whose scratch is a static device array of the library.  The
tests check, through the C ABI, that two calls in a row return the same
residuals as the solver's own (allocating) check step on the same pair of
potentials, that a grid of more than 1024 x 256 sites (several passes of the
block-stride loop, more than 256 partials in the final reduction) matches a
host evaluation, and what non-finite inputs give.  They live in a file of
their own that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def pk():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1504_05869_gb300 as pk
    return pk


def test_noalloc_residual_matches_solver_check(pk):
    import torch
    from paper_1504_05869_gb300.workloads import stiff_source
    shape = (12, 10, 14)
    rho, _ = stiff_source(shape, count=5, sigma=1.5, seed=21)
    prob = pk.problem("D3Q111", shape, 5, tau_lb=1.3, max_sweeps=1000, check_every=1)
    r = torch.from_numpy(rho).cuda()
    old = torch.empty_like(r)
    new = torch.empty_like(r)
    stream = torch.cuda.current_stream().cuda_stream
    out = (ctypes.c_double * 3)()
    with pk.Plan(prob) as P:
        P.load_source(r)
        P.run(5)
        for kind, idx in (("rel_l2", 1), ("max_abs", 0)):   # two calls in a row
            P.phi(old)
            rc, st = P.run(1, tol_kind=kind, check_every=1)
            assert rc == 0
            P.phi(new)
            torch.cuda.synchronize()
            status = pk._pkr.pkr_residual_noalloc(new.data_ptr(), old.data_ptr(), new.numel(),
                                                  out, stream)
            assert status == 0
            want = st["residual"]
            assert want > 0
            assert abs(out[idx] - want) <= TOL * want, (kind, out[idx], want)
            # the other two results against a host evaluation of the same pair
            a, b = new.cpu().numpy(), old.cpu().numpy()
            assert abs(out[0] - np.abs(a - b).max()) <= TOL * out[0]
            assert abs(out[2] - np.linalg.norm(a)) <= TOL * out[2]


def test_noalloc_rejects_bad_sizes(pk):
    out = (ctypes.c_double * 3)()
    import torch
    t = torch.zeros(4, dtype=torch.float64, device="cuda")
    assert pk._pkr.pkr_residual_noalloc(t.data_ptr(), t.data_ptr(), 0, out, None) == -1
    assert pk._pkr.pkr_residual_noalloc(t.data_ptr(), t.data_ptr(), 1 << 40, out, None) == -1
    assert pk._pkr.pkr_residual_noalloc(None, t.data_ptr(), 4, out, None) == -1


def _noalloc(pk, a, b):
    import torch
    out = (ctypes.c_double * 3)()
    stream = torch.cuda.current_stream().cuda_stream
    rc = pk._pkr.pkr_residual_noalloc(a.data_ptr(), b.data_ptr(), a.numel(), out, stream)
    return rc, list(out)


def test_noalloc_large_grid_against_host(pk):
    """72^3 = 373,248 sites > 1024 blocks x 256 threads: each thread takes
    two sites and the final reduction reads 1024 partials."""
    import torch
    rng = np.random.default_rng(5)
    a = rng.standard_normal((72, 72, 72))
    b = a + 1e-6 * rng.standard_normal(a.shape)
    b[71, 71, 71] += 3e-3           # the largest change, at the last site
    ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    for _ in range(2):               # two calls in a row share the scratch
        rc, out = _noalloc(pk, ta, tb)
        assert rc == 0
        d = a - b
        assert abs(out[0] - np.abs(d).max()) <= TOL * out[0]
        assert abs(out[1] - np.linalg.norm(d) / np.linalg.norm(a)) <= TOL * out[1]
        assert abs(out[2] - np.linalg.norm(a)) <= TOL * out[2]


def test_noalloc_non_finite_inputs(pk):
    """NaN in an input gives NaN in out[0] and out[1]; an infinite entry in
    phi_new gives out[1] = inf / inf = NaN with no NaN input (documented:
    a NaN out[1] means not finite)."""
    import torch
    a = torch.ones(1000, dtype=torch.float64, device="cuda")
    b = torch.zeros_like(a)
    c = a.clone()
    c[17] = float("nan")
    rc, out = _noalloc(pk, c, b)
    assert rc == 0 and np.isnan(out[0]) and np.isnan(out[1])
    c[17] = float("inf")
    rc, out = _noalloc(pk, c, b)
    assert rc == 0 and np.isnan(out[1]) and out[0] == float("inf") and out[2] == float("inf")
    rc, out = _noalloc(pk, a, b)      # the scratch holds no trace of the calls before
    assert rc == 0 and out[0] == 1.0 and out[1] == 1.0 and abs(out[2] - np.sqrt(1000)) <= 1e-12
