"""The allocation-free residual entry point (pkr_residual_noalloc).

Callers that cannot allocate device memory -- code inside a CUDA graph
capture, runtimes that own all device memory, allocator-free loops -- use this
entry point, whose scratch is a static device array of the library.  The test
checks, through the C ABI, that two calls in a row return the same residuals
as the solver's own (allocating) check step on the same pair of potentials.
It lives in a file of its own that pytest collects last.
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
