"""GB300-native high-order kinetic relaxation Poisson solver.

Thin Python layer over the C ABI of ``include/pkr.h`` (``_pkr``): it only
fills the ``pkr_problem`` struct and passes pointers.  Device tensors are
torch CUDA tensors (float64, contiguous); every step of a solve runs in the
library's CUDA kernels.
"""
from __future__ import annotations

import ctypes

from . import _pkr
from ._pkr import (LATTICE_DIM, LATTICES, PKR_EBUSY, PKR_FP16, PKR_FP32, PKR_FP64,  # noqa: F401
                   PKR_FX64, PKR_MIXED, PKR_MIXED16, PKR_MIXED_FX64,
                   PKR_TOL_MAX_ABS_DPHI, PKR_TOL_REL_L2_DPHI, PkrError, check, pkr_ctx_config,
                   pkr_problem, pkr_stats)

PRECISIONS = {"fp64": PKR_FP64, "fp32": PKR_FP32, "mixed": PKR_MIXED, "fp16": PKR_FP16,
              "mixed16": PKR_MIXED16, "fx64": PKR_FX64, "mixed_fx64": PKR_MIXED_FX64}
TOL_KINDS = {"max_abs": PKR_TOL_MAX_ABS_DPHI, "rel_l2": PKR_TOL_REL_L2_DPHI}


def problem(lattice: str, shape, order: int, tau_lb: float = 0.0, knudsen: float = 0.0,
            epsilon: float = 1.0, tol: float = 0.0, tol_kind: str = "rel_l2",
            check_every: int = 32, max_sweeps: int = 1000, precision: str = "fp64",
            variant: int = -1):
    """pkr_problem for a grid given in numpy/torch order (nz, ny, nx)."""
    n = list(int(v) for v in tuple(shape)[::-1]) + [1, 1, 1]
    p = pkr_problem()
    p.dim = LATTICE_DIM[lattice]
    p.lattice = LATTICES[lattice]
    p.n[0], p.n[1], p.n[2] = n[0], n[1], n[2]
    p.order = int(order)
    p.precision = PRECISIONS[precision]
    p.tau_lb = float(tau_lb)
    p.knudsen = float(knudsen)
    p.epsilon = float(epsilon)
    p.tol = float(tol)
    p.tol_kind = TOL_KINDS[tol_kind]
    p.check_every = int(check_every)
    p.max_sweeps = int(max_sweeps)
    p.variant = int(variant)
    return p


def lattice_info(lattice: str, order: int):
    """(vel (Q,3) int32, w, phi, chi, cs2) from the library's own tables."""
    import numpy as np
    Q = ctypes.c_int32()
    dim = ctypes.c_int32()
    check(_pkr.pkr_lattice_info(LATTICES[lattice], order, ctypes.byref(Q), ctypes.byref(dim),
                                None, None, None, None, None), "pkr_lattice_info")
    q = Q.value
    vel = np.zeros((q, 3), dtype=np.int32)
    w, phi, chi = (np.zeros(q) for _ in range(3))
    cs2 = ctypes.c_double()
    dp = ctypes.POINTER(ctypes.c_double)
    check(_pkr.pkr_lattice_info(LATTICES[lattice], order, None, None,
                                vel.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                w.ctypes.data_as(dp), phi.ctypes.data_as(dp),
                                chi.ctypes.data_as(dp), ctypes.byref(cs2)), "pkr_lattice_info")
    return vel, w, phi, chi, cs2.value


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _ptr(t):
    """Device pointer of a contiguous float64 CUDA tensor, or host pointer of a
    contiguous float64 numpy array / CPU tensor."""
    if hasattr(t, "data_ptr"):
        assert t.dtype.is_floating_point and t.element_size() == 8 and t.is_contiguous()
        return t.data_ptr(), (not t.is_cuda)
    assert t.dtype.itemsize == 8 and t.flags.c_contiguous
    return t.ctypes.data, True


def solve(rho, phi, prob, stream=None):
    """pkr_solve: rho and phi both device tensors or both host arrays.
    Returns (status, stats dict); raises on errors other than PKR_ENOCONV."""
    rp, rh = _ptr(rho)
    pp, ph = _ptr(phi)
    if rh != ph:
        raise ValueError("rho and phi must both be on the device or both on the host")
    st = pkr_stats()
    rc = _pkr.pkr_solve(ctypes.byref(prob), rp, pp, int(rh), ctypes.byref(st),
                        _stream_ptr(stream))
    if rc not in (_pkr.PKR_OK, _pkr.PKR_ENOCONV):
        raise PkrError(rc, "pkr_solve")
    return rc, st.as_dict()


def fixed_point_fft(rho, phi, prob, stream=None):
    """pkr_fixed_point_fft: the scheme's exact steady state by FFT (direct
    comparator; same lattice, order, tau_lb and source as ``solve``).
    Returns the stats dict; raises PkrError on any error."""
    rp, rh = _ptr(rho)
    pp, ph = _ptr(phi)
    if rh != ph:
        raise ValueError("rho and phi must both be on the device or both on the host")
    st = pkr_stats()
    check(_pkr.pkr_fixed_point_fft(ctypes.byref(prob), rp, pp, int(rh), ctypes.byref(st),
                                   _stream_ptr(stream)), "pkr_fixed_point_fft")
    return st.as_dict()


class Plan:
    """Device-resident solve state (pkr_plan_*)."""

    def __init__(self, prob, stream=None):
        self.prob = prob
        self._h = ctypes.c_void_p()
        check(_pkr.pkr_plan_create(ctypes.byref(prob), _stream_ptr(stream),
                                   ctypes.byref(self._h)), "pkr_plan_create")

    def load_source(self, rho):
        p, host = _ptr(rho)
        check(_pkr.pkr_plan_load_source(self._h, p, int(host)), "pkr_plan_load_source")

    def run(self, steps, tol=0.0, tol_kind="rel_l2", check_every=0):
        st = pkr_stats()
        rc = _pkr.pkr_plan_run(self._h, int(steps), float(tol), TOL_KINDS[tol_kind],
                               int(check_every), ctypes.byref(st))
        if rc not in (_pkr.PKR_OK, _pkr.PKR_EDIVERGED):
            raise PkrError(rc, "pkr_plan_run")
        return rc, st.as_dict()

    def autotune(self, steps_per_variant=4):
        best = ctypes.c_int32()
        ms = ctypes.c_double()
        check(_pkr.pkr_plan_autotune(self._h, int(steps_per_variant), ctypes.byref(best),
                                     ctypes.byref(ms)), "pkr_plan_autotune")
        return best.value, ms.value

    def import_state(self, other: "Plan"):
        check(_pkr.pkr_plan_import(self._h, other._h), "pkr_plan_import")

    def sweeps(self, count):
        check(_pkr.pkr_plan_sweeps(self._h, int(count)), "pkr_plan_sweeps")

    def phi(self, out):
        p, host = _ptr(out)
        check(_pkr.pkr_plan_phi(self._h, p, int(host)), "pkr_plan_phi")
        return out

    def steps(self) -> int:
        return int(_pkr.pkr_plan_steps(self._h))

    def populations_ptr(self) -> int:
        return int(_pkr.pkr_plan_populations(self._h) or 0)

    def close(self):
        if self._h:
            _pkr.pkr_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """Batch / serving context (pkr_ctx_*): many solves advanced together."""

    def __init__(self, lattice: str, order: int, precision: str = "fp32",
                 check_every: int = 32, hbm_budget_bytes: int = 150 * 10 ** 9,
                 variant: int = -1, probe_edge: int = 64, threaded: bool = False,
                 max_grids: int = 4096, stream=None):
        cfg = pkr_ctx_config()
        cfg.lattice = LATTICES[lattice]
        cfg.order = int(order)
        cfg.precision = PRECISIONS[precision]
        cfg.check_every = int(check_every)
        cfg.hbm_budget_bytes = int(hbm_budget_bytes)
        cfg.variant = int(variant)
        cfg.probe_edge = int(probe_edge)
        cfg.threaded = int(bool(threaded))
        cfg.max_grids = int(max_grids)
        self.lattice, self.order, self.precision = lattice, order, precision
        self._h = ctypes.c_void_p()
        self._keep = {}
        if stream is None:
            # a stream of its own, so that each window can be a captured graph
            import torch
            stream = torch.cuda.Stream()
        self.stream = stream
        check(_pkr.pkr_ctx_create(ctypes.byref(cfg), _stream_ptr(stream), ctypes.byref(self._h)),
              "pkr_ctx_create")

    def submit(self, rho, phi, shape=None, **kw):
        """Queue a solve; rho/phi device tensors or host arrays (kept alive
        here until poll or wait sees the request finished).  kw: problem()
        arguments."""
        prob = problem(self.lattice, shape if shape is not None else rho.shape, self.order,
                       precision=self.precision, **kw)
        rp, rh = _ptr(rho)
        pp, ph = _ptr(phi)
        if rh != ph:
            raise ValueError("rho and phi must both be on the device or both on the host")
        t = ctypes.c_uint64()
        check(_pkr.pkr_submit(self._h, ctypes.byref(prob), rp, pp, int(rh), ctypes.byref(t)),
              "pkr_submit")
        self._keep[t.value] = (rho, phi)
        return t.value

    def poll(self, ticket):
        st = pkr_stats()
        rc = _pkr.pkr_poll(self._h, ctypes.c_uint64(ticket), ctypes.byref(st))
        if rc != PKR_EBUSY:
            self._keep.pop(ticket, None)   # the library no longer touches rho/phi
        return rc, (st.as_dict() if rc != PKR_EBUSY else None)

    def wait(self, ticket):
        st = pkr_stats()
        rc = _pkr.pkr_ctx_wait(self._h, ctypes.c_uint64(ticket), ctypes.byref(st))
        if rc != PKR_EBUSY:
            self._keep.pop(ticket, None)
        return rc, st.as_dict()

    def release(self, ticket):
        """Forget a finished request (pkr_ctx_release): its ticket becomes
        invalid.  Returns PKR_OK, PKR_EBUSY (not finished) or PKR_EINVAL."""
        rc = _pkr.pkr_ctx_release(self._h, ctypes.c_uint64(ticket))
        if rc == 0:
            self._keep.pop(ticket, None)
        return rc

    def run(self, max_windows=0):
        check(_pkr.pkr_ctx_run(self._h, int(max_windows)), "pkr_ctx_run")

    def info(self):
        f, w = ctypes.c_int64(), ctypes.c_int64()
        su = ctypes.c_double()
        b = ctypes.c_size_t()
        v = ctypes.c_int32()
        check(_pkr.pkr_ctx_info(self._h, ctypes.byref(f), ctypes.byref(su), ctypes.byref(w),
                                ctypes.byref(b), ctypes.byref(v)), "pkr_ctx_info")
        return {"finished": f.value, "site_updates": su.value, "windows": w.value,
                "bytes_in_use": b.value, "variant": v.value}

    def close(self):
        if self._h:
            _pkr.pkr_ctx_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
