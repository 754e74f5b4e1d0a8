"""ctypes binding of the C ABI in ``include/pkr.h`` (argument marshalling only).

Every function here has the name and argument order of its C counterpart.
The library must have been built (``paper_1504_05869_gb300.build``); if it is
missing, importing the binding raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpkr.so")

# pkr_status
PKR_OK, PKR_EINVAL, PKR_ENOMEM, PKR_EUNSTABLE = 0, -1, -2, -3
PKR_ENOCONV, PKR_EDIVERGED, PKR_ECUDA, PKR_EBUSY = -4, -5, -6, -7
# pkr_lattice
LATTICES = {"D1Q5": 0, "D1Q9": 1, "D1Q13": 2, "D2Q25": 3, "D2Q81": 4, "D2Q169": 5,
            "D3Q19": 6, "D3Q111": 7}
LATTICE_DIM = {"D1Q5": 1, "D1Q9": 1, "D1Q13": 1, "D2Q25": 2, "D2Q81": 2, "D2Q169": 2,
               "D3Q19": 3, "D3Q111": 3}
# pkr_precision / pkr_tol_kind
PKR_FP64, PKR_FP32, PKR_MIXED, PKR_FP16, PKR_MIXED16, PKR_FX64 = 0, 1, 2, 3, 4, 5
PKR_MIXED_FX64 = 6
PKR_TOL_MAX_ABS_DPHI, PKR_TOL_REL_L2_DPHI = 0, 1

# Every symbol include/pkr.h declares (checked by the tests).
EXPORTS = [
    "pkr_status_str", "pkr_version", "pkr_lattice_info", "pkr_tau_from_knudsen",
    "pkr_plan_bytes", "pkr_plan_create", "pkr_plan_destroy", "pkr_plan_load_source",
    "pkr_plan_run", "pkr_plan_sweeps", "pkr_plan_phi", "pkr_plan_steps",
    "pkr_plan_populations", "pkr_solve", "pkr_residual_noalloc", "pkr_variant_count",
    "pkr_batch_variant_count",
    "pkr_plan_autotune", "pkr_ctx_create", "pkr_submit", "pkr_poll", "pkr_ctx_run",
    "pkr_ctx_wait", "pkr_ctx_info", "pkr_ctx_destroy", "pkr_plan_import",
    "pkr_fixed_point_fft", "pkr_ctx_release", "pkr_pull_copy_ceiling",
]


class pkr_problem(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("lattice", ctypes.c_int32),
                ("n", ctypes.c_int64 * 3), ("order", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("tau_lb", ctypes.c_double),
                ("knudsen", ctypes.c_double), ("epsilon", ctypes.c_double),
                ("tol", ctypes.c_double), ("tol_kind", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("max_sweeps", ctypes.c_int64),
                ("variant", ctypes.c_int32)]


class pkr_stats(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("residual", ctypes.c_double), ("rho_mean_removed", ctypes.c_double),
                ("tau_lb", ctypes.c_double), ("cs2", ctypes.c_double),
                ("wall_ms", ctypes.c_double), ("glups", ctypes.c_double),
                ("hbm_gbs", ctypes.c_double), ("variant", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class pkr_ctx_config(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int32), ("order", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("hbm_budget_bytes", ctypes.c_size_t), ("variant", ctypes.c_int32),
                ("probe_edge", ctypes.c_int32), ("threaded", ctypes.c_int32),
                ("max_grids", ctypes.c_int32)]


_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)

_SIGS = {
    "pkr_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "pkr_version": (ctypes.c_char_p, []),
    "pkr_lattice_info": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _I32, _I32, _I32, _D, _D,
                                        _D, _D]),
    "pkr_tau_from_knudsen": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, _I64, _D]),
    "pkr_plan_bytes": (ctypes.c_int, [ctypes.POINTER(pkr_problem),
                                      ctypes.POINTER(ctypes.c_size_t)]),
    "pkr_plan_create": (ctypes.c_int, [ctypes.POINTER(pkr_problem), _P, ctypes.POINTER(_P)]),
    "pkr_plan_destroy": (ctypes.c_int, [_P]),
    "pkr_plan_load_source": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "pkr_plan_run": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_double, ctypes.c_int,
                                    ctypes.c_int, ctypes.POINTER(pkr_stats)]),
    "pkr_plan_sweeps": (ctypes.c_int, [_P, ctypes.c_int64]),
    "pkr_plan_phi": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "pkr_plan_steps": (ctypes.c_int64, [_P]),
    "pkr_plan_populations": (_P, [_P]),
    "pkr_solve": (ctypes.c_int, [ctypes.POINTER(pkr_problem), _P, _P, ctypes.c_int,
                                 ctypes.POINTER(pkr_stats), _P]),
    "pkr_residual_noalloc": (ctypes.c_int, [_P, _P, ctypes.c_int64, _D, _P]),
    "pkr_fixed_point_fft": (ctypes.c_int, [ctypes.POINTER(pkr_problem), _P, _P, ctypes.c_int,
                                           ctypes.POINTER(pkr_stats), _P]),
    "pkr_variant_count": (ctypes.c_int, [ctypes.c_int]),
    "pkr_batch_variant_count": (ctypes.c_int, [ctypes.c_int]),
    "pkr_pull_copy_ceiling": (ctypes.c_int, [ctypes.c_int, _I64, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, _D, _P]),
    "pkr_plan_autotune": (ctypes.c_int, [_P, ctypes.c_int, _I32, _D]),
    "pkr_ctx_create": (ctypes.c_int, [ctypes.POINTER(pkr_ctx_config), _P, ctypes.POINTER(_P)]),
    "pkr_submit": (ctypes.c_int, [_P, ctypes.POINTER(pkr_problem), _P, _P, ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_uint64)]),
    "pkr_poll": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(pkr_stats)]),
    "pkr_ctx_run": (ctypes.c_int, [_P, ctypes.c_int64]),
    "pkr_ctx_wait": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(pkr_stats)]),
    "pkr_ctx_info": (ctypes.c_int, [_P, _I64, _D, _I64, ctypes.POINTER(ctypes.c_size_t), _I32]),
    "pkr_ctx_destroy": (ctypes.c_int, [_P]),
    "pkr_ctx_release": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "pkr_plan_import": (ctypes.c_int, [_P, _P]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libpkr.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(
                f"{path} is missing: build the CUDA library first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class PkrError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = load().pkr_status_str(status).decode()
        super().__init__(f"{where}: {msg} ({status})")


def check(status: int, where: str) -> int:
    if status != PKR_OK:
        raise PkrError(status, where)
    return status


def _fn(name):
    def call(*args):
        return getattr(load(), name)(*args)
    call.__name__ = name
    return call


pkr_status_str = _fn("pkr_status_str")
pkr_version = _fn("pkr_version")
pkr_lattice_info = _fn("pkr_lattice_info")
pkr_tau_from_knudsen = _fn("pkr_tau_from_knudsen")
pkr_plan_bytes = _fn("pkr_plan_bytes")
pkr_plan_create = _fn("pkr_plan_create")
pkr_plan_destroy = _fn("pkr_plan_destroy")
pkr_plan_load_source = _fn("pkr_plan_load_source")
pkr_plan_run = _fn("pkr_plan_run")
pkr_plan_sweeps = _fn("pkr_plan_sweeps")
pkr_plan_phi = _fn("pkr_plan_phi")
pkr_plan_steps = _fn("pkr_plan_steps")
pkr_plan_populations = _fn("pkr_plan_populations")
pkr_solve = _fn("pkr_solve")
pkr_residual_noalloc = _fn("pkr_residual_noalloc")
pkr_fixed_point_fft = _fn("pkr_fixed_point_fft")
pkr_variant_count = _fn("pkr_variant_count")
pkr_batch_variant_count = _fn("pkr_batch_variant_count")
pkr_pull_copy_ceiling = _fn("pkr_pull_copy_ceiling")
pkr_plan_autotune = _fn("pkr_plan_autotune")
pkr_ctx_create = _fn("pkr_ctx_create")
pkr_submit = _fn("pkr_submit")
pkr_poll = _fn("pkr_poll")
pkr_ctx_run = _fn("pkr_ctx_run")
pkr_ctx_wait = _fn("pkr_ctx_wait")
pkr_ctx_info = _fn("pkr_ctx_info")
pkr_ctx_destroy = _fn("pkr_ctx_destroy")
pkr_ctx_release = _fn("pkr_ctx_release")
pkr_plan_import = _fn("pkr_plan_import")
