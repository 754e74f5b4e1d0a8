"""Python face of the serial FP64 oracle (``pkr_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain CPU statement of the
kinetic relaxation scheme that the CUDA path is checked against.  Only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of the benchmark
may import it; the product library never does.

The C file is compiled with gcc into ``oracle/_build/`` on first use (or by
``__graft_entry__.build()``) with ``-O2 -ffp-contract=off`` so that x86 and
Arm hosts round identically.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

from .lattice import Lattice, lattice

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pkr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_LIB_OMP = os.path.join(_BUILD, "liboracle_omp.so")
_libs = {}

_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)
_I32 = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle into a shared library (no-op when up to date).
    ``openmp`` builds the multi-core baseline from the same source."""
    os.makedirs(_BUILD, exist_ok=True)
    out = _LIB_OMP if openmp else _LIB
    if (force or not os.path.exists(out)
            or os.path.getmtime(out) < os.path.getmtime(_SRC)):
        tmp = out + f".{os.getpid()}.tmp"
        extra = ["-fopenmp"] if openmp else []
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC",
                               "-shared", "-std=c11"] + extra + [_SRC, "-o", tmp, "-lm"])
        os.replace(tmp, out)
    return out


def _load(openmp: bool = False):
    if openmp not in _libs:
        lib = ctypes.CDLL(build(openmp=openmp))
        lib.oracle_threads.restype = ctypes.c_int
        lib.oracle_threads.argtypes = [ctypes.c_int]
        lib.oracle_source.restype = ctypes.c_double
        lib.oracle_source.argtypes = [ctypes.c_int64, _D, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, _D]
        lib.oracle_density.restype = None
        lib.oracle_density.argtypes = [ctypes.c_int, ctypes.c_int64, _D, _D]
        lib.oracle_step.restype = None
        lib.oracle_step.argtypes = [_I64, ctypes.c_int, _I32, _D, _D,
                                    ctypes.c_double, _D, _D, _D]
        lib.oracle_residual.restype = ctypes.c_double
        lib.oracle_residual.argtypes = [ctypes.c_int64, _D, _D, ctypes.c_int]
        lib.oracle_solve.restype = ctypes.c_int64
        lib.oracle_solve.argtypes = [_I64, ctypes.c_int, _I32, _D, _D,
                                     ctypes.c_double, _D, ctypes.c_double,
                                     ctypes.c_int, ctypes.c_int64,
                                     ctypes.c_int64, _D, _D, _D]
        _libs[openmp] = lib
    return _libs[openmp]


def threads(n: int = 0) -> int:
    """Threads of the OpenMP build's step (sets it when n > 0); returns the
    count in effect."""
    return int(_load(True).oracle_threads(int(n)))


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def tau_from_knudsen(kn: float, n, cs2: float) -> float:
    """Relaxation time for a Knudsen number.

    The paper defines Kn = lambda / L with lambda the mean free path and L the
    system size (Sec. "From Boltzmann kinetic theory to diffusion equation")
    and uses tau = tau_lb - 1/2 in lattice units (Sec. "Numerical Results").
    Reading: lambda = c_s tau, L = the shortest periodic edge, so
    tau_lb = 1/2 + Kn * L_min / c_s.
    """
    L = min(int(k) for k in n if int(k) > 1) if any(int(k) > 1 for k in n) else 1
    return 0.5 + kn * L / float(np.sqrt(cs2))


def grid3(shape):
    """(nx, ny, nz) from a numpy shape given as (nz, ny, nx) / (ny, nx) / (nx,)."""
    s = tuple(int(v) for v in shape)[::-1]
    return tuple(s) + (1,) * (3 - len(s))


def source(rho: np.ndarray, lat: Lattice, tau_lb: float, eps: float = 1.0):
    """S = (rho - <rho>) c_s^2 (tau_lb - 1/2) / eps; returns (S, mean)."""
    r = np.ascontiguousarray(rho, dtype=np.float64)
    S = np.empty_like(r)
    mean = _load().oracle_source(r.size, _dp(r), lat.cs2, float(tau_lb),
                                 float(eps), _dp(S))
    return S, mean


def density(g: np.ndarray) -> np.ndarray:
    Q = g.shape[0]
    gg = np.ascontiguousarray(g, dtype=np.float64)
    Phi = np.empty(gg.shape[1:], dtype=np.float64)
    _load().oracle_density(Q, Phi.size, _dp(gg), _dp(Phi))
    return Phi


def _tables(lat: Lattice):
    vel = np.ascontiguousarray(lat.vel, dtype=np.int32)
    return (vel, np.ascontiguousarray(lat.phi), np.ascontiguousarray(lat.chi))


def step(g: np.ndarray, S: np.ndarray, lat: Lattice, omega: float,
         openmp: bool = False) -> np.ndarray:
    """One collide-and-stream step of the state g (shape (Q,) + grid);
    ``openmp`` runs the multi-core build (bitwise the same result)."""
    n = np.array(grid3(S.shape), dtype=np.int64)
    vel, phi, chi = _tables(lat)
    gi = np.ascontiguousarray(g, dtype=np.float64)
    go = np.empty_like(gi)
    Sc = np.ascontiguousarray(S, dtype=np.float64)
    _load(openmp).oracle_step(n.ctypes.data_as(_I64), lat.Q, vel.ctypes.data_as(_I32),
                        _dp(phi), _dp(chi), float(omega), _dp(Sc), _dp(gi), _dp(go))
    return go


@dataclass
class Result:
    phi: np.ndarray       # Phi = sum_i g_i after the final step
    g: np.ndarray         # final populations (Q,) + grid
    steps: int
    residual: float       # last checked change of Phi (-1 if never checked)
    rho_mean: float
    tau_lb: float


def solve(rho: np.ndarray, lattice_name: str, order: int, tau_lb: float = None,
          knudsen: float = None, eps: float = 1.0, tol: float = 0.0,
          tol_kind: int = 1, check_every: int = 1, max_steps: int = 1000,
          g0: np.ndarray = None, S: np.ndarray = None, openmp: bool = False) -> Result:
    """Run the scheme from g = 0 (or g0).

    tol <= 0 runs exactly ``max_steps`` steps.  tol_kind 0 stops on
    max|dPhi| < tol, 1 on ||dPhi||_2/||Phi||_2 < tol, checked every
    ``check_every`` steps.  If S is given it is used as the source directly
    (no mean removal, no scaling).  ``openmp`` runs the multi-core build
    (bitwise the same result).
    """
    lat = lattice(lattice_name, order)
    n3 = grid3(rho.shape)
    if tau_lb is None:
        tau_lb = tau_from_knudsen(knudsen, n3, lat.cs2)
    mean = 0.0
    if S is None:
        S, mean = source(rho, lat, tau_lb, eps)
    S = np.ascontiguousarray(S, dtype=np.float64)
    if g0 is None:
        g = np.zeros((lat.Q,) + rho.shape, dtype=np.float64)
    else:
        g = np.array(g0, dtype=np.float64, order="C", copy=True)
    Phi = np.empty(rho.shape, dtype=np.float64)
    res = ctypes.c_double(0.0)
    vel, phi, chi = _tables(lat)
    n = np.array(n3, dtype=np.int64)
    t = _load(openmp).oracle_solve(n.ctypes.data_as(_I64), lat.Q,
                             vel.ctypes.data_as(_I32), _dp(phi), _dp(chi),
                             1.0 / float(tau_lb), _dp(S), float(tol),
                             int(tol_kind), int(check_every), int(max_steps),
                             _dp(g), _dp(Phi), ctypes.byref(res))
    if t < 0:
        raise MemoryError("oracle_solve: allocation failed")
    return Result(phi=Phi, g=g, steps=int(t), residual=res.value,
                  rho_mean=mean, tau_lb=float(tau_lb))
