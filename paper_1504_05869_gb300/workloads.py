"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle
checks.  Holds no arithmetic of the solver itself: only charge densities,
grid shapes and request traces.

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15,
then two xor-shift-multiply rounds.  A double is the top 53 bits times
2^-53.  Draws are consumed in a fixed order (centre x, y, z, then sigma where
ranged, then count where ranged) so every workload is reproducible.

Gaussian charge: q (2 pi sigma^2)^(-D/2) exp(-d^2 / (2 sigma^2)) with d the
periodic minimum-image distance to the centre, evaluated on the cells whose
per-axis distance is at most ceil(10 sigma) (beyond that the factor is below
e^-50 of the peak and is taken as zero).  Charges alternate +1, -1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_M64 = (1 << 64) - 1


class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & _M64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))


def _axis_window(n: int, c: float, sigma: float, half: int):
    """Cells within +-half of c on a periodic axis (each once) and their
    exp(-d^2 / 2 sigma^2) factors, d the minimum-image distance."""
    lo = int(math.floor(c)) - half
    idx = np.arange(lo, lo + 2 * half + 2)
    if len(idx) >= n:
        idx = np.arange(n)
    idx = np.unique(idx % n)
    d = np.abs(idx.astype(np.float64) - c)
    d = np.minimum(d, n - d)
    keep = d <= half
    idx, d = idx[keep], d[keep]
    return idx, np.exp(-d * d / (2.0 * sigma * sigma))


def gaussian_charges(shape, centres, sigmas, charges) -> np.ndarray:
    """Sum of periodic Gaussians on a grid of numpy shape (nz, ny, nx) (or
    (ny, nx), (nx,)); centres are (x, y, z) tuples in cell units."""
    dim = len(shape)
    rho = np.zeros(shape, dtype=np.float64)
    n_xyz = tuple(shape[::-1])
    for c, s, q in zip(centres, sigmas, charges):
        half = int(math.ceil(10.0 * s))
        norm = q * (2.0 * math.pi * s * s) ** (-dim / 2.0)
        wins = [_axis_window(n_xyz[a], c[a], s, half) for a in range(dim)]
        # outer product in numpy's (z, y, x) order
        field = wins[dim - 1][1]
        for a in range(dim - 2, -1, -1):
            field = np.multiply.outer(field, wins[a][1])
        rho[np.ix_(*[wins[a][0] for a in range(dim - 1, -1, -1)])] += norm * field
    return rho


def stiff_source(shape, count: int, sigma: float, seed: int):
    """`count` Gaussians of width sigma, centres uniform on the grid from
    SplitMix64(seed), charges alternating +1/-1.  Returns (rho, centres)."""
    rng = SplitMix64(seed)
    n_xyz = tuple(shape[::-1])
    centres = []
    for _ in range(count):
        centres.append(tuple(rng.uniform() * n_xyz[a] for a in range(len(shape))))
    charges = [1.0 if j % 2 == 0 else -1.0 for j in range(count)]
    rho = gaussian_charges(shape, centres, [sigma] * count, charges)
    return rho, centres


def sinusoid(shape, modes=None, amplitude: float = 1.0) -> np.ndarray:
    """prod_a sin(2 pi l_a x_a / n_a) (the paper's smooth source, Eq.
    eq:source, with l_a = 1 by default)."""
    n_xyz = tuple(shape[::-1])
    modes = modes or (1,) * len(shape)
    field = np.ones((), dtype=np.float64)
    for a in range(len(shape) - 1, -1, -1):
        x = np.arange(n_xyz[a], dtype=np.float64)
        field = np.multiply.outer(field, np.sin(2 * np.pi * modes[a] * x / n_xyz[a]))
    return amplitude * field


def log_uniform_int(rng: SplitMix64, lo: int, hi: int) -> int:
    return int(round(math.exp(math.log(lo) + rng.uniform() * (math.log(hi) - math.log(lo)))))


@dataclass
class GridJob:
    shape: tuple          # numpy order (nz, ny, nx)
    centres: list
    sigmas: list
    charges: list

    def rho(self) -> np.ndarray:
        return gaussian_charges(self.shape, self.centres, self.sigmas, self.charges)


def batch_jobs(count: int = 256, lo: int = 32, hi: int = 128, seed: int = 2,
               max_sources: int = 16, sig_lo: float = 1.0, sig_hi: float = 4.0):
    """Independent periodic 3D grids: edges log-uniform in [lo, hi] per axis,
    1..max_sources Gaussians with sigma uniform in [sig_lo, sig_hi]."""
    rng = SplitMix64(seed)
    jobs = []
    for _ in range(count):
        nx = log_uniform_int(rng, lo, hi)
        ny = log_uniform_int(rng, lo, hi)
        nz = log_uniform_int(rng, lo, hi)
        k = 1 + int(rng.uniform() * max_sources)
        cs, ss = [], []
        for _ in range(k):
            cs.append((rng.uniform() * nx, rng.uniform() * ny, rng.uniform() * nz))
            ss.append(sig_lo + rng.uniform() * (sig_hi - sig_lo))
        qs = [1.0 if j % 2 == 0 else -1.0 for j in range(k)]
        jobs.append(GridJob((nz, ny, nx), cs, ss, qs))
    return jobs


@dataclass
class Request:
    arrival_s: float
    shape: tuple
    tol: float
    smooth: bool
    job: GridJob

    def rho(self) -> np.ndarray:
        if self.smooth:
            return sinusoid(self.shape)
        return self.job.rho()


def serving_trace(count: int, rate_hz: float = 200.0, lo: int = 32, hi: int = 256,
                  seed: int = 3, tols=(1e-6, 1e-8, 1e-10)):
    """Poisson arrivals (exponential gaps) of periodic 3D solves."""
    rng = SplitMix64(seed)
    t = 0.0
    out = []
    for _ in range(count):
        t += -math.log(1.0 - rng.uniform()) / rate_hz
        nx = log_uniform_int(rng, lo, hi)
        ny = log_uniform_int(rng, lo, hi)
        nz = log_uniform_int(rng, lo, hi)
        tol = tols[min(int(rng.uniform() * len(tols)), len(tols) - 1)]
        smooth = rng.uniform() < 0.5
        k = 1 + int(rng.uniform() * 16)
        cs, ss = [], []
        for _ in range(k):
            cs.append((rng.uniform() * nx, rng.uniform() * ny, rng.uniform() * nz))
            ss.append(1.0 + rng.uniform() * 3.0)
        qs = [1.0 if j % 2 == 0 else -1.0 for j in range(k)]
        out.append(Request(t, (nz, ny, nx), tol, smooth, GridJob((nz, ny, nx), cs, ss, qs)))
    return out
