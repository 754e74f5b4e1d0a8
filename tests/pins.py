"""Independent pins for the oracle (test-side only).

Each function here computes something the oracle's result must equal, by a
route that shares nothing with the oracle's real-space loops:

* ``fourier_steps``  -- the scheme is linear and translation invariant, so
  each Fourier mode k evolves on its own: g^(t+1)(k) = E(k) [(1-w) g^t(k) +
  w phi (1^T g^t(k)) + chi S(k)], E = diag(exp(-i k.v_j)).  Iterating that
  per mode and transforming back gives Phi after any number of steps.
* ``fixed_point``    -- the same recursion at steady state, solved in closed
  form with the Sherman-Morrison formula (the collision is a scaled identity
  plus a rank-one term):
      Phi(k) = S(k) sum_j e_j chi_j / (1-(1-w) e_j)
               / (1 - w sum_j e_j phi_j / (1-(1-w) e_j)),   Phi(0) = 0.
* ``dense_fixed_point`` -- brute force: assemble the full linear map on the
  Q*V populations as a sparse matrix and solve (I - P) g = c directly,
  bordered with the gauge sum_x Phi = 0.
* ``spectral_poisson`` -- continuum periodic Poisson solution
  Phi(k) = rho(k) / (eps |k|^2) (continuum reference, not the scheme).
* ``stencil_omega1`` -- at w = 1 the collision forgets g, so
  Phi^(t+1)(x) = sum_j phi_j Phi^t(x - v_j) + sum_j chi_j S(x - v_j).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def _wavenumbers(shape3):
    nx, ny, nz = shape3
    kx = 2 * np.pi * np.fft.fftfreq(nx)
    ky = 2 * np.pi * np.fft.fftfreq(ny)
    kz = 2 * np.pi * np.fft.fftfreq(nz)
    return kx, ky, kz


def _phases(vel, shape3):
    """e_j(k) = exp(-i k.v_j) on the grid's FFT modes, array (Q, nz, ny, nx)."""
    kx, ky, kz = _wavenumbers(shape3)
    out = []
    for v in vel:
        ex = np.exp(-1j * kx * v[0])
        ey = np.exp(-1j * ky * v[1])
        ez = np.exp(-1j * kz * v[2])
        out.append(ez[:, None, None] * ey[None, :, None] * ex[None, None, :])
    return np.array(out)


def _as3(a):
    a = np.asarray(a)
    return a.reshape((1,) * (3 - a.ndim) + a.shape)


def fourier_steps(S, vel, phi, chi, omega, steps):
    """Phi after ``steps`` steps from g = 0, computed mode by mode."""
    shape = np.shape(S)
    S3 = _as3(S)
    shape3 = S3.shape[::-1]
    Sk = np.fft.fftn(S3)
    E = _phases(vel, shape3)
    ph = np.asarray(phi)[:, None, None, None]
    ch = np.asarray(chi)[:, None, None, None]
    g = np.zeros_like(E)
    for _ in range(steps):
        Phi = g.sum(axis=0)
        g = E * ((1 - omega) * g + omega * ph * Phi + ch * Sk)
    return np.real(np.fft.ifftn(g.sum(axis=0))).reshape(shape)


def fourier_phi_sequence(S, vel, phi, chi, omega, steps):
    """Phi^1 .. Phi^steps from g = 0, computed mode by mode (the recurrence
    of fourier_steps, every step kept)."""
    shape = np.shape(S)
    S3 = _as3(S)
    shape3 = S3.shape[::-1]
    Sk = np.fft.fftn(S3)
    E = _phases(vel, shape3)
    ph = np.asarray(phi)[:, None, None, None]
    ch = np.asarray(chi)[:, None, None, None]
    g = np.zeros_like(E)
    out = []
    for _ in range(steps):
        Phi = g.sum(axis=0)
        g = E * ((1 - omega) * g + omega * ph * Phi + ch * Sk)
        out.append(np.real(np.fft.ifftn(g.sum(axis=0))).reshape(shape))
    return out


def fixed_point(S, vel, phi, chi, omega):
    """Exact steady state of the scheme (closed form per Fourier mode)."""
    shape = np.shape(S)
    S3 = _as3(S)
    shape3 = S3.shape[::-1]
    Sk = np.fft.fftn(S3)
    num = np.zeros(S3.shape, dtype=complex)
    den = np.ones(S3.shape, dtype=complex)
    kx, ky, kz = _wavenumbers(shape3)
    for v, p, c in zip(vel, phi, chi):
        e = (np.exp(-1j * kz * v[2])[:, None, None]
             * np.exp(-1j * ky * v[1])[None, :, None]
             * np.exp(-1j * kx * v[0])[None, None, :])
        q = e / (1 - (1 - omega) * e)
        num += c * q
        den -= omega * p * q
    T = np.zeros_like(num)
    nz0 = np.ones(S3.shape, dtype=bool)
    nz0[0, 0, 0] = False
    T[nz0] = num[nz0] / den[nz0]
    return np.real(np.fft.ifftn(T * Sk)).reshape(shape)


def transfer(k, vel, phi, chi, omega):
    """T(k) for a single wave vector k (3-vector)."""
    e = np.exp(-1j * (np.asarray(vel) @ np.asarray(k, dtype=float)))
    q = e / (1 - (1 - omega) * e)
    return (np.sum(chi * q) / (1 - omega * np.sum(phi * q)))


def dense_fixed_point(S, vel, phi, chi, omega):
    """Steady state by a direct sparse solve over all Q*V populations."""
    shape = np.shape(S)
    S3 = _as3(S)
    nz, ny, nx = S3.shape
    V = S3.size
    Q = len(vel)
    idx = np.arange(V).reshape(nz, ny, nx)
    rows, cols, vals = [], [], []
    c = np.zeros(Q * V)
    for i, v in enumerate(vel):
        # population i at x comes from site x - v_i
        src = np.roll(idx, shift=(v[2], v[1], v[0]), axis=(0, 1, 2)).ravel()
        r = i * V + np.arange(V)
        rows.append(r)
        cols.append(i * V + src)
        vals.append(np.full(V, 1 - omega))
        for j in range(Q):
            rows.append(r)
            cols.append(j * V + src)
            vals.append(np.full(V, omega * phi[i]))
        c[r] = chi[i] * S3.ravel()[src]
    P = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows),
                                              np.concatenate(cols))),
                      shape=(Q * V, Q * V))
    A = sp.identity(Q * V, format="csr") - P
    ones = sp.csr_matrix(np.ones((1, Q * V)))
    B = sp.bmat([[A, ones.T], [ones, None]], format="csc")
    rhs = np.concatenate([c, [0.0]])
    sol = spla.spsolve(B, rhs)
    g = sol[:Q * V].reshape(Q, V)
    return g.sum(axis=0).reshape(shape)


def spectral_poisson(rho, eps=1.0):
    """Continuum periodic Poisson: lap Phi = -(rho - <rho>)/eps, <Phi> = 0."""
    shape = np.shape(rho)
    r3 = _as3(rho)
    kx, ky, kz = _wavenumbers(r3.shape[::-1])
    k2 = (kz[:, None, None] ** 2 + ky[None, :, None] ** 2
          + kx[None, None, :] ** 2)
    rk = np.fft.fftn(r3)
    out = np.zeros_like(rk)
    m = k2 > 0
    out[m] = rk[m] / (eps * k2[m])
    return np.real(np.fft.ifftn(out)).reshape(shape)


def stencil_omega1(S, vel, phi, chi, steps):
    """Phi after ``steps`` steps at omega = 1 via the scalar stencil."""
    shape = np.shape(S)
    S3 = _as3(S)

    def conv(field, wts):
        out = np.zeros_like(field)
        for v, wt in zip(vel, wts):
            out += wt * np.roll(field, shift=(v[2], v[1], v[0]), axis=(0, 1, 2))
        return out

    St = conv(S3, chi)
    Phi = np.zeros_like(S3)
    for _ in range(steps):
        Phi = conv(Phi, phi) + St
    return Phi.reshape(shape)
