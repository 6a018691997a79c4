"""Independent spectral formulations used to pin the oracle (tests only).

On a periodic grid every constant-coefficient finite-difference operator of the
scheme is diagonalised by the DFT, so the whole ADI step of Eq. 3.1 can be
written mode by mode: each difference operator becomes its symbol and each
implicit solve a division.  This shares nothing with the oracle's bordered LU
solves or its direct stencil sums, so agreement pins both.
"""
from __future__ import annotations

import numpy as np


def second_diff_symbol(n: int, h: float) -> np.ndarray:
    """Symbol p(k) >= 0 of -(f_{i+1} - 2 f_i + f_{i-1}) / h^2: 4 sin^2(pi k / n) / h^2."""
    k = np.fft.fftfreq(n) * n
    return 4.0 * np.sin(np.pi * k / n) ** 2 / h**2


def ch_step_spectral(cn, cp, lx, ly, gamma, dt):
    """One step of Eq. 3.1 (C-bar = 2C^n - C^{n-1}) evaluated in Fourier space."""
    ny, nx = cn.shape
    dx, dy = lx / nx, ly / ny
    px = second_diff_symbol(nx, dx)[None, :]
    py = second_diff_symbol(ny, dy)[:, None]
    cb = 2.0 * cn - cp
    nl = cn**3 - cn
    lap = -(px + py)
    rh = (-(2.0 / 3.0) * np.fft.fft2(cn - cp)
          - (2.0 / 3.0) * gamma * dt * lap**2 * np.fft.fft2(cb)
          + (2.0 / 3.0) * dt * lap * np.fft.fft2(nl))
    vh = rh / ((1.0 + (2.0 / 3.0) * gamma * dt * px**2) * (1.0 + (2.0 / 3.0) * gamma * dt * py**2))
    return cb + np.real(np.fft.ifft2(vh))


def circulant_solve(first_col: np.ndarray, f: np.ndarray) -> np.ndarray:
    """Solve C x = f for the circulant C whose first column is ``first_col`` (axis 0 of f)."""
    lam = np.fft.fft(first_col)
    fh = np.fft.fft(f, axis=0)
    if f.ndim == 2:
        lam = lam[:, None]
    return np.real(np.fft.ifft(fh / lam, axis=0))


def dense_cyclic_penta(a, b, c, d, e):
    n = len(c)
    A = np.zeros((n, n))
    for i in range(n):
        for o, v in zip(range(-2, 3), (a, b, c, d, e)):
            A[i, (i + o) % n] += v[i]
    return A


def dense_cyclic_tri(a, b, c):
    n = len(b)
    A = np.zeros((n, n))
    for i in range(n):
        for o, v in zip(range(-1, 2), (a, b, c)):
            A[i, (i + o) % n] += v[i]
    return A


def penta_matvec_interleaved(a, b, c, d, e, x, batch):
    """y = A x for interleaved batches, via array shifts (coefficient arrays shared or per system)."""
    n = x.size // batch
    X = x.reshape(n, batch)
    co = []
    for v in (a, b, c, d, e):
        v = np.asarray(v, dtype=np.float64)
        co.append(v.reshape(n, batch) if v.size == n * batch else v.reshape(n, 1))
    y = np.zeros_like(X)
    for o, v in zip(range(-2, 3), co):
        y += v * np.roll(X, -o, axis=0)
    return y.ravel()


def tri_matvec_interleaved(a, b, c, x, batch):
    n = x.size // batch
    X = x.reshape(n, batch)
    co = []
    for v in (a, b, c):
        v = np.asarray(v, dtype=np.float64)
        co.append(v.reshape(n, batch) if v.size == n * batch else v.reshape(n, 1))
    y = np.zeros_like(X)
    for o, v in zip(range(-1, 2), co):
        y += v * np.roll(X, -o, axis=0)
    return y.ravel()
