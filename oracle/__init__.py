"""FP64 CPU oracle for the ADI Cahn-Hilliard step and its batched cyclic solvers.

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the benchmark's
CPU-baseline leg may import this; the library never does.  It shares no code
with the CUDA path.  See ``oracle.c`` for the paper passages each function
follows.  All arrays are float64 numpy arrays; layouts match the C ABI
(row-major fields ``c[j, i]``, interleaved batches ``x[i * batch + s]``).

Parity pins: every function is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_pins.py`` against dense solves, circulant FFT solves, closed
forms of the discrete scheme, conservation laws and symmetries.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None
_D = ctypes.POINTER(ctypes.c_double)

ERRORS = {0: "ok", -1: "invalid argument", -2: "singular", -3: "out of memory"}


class OracleError(RuntimeError):
    pass


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        i, l, d = ctypes.c_int, ctypes.c_long, ctypes.c_double
        L.oracle_penta_cyclic_solve.argtypes = [i, _D, _D, _D, _D, _D, l, _D, l, _D, l]
        L.oracle_penta_cyclic_batch.argtypes = [i, i, i, _D, _D, _D, _D, _D, _D, _D]
        L.oracle_tri_cyclic_solve.argtypes = [i, _D, _D, _D, l, _D, l, _D, l]
        L.oracle_tri_cyclic_batch.argtypes = [i, i, i, _D, _D, _D, _D, _D]
        L.oracle_stencil_apply_2d.argtypes = [_D, _D, i, i, i, _D, i, i, i, i, i, i]
        L.oracle_ch_step.argtypes = [i, i, d, d, d, d, _D, _D]
        L.oracle_ch_run.argtypes = [i, i, d, d, d, d, i, _D, _D]
        L.oracle_ch_diagnostics.argtypes = [i, i, d, d, d, _D, _D, _D]
        L.oracle_ch1d_run.argtypes = [i, i, d, d, d, i, _D]
        L.oracle_cn1d_run.argtypes = [i, i, i, d, d, d, i, _D]
        u64, U64 = ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)
        L.oracle_philox4x64.argtypes = [U64, U64, U64]
        L.oracle_philox4x64.restype = None
        L.oracle_noise_normals.argtypes = [i, i, u64, u64, u64, _D]
        L.oracle_cook_forcing.argtypes = [i, i, d, d, d, d, _D, _D]
        L.oracle_ch_cook_step.argtypes = [i, i, d, d, d, d, d, _D, _D, _D]
        L.oracle_ch_cook_run.argtypes = [i, i, d, d, d, d, d, u64, u64, u64, i, _D, _D]
        for fn in ("oracle_penta_cyclic_solve", "oracle_penta_cyclic_batch", "oracle_tri_cyclic_solve",
                   "oracle_tri_cyclic_batch", "oracle_stencil_apply_2d", "oracle_ch_step",
                   "oracle_ch_run", "oracle_ch_diagnostics", "oracle_ch1d_run",
                   "oracle_cn1d_run", "oracle_noise_normals", "oracle_cook_forcing", "oracle_ch_cook_step",
                   "oracle_ch_cook_run"):
            getattr(L, fn).restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _check(rc: int):
    if rc != 0:
        raise OracleError(ERRORS.get(rc, str(rc)))


def penta_cyclic_batch(a, b, c, d, e, f, batch: int):
    """Solve ``batch`` cyclic pentadiagonal systems, interleaved ``f[i*batch + s]``.

    Coefficients of length n are shared by all systems; of length n*batch they
    are per system (interleaved like ``f``).
    """
    f = _f64(f).ravel()
    n = f.size // batch
    co = [_f64(v).ravel() for v in (a, b, c, d, e)]
    mode = 1 if co[0].size == n * batch and batch > 1 else 0
    x = np.empty_like(f)
    _check(lib().oracle_penta_cyclic_batch(n, batch, mode, *[_p(v) for v in co], _p(f), _p(x)))
    return x


def penta_cyclic_solve(a, b, c, d, e, f):
    """One cyclic pentadiagonal system (vectors of length n)."""
    return penta_cyclic_batch(a, b, c, d, e, f, 1)


def tri_cyclic_batch(a, b, c, f, batch: int):
    """Solve ``batch`` cyclic tridiagonal systems, interleaved ``f[i*batch + s]``."""
    f = _f64(f).ravel()
    n = f.size // batch
    co = [_f64(v).ravel() for v in (a, b, c)]
    mode = 1 if co[0].size == n * batch and batch > 1 else 0
    x = np.empty_like(f)
    _check(lib().oracle_tri_cyclic_batch(n, batch, mode, *[_p(v) for v in co], _p(f), _p(x)))
    return x


def tri_cyclic_solve(a, b, c, f):
    return tri_cyclic_batch(a, b, c, f, 1)


def stencil_apply_2d(inp, w, left, right, top, bottom, premap=False, periodic=True, out=None):
    """General box stencil on a (ny, nx) field; ``w`` is (top+bottom+1, left+right+1)."""
    inp = _f64(inp)
    ny, nx = inp.shape
    w = _f64(w)
    assert w.shape == (top + bottom + 1, left + right + 1)
    out = np.zeros_like(inp) if out is None else _f64(out).copy()
    _check(lib().oracle_stencil_apply_2d(_p(inp), _p(out), nx, ny, nx, _p(w), left, right, top, bottom,
                                         int(bool(premap)), int(bool(periodic))))
    return out


def ch_run(c_now, c_prev, lx, ly, gamma, dt, nsteps=1):
    """Advance ``nsteps`` ADI steps; returns (C^{n+nsteps}, C^{n+nsteps-1}) as new arrays."""
    cn = _f64(c_now).copy()
    cp = _f64(c_prev).copy()
    ny, nx = cn.shape
    _check(lib().oracle_ch_run(nx, ny, float(lx), float(ly), float(gamma), float(dt), int(nsteps),
                               _p(cn), _p(cp)))
    return cn, cp


def ch_step(c_now, c_prev, lx, ly, gamma, dt):
    return ch_run(c_now, c_prev, lx, ly, gamma, dt, 1)


def ch_diagnostics(c, lx, ly, gamma):
    """(mass, free energy) of a (ny, nx) field."""
    c = _f64(c)
    ny, nx = c.shape
    m = ctypes.c_double()
    e = ctypes.c_double()
    _check(lib().oracle_ch_diagnostics(nx, ny, float(lx), float(ly), float(gamma), _p(c),
                                       ctypes.byref(m), ctypes.byref(e)))
    return m.value, e.value


def ch1d_run(c, l, gamma, dt, nsteps=1, batch=1):
    """Batched 1D Cahn-Hilliard steps (Sec. 6.2.1) on an interleaved (n * batch) array; returns a new array."""
    c = _f64(c).ravel().copy()
    n = c.size // batch
    _check(lib().oracle_ch1d_run(n, batch, float(l), float(gamma), float(dt), int(nsteps), _p(c)))
    return c


def cn1d_run(order, c, l, kappa, dt, nsteps=1, batch=1):
    """Crank-Nicolson hyperdiffusion (order 4) or diffusion (order 2) steps (Secs. 4.2.1, 5.3.2)."""
    c = _f64(c).ravel().copy()
    n = c.size // batch
    _check(lib().oracle_cn1d_run(int(order), n, batch, float(l), float(kappa), float(dt), int(nsteps), _p(c)))
    return c


def philox4x64(ctr, key):
    """Philox4x64-10 block (Salmon et al., SC 2011): four 64-bit words."""
    U = ctypes.c_uint64
    c, k, o = (U * 4)(*[int(v) for v in ctr]), (U * 2)(*[int(v) for v in key]), (U * 4)()
    lib().oracle_philox4x64(c, k, o)
    return [int(v) for v in o]


def noise_normals(nx, ny, seed, sim, step):
    """Box-Muller deviates (rho^x, rho^y) of one Cahn-Hilliard-Cook step, shape (2, ny, nx)."""
    rho = np.empty(2 * nx * ny)
    _check(lib().oracle_noise_normals(nx, ny, int(seed), int(sim), int(step), _p(rho)))
    return rho.reshape(2, ny, nx)


def cook_forcing(rho, lx, ly, dt, sigma):
    """eta = sqrt(sigma / (dx dy dt)) div_h rho for rho of shape (2, ny, nx) (Sec. 7.7)."""
    rho = _f64(rho)
    _, ny, nx = rho.shape
    eta = np.empty((ny, nx))
    _check(lib().oracle_cook_forcing(nx, ny, float(lx), float(ly), float(dt), float(sigma), _p(rho), _p(eta)))
    return eta


def ch_cook_step(c_now, c_prev, rho, lx, ly, gamma, dt, sigma):
    """One Cahn-Hilliard-Cook ADI step with the given deviates; returns (C^{n+1}, C^n)."""
    cn, cp, rho = _f64(c_now).copy(), _f64(c_prev).copy(), _f64(rho)
    ny, nx = cn.shape
    _check(lib().oracle_ch_cook_step(nx, ny, float(lx), float(ly), float(gamma), float(dt), float(sigma), _p(rho),
                                     _p(cn), _p(cp)))
    return cn, cp


def ch_cook_run(c_now, c_prev, lx, ly, gamma, dt, sigma, seed, sim, step0, nsteps):
    """nsteps Cahn-Hilliard-Cook steps drawing the deviates of steps step0.. ; returns (C, C_prev)."""
    cn, cp = _f64(c_now).copy(), _f64(c_prev).copy()
    ny, nx = cn.shape
    _check(lib().oracle_ch_cook_run(nx, ny, float(lx), float(ly), float(gamma), float(dt), float(sigma), int(seed),
                                    int(sim), int(step0), int(nsteps), _p(cn), _p(cp)))
    return cn, cp


# --------------------------------------------------------------------------- coarsening observables
def simpson_mean(v):
    """Spatial average of a periodic (ny, nx) field by the composite Simpson rule
    (Sec. 3.5.4) in each direction.  Closing the periodic interval [0, L] with
    f(L) = f(0), the rule's weights h/3 (1, 4, 2, ..., 4, 1) fold onto the grid as
    h/3 (2, 4, 2, 4, ...).  Reading: it needs an even number of intervals; for an
    odd count the trapezoid rule (all weights h) is used in that direction."""
    v = _f64(v)

    def weights(n):
        if n % 2:
            return np.ones(n)
        w = np.full(n, 2.0 / 3.0)
        w[1::2] = 4.0 / 3.0
        return w

    ny, nx = v.shape
    return float(np.sum(weights(ny)[:, None] * weights(nx)[None, :] * v) / (nx * ny))


def s_of_t(c):
    """s = 1 / (1 - <C^2>) with <.> the Simpson average (Sec. 3.5.4)."""
    return 1.0 / (1.0 - simpson_mean(_f64(c) ** 2))


def k1_of_t(c, lx, ly):
    """k1 = sum |C^(k)|^2 / sum |k|^-1 |C^(k)|^2 over the discrete Fourier modes (Sec. 3.5.4),
    k = (2 pi mx / lx, 2 pi my / ly).  Reading: the k = 0 mode (the mean, with no
    length scale and an infinite weight |k|^-1) is left out of both sums."""
    c = _f64(c)
    ny, nx = c.shape
    ch = np.fft.fft2(c)
    kx = 2 * np.pi * np.fft.fftfreq(nx, d=lx / nx)[None, :]
    ky = 2 * np.pi * np.fft.fftfreq(ny, d=ly / ny)[:, None]
    kk = np.sqrt(kx**2 + ky**2)
    p = np.abs(ch) ** 2
    mask = kk > 0
    return float(np.sum(p[mask]) / np.sum(p[mask] / kk[mask]))


def observables(c, lx, ly, gamma):
    """(mass, free energy F_h, s, k1) of a (ny, nx) field."""
    m, e = ch_diagnostics(c, lx, ly, gamma)
    return m, e, s_of_t(c), k1_of_t(c, lx, ly)


def coarsening_rate(t, F):
    """beta = -(t / F) dF/dt along a sampled series (Eq. eq7:betaN, Sec. 7.2.3), dF/dt
    from second-order finite differences on the (possibly uneven) sample times:
    three-point central differences inside, three-point one-sided at the ends."""
    t, F = _f64(t), _f64(F)
    return -(t / F) * np.gradient(F, t, edge_order=2)


# --------------------------------------------------------------------------- grid-refinement error
def refinement_error_1d(fine, coarse):
    """E_N of Eq. eq2:converge1D (Sec. 2.1.3): the mean absolute difference between
    a periodic solution on N points and the one on N/2 points, taken at the
    coarse grid's points (fine points 0, 2, 4, ... in 0-based indexing)."""
    fine, coarse = _f64(fine), _f64(coarse)
    if fine.shape[-1] != 2 * coarse.shape[-1]:
        raise OracleError("fine grid must have twice the coarse grid's points")
    return float(np.mean(np.abs(fine[..., 0::2] - coarse)))


def refinement_error_2d(fine, coarse):
    """E_N of Eq. eq2:converge2D (Sec. 2.1.3): the mean absolute difference between
    each coarse point's value and the average of the 2x2 block of fine points
    whose first corner it shares (fine rows and columns 2i, 2i + 1 in 0-based
    indexing), over the (N/2)^2 coarse points."""
    fine, coarse = _f64(fine), _f64(coarse)
    if fine.shape != (2 * coarse.shape[0], 2 * coarse.shape[1]):
        raise OracleError("fine grid must have twice the coarse grid's points in each direction")
    block = 0.25 * (fine[0::2, 0::2] + fine[1::2, 0::2] + fine[0::2, 1::2] + fine[1::2, 1::2])
    return float(np.mean(np.abs(block - coarse)))
