"""Pins for the CPU oracle: each check compares it with something other than itself.

- cyclic band solves: dense LU with partial pivoting (numpy.linalg.solve, brute
  force), circulant FFT solves for constant coefficients, residuals computed by
  array shifts;
- stencil: exactness on polynomials, the Fourier symbol on periodic modes,
  an array-shift formulation on random asymmetric boxes;
- ADI step (Eq. 3.1): the spectral form of the whole step, the closed-form
  single-mode recurrence of the linearised scheme and its continuum limit
  sigma(k) = k^2 - gamma k^4, mass conservation, odd symmetry (bit exact),
  shift and transpose equivariance, constant states;
- diagnostics: closed-form discrete sums.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import spectral

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# --------------------------------------------------------------------------- penta
@pytest.mark.parametrize("n", [5, 6, 7, 8, 13, 32, 64])
def test_penta_matches_dense_lu(n):
    batch = 3
    a, b, c, d, e = synth.diag_dominant_penta(11 + n, n, batch)
    f = synth.uniform(7 + n, n * batch, -1.0, 1.0)
    x = oracle.penta_cyclic_batch(a, b, c, d, e, f, batch)
    for s in range(batch):
        co = [v.reshape(n, batch)[:, s] for v in (a, b, c, d, e)]
        A = spectral.dense_cyclic_penta(*co)
        ref = np.linalg.solve(A, f.reshape(n, batch)[:, s])
        got = x.reshape(n, batch)[:, s]
        assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_penta_shared_coefficients_dense():
    n, batch = 24, 5
    a, b, c, d, e = synth.diag_dominant_penta(3, n, 1)
    f = synth.uniform(4, n * batch, -1.0, 1.0)
    x = oracle.penta_cyclic_batch(a, b, c, d, e, f, batch)
    A = spectral.dense_cyclic_penta(a, b, c, d, e)
    ref = np.linalg.solve(A, f.reshape(n, batch))
    assert np.max(np.abs(x.reshape(n, batch) - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("n,sigma", [(16, 0.3), (256, 18.4), (1024, 7.05e3), (512, 1.9e4)])
def test_penta_constant_matches_circulant_fft(n, sigma):
    # The ADI matrix (sigma, -4 sigma, 1 + 6 sigma, -4 sigma, sigma) (eq:1d_hyper_scheme).
    batch = 4
    co = [np.full(n, v) for v in (sigma, -4 * sigma, 1 + 6 * sigma, -4 * sigma, sigma)]
    f = synth.uniform(5, n * batch, -1.0, 1.0)
    x = oracle.penta_cyclic_batch(*co, f, batch).reshape(n, batch)
    col = np.zeros(n)
    col[0], col[1], col[2], col[-1], col[-2] = 1 + 6 * sigma, -4 * sigma, sigma, -4 * sigma, sigma
    ref = spectral.circulant_solve(col, f.reshape(n, batch))
    # forward error of an LU solve grows with cond(A) ~ 1 + 16 sigma
    tol = 1e-15 * (1 + 16 * sigma) * 50
    assert np.max(np.abs(x - ref)) <= tol * np.max(np.abs(ref))


def test_penta_large_residual_per_system():
    n, batch = 1024, 16
    a, b, c, d, e = synth.diag_dominant_penta(2, n, batch)
    f = synth.uniform(1, n * batch, -1.0, 1.0)
    x = oracle.penta_cyclic_batch(a, b, c, d, e, f, batch)
    res = spectral.penta_matvec_interleaved(a, b, c, d, e, x, batch) - f
    assert np.max(np.abs(res)) <= 1e-14 * np.max(np.abs(f)) * 10


def test_penta_detects_swapped_diagonals():
    # a plausible slip (a <-> e) must change the answer on non-symmetric rows
    n = 16
    a, b, c, d, e = synth.diag_dominant_penta(9, n, 1)
    f = synth.uniform(9, n, -1, 1)
    x1 = oracle.penta_cyclic_solve(a, b, c, d, e, f)
    x2 = oracle.penta_cyclic_solve(e, b, c, d, a, f)
    assert np.max(np.abs(x1 - x2)) > 1e-3


def test_penta_singular_reported():
    n = 8
    z = np.zeros(n)
    with pytest.raises(oracle.OracleError):
        oracle.penta_cyclic_solve(z, z, z, z, z, np.ones(n))


# --------------------------------------------------------------------------- tri
@pytest.mark.parametrize("n", [3, 4, 5, 9, 33, 64])
def test_tri_matches_dense_lu(n):
    batch = 3
    a, b, c = synth.diag_dominant_tri(21 + n, n, batch)
    f = synth.uniform(8 + n, n * batch, -1.0, 1.0)
    x = oracle.tri_cyclic_batch(a, b, c, f, batch)
    for s in range(batch):
        co = [v.reshape(n, batch)[:, s] for v in (a, b, c)]
        ref = np.linalg.solve(spectral.dense_cyclic_tri(*co), f.reshape(n, batch)[:, s])
        got = x.reshape(n, batch)[:, s]
        assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("n,sigma", [(64, 0.5), (1024, 8.5e3)])
def test_tri_constant_matches_circulant_fft(n, sigma):
    # periodic Crank-Nicolson diffusion matrix (-sigma, 1 + 2 sigma, -sigma) (eq5:1ddiffscheme)
    batch = 3
    f = synth.uniform(6, n * batch, -1.0, 1.0)
    x = oracle.tri_cyclic_batch(np.full(n, -sigma), np.full(n, 1 + 2 * sigma), np.full(n, -sigma), f, batch)
    col = np.zeros(n)
    col[0], col[1], col[-1] = 1 + 2 * sigma, -sigma, -sigma
    ref = spectral.circulant_solve(col, f.reshape(n, batch))
    tol = 1e-15 * (1 + 4 * sigma) * 50
    assert np.max(np.abs(x.reshape(n, batch) - ref)) <= tol * np.max(np.abs(ref))


def test_tri_large_residual():
    n, batch = 1024, 8
    a, b, c = synth.diag_dominant_tri(4, n, batch)
    f = synth.uniform(3, n * batch, -1.0, 1.0)
    x = oracle.tri_cyclic_batch(a, b, c, f, batch)
    res = spectral.tri_matvec_interleaved(a, b, c, x, batch) - f
    assert np.max(np.abs(res)) <= 1e-14 * np.max(np.abs(f)) * 10


# --------------------------------------------------------------------------- stencil
def _lap5(h):
    return np.array([[0, 1, 0], [1, -4, 1], [0, 1, 0]], dtype=float) / h**2


def test_stencil_laplacian_exact_on_quadratics():
    nx, ny, h = 20, 17, 0.1
    y, x = np.meshgrid(np.arange(ny) * h, np.arange(nx) * h, indexing="ij")
    f = 1.5 * x**2 + 3 * x * y - 2 * y**2 + x - 4 * y + 0.5
    out = oracle.stencil_apply_2d(f, _lap5(h), 1, 1, 1, 1, periodic=False)
    inner = out[1:-1, 1:-1]
    assert np.allclose(inner, 3.0 - 4.0, atol=1e-9)
    # the untouched border stays at the incoming value (zeros here)
    assert np.all(out[0, :] == 0) and np.all(out[:, -1] == 0)


def test_stencil_biharmonic_exact_on_quartics():
    # 13-point biharmonic (dxxxx + 2 dxxyy + dyyyy) is exact on quartic polynomials
    nx, ny, h = 16, 15, 0.5
    w = np.zeros((5, 5))
    w[2, :] += np.array([1, -4, 6, -4, 1])
    w[:, 2] += np.array([1, -4, 6, -4, 1])
    w[1:4, 1:4] += 2 * np.array([[1, -2, 1], [-2, 4, -2], [1, -2, 1]])
    w /= h**4
    y, x = np.meshgrid(np.arange(ny) * h, np.arange(nx) * h, indexing="ij")
    f = x**4 + 2 * x**2 * y**2 - 3 * y**4 + x**3 * y + 5 * x * y
    # d4/dx4 = 24, 2 d4/dx2dy2 = 2*8 = 16, d4/dy4 = -72
    out = oracle.stencil_apply_2d(f, w, 2, 2, 2, 2, periodic=False)
    assert np.allclose(out[2:-2, 2:-2], 24 + 16 - 72, rtol=0, atol=1e-8)


@pytest.mark.parametrize("kx,ky", [(1, 0), (3, 2), (7, 5)])
def test_stencil_periodic_fourier_symbol(kx, ky):
    nx, ny = 32, 24
    lx, ly = 2 * np.pi, 3.0
    dx, dy = lx / nx, ly / ny
    y, x = np.meshgrid(np.arange(ny) * dy, np.arange(nx) * dx, indexing="ij")
    th = 2 * np.pi * (kx * x / lx + ky * y / ly)
    f = np.cos(th)
    w = np.array([[0, 1 / dy**2, 0], [1 / dx**2, -2 / dx**2 - 2 / dy**2, 1 / dx**2], [0, 1 / dy**2, 0]])
    out = oracle.stencil_apply_2d(f, w, 1, 1, 1, 1)
    sym = -4 * np.sin(np.pi * kx / nx) ** 2 / dx**2 - 4 * np.sin(np.pi * ky / ny) ** 2 / dy**2
    assert np.max(np.abs(out - sym * f)) <= 1e-12 * max(1.0, abs(sym))


def test_stencil_asymmetric_box_matches_shifts():
    nx, ny = 19, 11
    left, right, top, bottom = 3, 1, 0, 2
    f = synth.field(5, ny, nx, -1, 1)
    w = synth.uniform(6, (top + bottom + 1) * (left + right + 1), -1, 1).reshape(top + bottom + 1, -1)
    for premap in (False, True):
        out = oracle.stencil_apply_2d(f, w, left, right, top, bottom, premap=premap)
        g = f**3 - f if premap else f
        ref = np.zeros_like(f)
        for dj in range(-top, bottom + 1):
            for di in range(-left, right + 1):
                ref += w[dj + top, di + left] * np.roll(np.roll(g, -dj, axis=0), -di, axis=1)
        assert np.max(np.abs(out - ref)) <= 1e-14 * 20


def test_stencil_premap_constant_field():
    f = np.full((9, 10), 0.7)
    w = np.arange(9, dtype=float).reshape(3, 3)
    out = oracle.stencil_apply_2d(f, w, 1, 1, 1, 1, premap=True)
    assert np.allclose(out, (0.7**3 - 0.7) * w.sum(), rtol=1e-14)


# --------------------------------------------------------------------------- ch_step
def test_ch_step_matches_spectral_form():
    ny, nx = 24, 32
    lx, ly, gamma, dt = 2 * np.pi, 1.7 * np.pi, 0.01, 1e-3
    cn = synth.field(0, ny, nx, -0.1, 0.1)
    cp = synth.field(1, ny, nx, -0.1, 0.1)
    got, prev = oracle.ch_step(cn, cp, lx, ly, gamma, dt)
    ref = spectral.ch_step_spectral(cn, cp, lx, ly, gamma, dt)
    assert np.array_equal(prev, cn)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_ch_step_stiff_matches_spectral_form():
    # large a' (stiff implicit part), non-square and anisotropic spacing
    ny, nx = 40, 64
    lx, ly, gamma, dt = 2 * np.pi, np.pi, 0.005, 5e-3
    cn = synth.field(2, ny, nx, -0.6, 0.6)
    cp = cn + 0.01 * synth.field(3, ny, nx, -1, 1)
    got, _ = oracle.ch_step(cn, cp, lx, ly, gamma, dt)
    ref = spectral.ch_step_spectral(cn, cp, lx, ly, gamma, dt)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def _amplification(kx, ky, nx, ny, lx, ly, gamma, dt):
    dx, dy = lx / nx, ly / ny
    px = 4 * np.sin(np.pi * kx / nx) ** 2 / dx**2
    py = 4 * np.sin(np.pi * ky / ny) ** 2 / dy**2
    lam = -(px + py)
    g = (2 / 3) * gamma * dt
    P = (1 + g * px**2) * (1 + g * py**2)
    A = 2 + (-2 / 3 - 2 * g * lam**2 - (2 / 3) * dt * lam) / P
    B = -1 + (2 / 3 + g * lam**2) / P
    return A, B


@pytest.mark.parametrize("kx,ky", [(0, 0), (1, 0), (2, 3), (5, 4), (9, 1)])
def test_ch_step_linear_mode_closed_form(kx, ky):
    # single small mode: the cubic term is O(eps^3), so amplitudes follow
    # c^{n+1} = A c^n + B c^{n-1} with A, B from the symbols of the scheme
    nx, ny, lx, ly, gamma, dt, eps = 32, 24, 2 * np.pi, 2 * np.pi, 0.01, 2e-3, 1e-8
    y, x = np.meshgrid(np.arange(ny) * ly / ny, np.arange(nx) * lx / nx, indexing="ij")
    mode = np.cos(kx * x * 2 * np.pi / lx + ky * y * 2 * np.pi / ly)
    cn = eps * mode
    cp = cn.copy()
    A, B = _amplification(kx, ky, nx, ny, lx, ly, gamma, dt)
    an, ap = eps, eps
    for _ in range(25):
        cn, cp = oracle.ch_step(cn, cp, lx, ly, gamma, dt)
        an, ap = A * an + B * ap, an
        assert np.max(np.abs(cn - an * mode)) <= 1e-11 * max(abs(an), eps)
    if kx == 0 and ky == 0:
        assert A == pytest.approx(4 / 3) and B == pytest.approx(-1 / 3)


@pytest.mark.parametrize("k", [1, 3, 5, 7, 10])
def test_linear_growth_rate_continuum_limit(k):
    # dominant root of l^2 = A l + B approaches exp(sigma dt), sigma = k^2 - gamma k^4
    nx = ny = 512
    gamma, dt = 0.01, 1e-5
    A, B = _amplification(k, 0, nx, ny, 2 * np.pi, 2 * np.pi, gamma, dt)
    lam = (A + np.sqrt(A * A + 4 * B)) / 2
    sigma = k**2 - gamma * k**4
    # O(dx^2, dt) discretisation error, measured against the size of the terms (k^2)
    assert abs(np.log(lam) / dt - sigma) <= 2e-3 * k**2


def test_ch_mass_conserved_and_energy_decays():
    ny = nx = 48
    lx = ly = 2 * np.pi
    gamma, dt = 0.01, 1e-3
    c0 = synth.field(0, ny, nx, -0.1, 0.1) + 0.05
    m0, e0 = oracle.ch_diagnostics(c0, lx, ly, gamma)
    cn, cp = oracle.ch_run(c0, c0, lx, ly, gamma, dt, 200)
    m1, e1 = oracle.ch_diagnostics(cn, lx, ly, gamma)
    scale = np.sum(np.abs(c0)) * (lx / nx) * (ly / ny)
    assert abs(m1 - m0) <= 1e-13 * scale * 10
    assert e1 < e0


def test_ch_odd_symmetry_bit_exact():
    ny, nx = 16, 20
    cn = synth.field(4, ny, nx, -0.5, 0.5)
    cp = synth.field(5, ny, nx, -0.5, 0.5)
    a, _ = oracle.ch_run(cn, cp, 2 * np.pi, 2 * np.pi, 0.01, 1e-3, 3)
    b, _ = oracle.ch_run(-cn, -cp, 2 * np.pi, 2 * np.pi, 0.01, 1e-3, 3)
    assert np.array_equal(a, -b)


def test_ch_shift_and_transpose_equivariance():
    n = 24
    cn = synth.field(6, n, n, -0.5, 0.5)
    cp = cn.copy()
    args = (2 * np.pi, 2 * np.pi, 0.01, 1e-3)
    base, _ = oracle.ch_run(cn, cp, *args, 4)
    sh, _ = oracle.ch_run(np.roll(cn, (3, -5), (0, 1)), np.roll(cp, (3, -5), (0, 1)), *args, 4)
    assert np.max(np.abs(np.roll(base, (3, -5), (0, 1)) - sh)) <= 1e-13
    tr, _ = oracle.ch_run(cn.T.copy(), cp.T.copy(), *args, 4)
    assert np.max(np.abs(base.T - tr)) <= 1e-13


def test_ch_constant_state_is_fixed():
    c = np.full((12, 10), 0.3)
    got, _ = oracle.ch_run(c, c, 2 * np.pi, 2 * np.pi, 0.01, 1e-3, 5)
    assert np.max(np.abs(got - 0.3)) <= 1e-15


# --------------------------------------------------------------------------- diagnostics
def test_diagnostics_closed_forms():
    nx, ny, lx, ly, gamma = 64, 32, 2 * np.pi, 1.0, 0.02
    dx, dy = lx / nx, ly / ny
    m, e = oracle.ch_diagnostics(np.ones((ny, nx)), lx, ly, gamma)
    assert m == pytest.approx(lx * ly, rel=1e-14) and e == 0.0
    amp, k = 0.8, 3
    th = 2 * np.pi * k * np.arange(nx) / nx
    c = np.tile(amp * np.cos(th), (ny, 1))
    m, e = oracle.ch_diagnostics(c, lx, ly, gamma)
    assert abs(m) <= 1e-13
    # sum cos^2 = n/2, sum cos^4 = 3n/8 (k not 0, n/4, n/2); sum (c_{i+1}-c_i)^2 = amp^2 n (1 - cos(2 pi k/n))
    bulk = 0.25 * ny * (amp**4 * 3 * nx / 8 - 2 * amp**2 * nx / 2 + nx)
    grad = 0.5 * gamma * ny * amp**2 * nx * (1 - np.cos(2 * np.pi * k / nx)) / dx**2
    assert e == pytest.approx((bulk + grad) * dx * dy, rel=1e-12)


def test_synth_torch_matches_numpy():
    torch = pytest.importorskip("torch")
    a = synth.uniform(123, 1000, -1, 1, offset=17)
    b = synth.uniform_torch(123, 1000, -1, 1, device="cpu", offset=17).numpy()
    assert np.array_equal(a, b)


# --------------------------------------------------------------------------- 1D Cahn-Hilliard (Sec. 6.2.1)
def test_ch1d_linear_mode_closed_form():
    # small single mode: N(c) ~ -c, so each step multiplies the mode by
    # G = (1 + dt p) / (1 + gamma dt p^2), p = 4 sin^2(k dx / 2) / dx^2
    n, l, gamma, dt, eps, k = 64, 2 * np.pi, 0.01, 1e-3, 1e-8, 5
    x = np.arange(n) * l / n
    batch = 3
    c = np.repeat((eps * np.cos(k * x))[:, None], batch, axis=1).ravel()
    dx = l / n
    p = 4 * np.sin(k * dx / 2) ** 2 / dx**2
    G = (1 + dt * p) / (1 + gamma * dt * p**2)
    got = oracle.ch1d_run(c, l, gamma, dt, 20, batch).reshape(n, batch)
    ref = eps * G**20 * np.cos(k * x)
    for s in range(batch):
        assert np.max(np.abs(got[:, s] - ref)) <= 1e-11 * eps * G**20


def test_ch1d_spatial_order_two_against_continuum():
    # linear regime, tiny dt: error against eps e^{sigma t} cos(kx), sigma = k^2 - gamma k^4,
    # falls as N^-2 (the O(dx^2) differencing of the scheme)
    l, gamma, eps, k, T, dt = 2 * np.pi, 0.01, 1e-8, 3, 0.02, 1e-5
    sig = k**2 - gamma * k**4
    errs = []
    for n in (32, 64, 128):
        x = np.arange(n) * l / n
        got = oracle.ch1d_run(eps * np.cos(k * x), l, gamma, dt, int(round(T / dt)))
        errs.append(np.max(np.abs(got - eps * np.exp(sig * T) * np.cos(k * x))) / eps)
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(orders - 2.0) < 0.1), orders


def test_ch1d_mass_conservation():
    n, batch = 48, 4
    c = synth.uniform(3, n * batch, -0.1, 0.1) + 0.02
    got = oracle.ch1d_run(c, 2 * np.pi, 0.01, 2e-3, 100, batch)
    m0 = c.reshape(n, batch).sum(0)
    m1 = got.reshape(n, batch).sum(0)
    assert np.max(np.abs(m1 - m0)) <= 1e-13 * np.abs(c).reshape(n, batch).sum(0).max()


# --------------------------------------------------------------------------- CN benchmarks (Secs. 4.2, 5.3)
def _golden(name):
    import os

    vals = {}
    for ln in open(os.path.join(os.path.dirname(__file__), "golden", name)):
        if ln.strip() and not ln.startswith("#"):
            k, v = ln.split()
            vals[k] = float(v)
    return vals


def test_cn_hyperdiffusion_exact_solution_slope():
    # the paper's validation (Eq. exact, Eq. myerr): slope of the L2 error vs N
    g = _golden("hyperdiffusion_slope.txt")
    T, dt, wave = g["T"], g["dt"], int(g["wave"])
    k = 2 * np.pi * wave
    steps = int(round(T / dt))
    errs, ns = [], [16, 32, 64]
    for n in ns:
        x = np.arange(n) / n
        got = oracle.cn1d_run(4, np.cos(k * x), 1.0, 1.0, dt, steps)
        exact = np.exp(-k**4 * T) * np.cos(k * x)
        errs.append(np.sqrt(np.mean((got - exact) ** 2)))
    slope = np.polyfit(np.log(ns), np.log(errs), 1)[0]
    assert abs(slope - g["slope"]) < 0.05, slope


def test_cn_diffusion_exact_solution_order_two():
    k, T, dt = 2 * np.pi * 3, 1e-3, 1e-6
    errs = []
    for n in (32, 64, 128):
        x = np.arange(n) / n
        got = oracle.cn1d_run(2, np.cos(k * x), 1.0, 1.0, dt, int(round(T / dt)))
        errs.append(np.max(np.abs(got - np.exp(-k**2 * T) * np.cos(k * x))))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(orders - 2.0) < 0.05), orders


@pytest.mark.parametrize("order", [2, 4])
def test_cn_mode_amplification_closed_form(order):
    # CN multiplies a Fourier mode by (1 - s)/(1 + s), s = sigma * symbol
    n, l, kappa, dt, kk = 40, 1.0, 0.7, 2e-4, 3
    x = np.arange(n) / n
    dx = l / n
    th = 2 * np.pi * kk / n
    sym = (2 - 2 * np.cos(th)) ** (order // 2)
    sig = kappa * dt / (2 * dx**order)
    G = (1 - sig * sym) / (1 + sig * sym)
    got = oracle.cn1d_run(order, np.cos(2 * np.pi * kk * x), l, kappa, dt, 10)
    assert np.max(np.abs(got - G**10 * np.cos(2 * np.pi * kk * x))) <= 1e-12


# --------------------------------------------------------------------------- Cahn-Hilliard-Cook (Sec. 7.7)
@pytest.mark.parametrize("key,ctr", [((5, 7), (0, 0, 0, 0)), ((0, 0), (41, 3, 0, 0)),
                                     ((2**64 - 1, 12345), (2**64 - 1, 5, 9, 0))])
def test_philox4x64_matches_numpy(key, ctr):
    # numpy's Philox bit generator is Philox4x64-10; it advances its 256-bit
    # counter by one before producing each block of four words
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(ctr, dtype=np.uint64))
    ref = [int(v) for v in bg.random_raw(12)]
    c = list(ctr)
    for blk in range(3):
        c[0] += 1
        for w in range(3):  # carry into the next word
            if c[w] == 2**64:
                c[w] = 0
                c[w + 1] += 1
        assert oracle.philox4x64(c, key) == ref[4 * blk:4 * blk + 4]


def test_noise_normals_are_standard_normal():
    from scipy import stats

    nx = ny = 256
    z = np.concatenate([oracle.noise_normals(nx, ny, 2021, 3, step).reshape(2, -1) for step in range(4)], axis=1)
    n = z.shape[1]
    for comp in z:
        assert abs(comp.mean()) < 5 / np.sqrt(n)
        assert abs(comp.var() - 1.0) < 5 * np.sqrt(2.0 / n)
        assert stats.kstest(comp, "norm").pvalue > 1e-3
    assert abs(np.corrcoef(z[0], z[1])[0, 1]) < 5 / np.sqrt(n)
    # different steps, simulations and seeds give unrelated deviates
    a = oracle.noise_normals(64, 64, 1, 0, 0).ravel()
    for other in (oracle.noise_normals(64, 64, 1, 0, 1), oracle.noise_normals(64, 64, 1, 1, 0),
                  oracle.noise_normals(64, 64, 2, 0, 0)):
        assert abs(np.corrcoef(a, other.ravel())[0, 1]) < 5 / np.sqrt(a.size)
    # odd point count: the last pair is half used; the rest is unchanged
    odd = oracle.noise_normals(7, 5, 9, 0, 0).reshape(2, -1)
    full = oracle.noise_normals(6, 6, 9, 0, 0).reshape(2, -1)
    assert np.array_equal(odd[:, :35], full[:, :35])


def test_cook_forcing_conserves_mass_and_has_laplacian_covariance():
    nx, ny, lx, ly, dt, sigma = 96, 64, 2 * np.pi, 1.5 * np.pi, 1e-3, 1e-14
    dx, dy = lx / nx, ly / ny
    amp2 = sigma / (dx * dy * dt)
    etas = np.stack([oracle.cook_forcing(oracle.noise_normals(nx, ny, 77, 0, s), lx, ly, dt, sigma)
                     for s in range(40)])
    scale = np.sqrt(amp2) / min(dx, dy)
    assert np.max(np.abs(etas.sum(axis=(1, 2)))) <= 1e-12 * scale * nx * ny
    var = np.mean(etas**2)
    cx = np.mean(etas * np.roll(etas, -1, axis=2))
    cy = np.mean(etas * np.roll(etas, -1, axis=1))
    cd = np.mean(etas * np.roll(np.roll(etas, -1, axis=2), -1, axis=1))
    # <eta eta'> = -sigma/(dx dy dt) * (5-point Laplacian of the Kronecker delta)
    assert var == pytest.approx(amp2 * (2 / dx**2 + 2 / dy**2), rel=0.03)
    assert cx == pytest.approx(-amp2 / dx**2, rel=0.06)
    assert cy == pytest.approx(-amp2 / dy**2, rel=0.06)
    assert abs(cd) < 0.03 * var
    # a unit deviate at one point is a dipole along its own axis
    rho = np.zeros((2, ny, nx))
    rho[0, 5, 9] = 1.0
    eta = oracle.cook_forcing(rho, lx, ly, dt, sigma)
    want = np.zeros((ny, nx))
    want[5, 9], want[5, 10] = np.sqrt(amp2) / dx, -np.sqrt(amp2) / dx
    assert np.allclose(eta, want, rtol=1e-15, atol=0)


def test_cook_step_from_rest_matches_fourier_solution():
    # from C = 0 the nonlinear and biharmonic terms vanish: the step is
    # C^1 = (I + a dxxxx)^{-1} (I + a dyyyy)^{-1} (2/3) dt eta, evaluated here with
    # the backward-difference divergence written as a Fourier multiplier
    nx, ny, lx, ly, gamma, dt, sigma = 48, 40, 2 * np.pi, 2.5, 0.01, 2e-3, 1e-6
    dx, dy = lx / nx, ly / ny
    rho = oracle.noise_normals(nx, ny, 5, 1, 0)
    zero = np.zeros((ny, nx))
    got, prev = oracle.ch_cook_step(zero, zero, rho, lx, ly, gamma, dt, sigma)
    assert np.array_equal(prev, zero)
    tx = 2 * np.pi * np.fft.fftfreq(nx)[None, :]
    ty = 2 * np.pi * np.fft.fftfreq(ny)[:, None]
    amp = np.sqrt(sigma / (dx * dy * dt))
    eta_h = amp * ((1 - np.exp(-1j * tx)) / dx * np.fft.fft2(rho[0]) + (1 - np.exp(-1j * ty)) / dy * np.fft.fft2(rho[1]))
    px = spectral.second_diff_symbol(nx, dx)[None, :]
    py = spectral.second_diff_symbol(ny, dy)[:, None]
    a = (2.0 / 3.0) * gamma * dt
    want = np.real(np.fft.ifft2((2.0 / 3.0) * dt * eta_h / ((1 + a * px**2) * (1 + a * py**2))))
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def test_cook_step_without_noise_is_the_plain_step_and_conserves_mass():
    n, l, gamma, dt = 32, 2 * np.pi, 0.02, 1e-3
    c0 = synth.field(4, n, n, -0.1, 0.1)
    rho = oracle.noise_normals(n, n, 1, 0, 0)
    a, _ = oracle.ch_cook_step(c0, c0, rho, l, l, gamma, dt, 0.0)
    b, _ = oracle.ch_run(c0, c0, l, l, gamma, dt, 1)
    assert np.array_equal(a, b)
    c, cp = oracle.ch_cook_run(c0, c0, l, l, gamma, dt, 1e-6, 8, 0, 0, 6)
    assert abs(c.sum() - c0.sum()) <= 1e-13 * np.abs(c0).sum()
    assert np.max(np.abs(c - c0)) > 1e-6  # the forcing acted


# --------------------------------------------------------------------------- coarsening observables (Secs. 3.5.4, 7.2.3)
def test_simpson_mean_is_scipy_simpson_on_the_closed_interval():
    from scipy.integrate import simpson

    ny, nx, lx, ly = 24, 40, 2.0, 3.0
    v = synth.field(8, ny, nx, -1, 1)
    closed = np.concatenate([v, v[:1]], axis=0)
    closed = np.concatenate([closed, closed[:, :1]], axis=1)
    x = np.linspace(0, lx, nx + 1)
    y = np.linspace(0, ly, ny + 1)
    want = simpson(simpson(closed, x=x, axis=1), x=y) / (lx * ly)
    assert oracle.simpson_mean(v) == pytest.approx(want, rel=1e-14, abs=1e-15)
    # odd counts fall back to the trapezoid rule: the plain mean
    w = synth.field(9, 15, 9, -1, 1)
    assert oracle.simpson_mean(w) == pytest.approx(w.mean(), rel=1e-14)


def test_s_of_t_closed_forms():
    n = 64
    x = np.arange(n) * 2 * np.pi / n
    c = 0.8 * np.cos(3 * x)[None, :] * np.ones((n, 1))
    assert oracle.s_of_t(c) == pytest.approx(1.0 / (1.0 - 0.32), rel=1e-14)  # <C^2> = A^2 / 2
    assert oracle.s_of_t(np.zeros((8, 8))) == 1.0
    tanh = np.tanh(5 * np.sin(x))[None, :] * np.ones((4, 1))  # sharp interfaces: <C^2> -> 1, s grows
    assert oracle.s_of_t(tanh) > 5


def test_k1_closed_forms():
    ny, nx, lx, ly = 48, 64, 2 * np.pi, 3.0
    x = np.arange(nx) * lx / nx
    y = np.arange(ny) * ly / ny
    X, Y = np.meshgrid(x, y)
    k = 5.0
    assert oracle.k1_of_t(0.3 + np.cos(k * X), lx, ly) == pytest.approx(k, rel=1e-13)  # the mean is left out
    ky = 2 * np.pi * 4 / ly
    kk = np.hypot(2.0, ky)
    assert oracle.k1_of_t(np.sin(2 * X + ky * Y), lx, ly) == pytest.approx(kk, rel=1e-13)
    a, b, ka, kb = 1.0, 0.5, 3.0, 7.0
    c = a * np.cos(ka * X) + b * np.sin(kb * X)
    assert oracle.k1_of_t(c, lx, ly) == pytest.approx((a * a + b * b) / (a * a / ka + b * b / kb), rel=1e-13)


def test_coarsening_rate_closed_forms():
    # F ~ t^-1/3 (the LSW law) has beta = 1/3; the error falls as h^2 inside and at the ends
    errs = []
    for m in (91, 181, 361):
        t = np.linspace(10, 100, m)
        errs.append(np.abs(oracle.coarsening_rate(t, 3.0 * t ** (-1 / 3)) - 1 / 3)[[0, m // 2, -1]])
    errs = np.array(errs)
    assert np.all(errs[0] < 4e-3)
    assert np.all(np.abs(np.log2(errs[1:-1] / errs[2:]) - 2) < 0.1)  # asymptotic by the finest pair
    t = np.linspace(10, 100, 181)
    assert np.allclose(oracle.coarsening_rate(t, np.exp(-0.01 * t)), 0.01 * t, rtol=1e-4)
    # uneven sampling: second order, exact on quadratics
    tu = np.sort(synth.uniform(4, 40, 1.0, 2.0))
    F = 5 + tu - 0.5 * tu**2
    assert np.allclose(oracle.coarsening_rate(tu, F), -(tu / F) * (1 - tu), rtol=1e-9)


def _table(name):
    """Rows of a printed table: {N: (E_N, order, half a unit of E_N's last printed digit)}."""
    import decimal
    import os

    rows = {}
    for ln in open(os.path.join(os.path.dirname(__file__), "golden", name)):
        if ln.strip() and not ln.startswith("#"):
            n, e, o = ln.split()
            half = 0.5 * 10.0 ** decimal.Decimal(e).as_tuple().exponent
            rows[int(n)] = (float(e), float(o), half)
    return rows


def _steps_to(t_end, dt):
    # the studies run whole steps until t >= T (reading: rounding the step count
    # down or to nearest misses the printed N = 128 rows in their last digit)
    return int(np.ceil(t_end / dt - 1e-9))


def test_ch1d_convergence_reproduces_the_paper_table():
    # Table table5:converge1D: the oracle's 1D scheme (Sec. 6.2.1) on the printed
    # study, measured by Eq. eq2:converge1D.  The final time is not printed; t = 20
    # reproduces every printed E_N from N = 128 to 512 to its last digit and the
    # observed orders to four decimals.
    rows = _table("table_converge1d.txt")
    l, gamma, t_end, eps = 2 * np.pi, 0.01, 20.0, 1e-6
    res = {}
    for n in (64, 128, 256, 512, 1024):
        x = np.arange(n) * l / n
        dt = 0.1 * l / n
        res[n] = oracle.ch1d_run(eps * np.cos(5 * x), l, gamma, dt, _steps_to(t_end, dt), 1)
    e = {n: oracle.refinement_error_1d(res[n], res[n // 2]) for n in (128, 256, 512, 1024)}
    for n in (128, 256, 512):
        printed, order, half = rows[n]
        assert abs(e[n] - printed) <= half, (n, e[n], printed)
        assert abs(np.log2(e[n] / e[2 * n]) - order) <= 2e-4, (n, np.log2(e[n] / e[2 * n]), order)


def test_ch2d_convergence_reproduces_the_paper_table():
    # Table table:converge2D, N = 128 row: the oracle's ADI step (Eq. 3.1) on the
    # printed study (Sec. 3.5.3), measured by Eq. eq2:converge2D, matches the
    # printed E_N to its last digit.  The GPU tests carry the study to N = 1024.
    rows = _table("table_converge2d.txt")
    l, gamma, t_end, eps = 2 * np.pi, 0.01, 10.0, 1e-6
    f = {}
    for n in (64, 128):
        x = np.arange(n) * l / n
        xx, yy = np.meshgrid(x, x)
        c0 = eps * np.tanh(np.sqrt((xx - np.pi) ** 2 + (yy - np.pi) ** 2) - np.pi)
        dt = 0.1 * l / n
        f[n], _ = oracle.ch_run(c0, c0, l, l, gamma, dt, _steps_to(t_end, dt))
    printed, _, half = rows[128]
    e = oracle.refinement_error_2d(f[128], f[64])
    assert abs(e - printed) <= half, (e, printed)


def test_refinement_errors_on_closed_forms():
    # Eq. eq2:converge1D / eq2:converge2D on functions whose answer is known:
    # identical samplings give 0, a constant offset gives the offset, and the 2x2
    # block average of a linear ramp sits half a fine cell off the coarse point.
    n = 32
    x = np.arange(2 * n) / (2 * n)
    assert oracle.refinement_error_1d(np.sin(2 * np.pi * x), np.sin(2 * np.pi * x[0::2])) == 0.0
    assert abs(oracle.refinement_error_1d(x + 0.25, x[0::2]) - 0.25) < 1e-15
    xx, yy = np.meshgrid(x, x)
    h = 1.0 / (2 * n)
    e2 = oracle.refinement_error_2d(xx + 2 * yy, (xx + 2 * yy)[0::2, 0::2])
    assert abs(e2 - 1.5 * h) < 1e-14
    with pytest.raises(oracle.OracleError):
        oracle.refinement_error_1d(x, x)
