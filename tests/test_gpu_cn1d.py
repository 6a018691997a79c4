"""GPU parity of the batched Crank-Nicolson hyperdiffusion / diffusion steps
(Secs. 4.2.1, 5.3.2) against the oracle, and the exact-solution validation of
Sec. 4.2.4 run on the device."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


def _chx():
    import paper_2101_06550_gb300 as chx

    return chx


def _sigma(order, n, l, kappa, dt):
    dx = l / n
    return kappa * dt / (2 * dx**order)


def _tol(order, sigma, nsteps, scale):
    # per step both sides solve A x = B c in FP64; the difference is rounding,
    # bounded by a small multiple of eps * cond(A) * |c|, cond(A) <= 1 + 16 sigma
    # (order 4) or 1 + 4 sigma (order 2), and it accumulates at most linearly
    kappa_a = 1 + (16 if order == 4 else 4) * sigma
    return max(nsteps, 1) * 64 * EPS * kappa_a * scale


def _run_gpu(order, c_inter, n, batch, l, kappa, dt, steps, rewrite):
    chx = _chx()
    plan = chx.CN1DPlan(order, n, batch, l, kappa, dt, rewrite)
    c = torch.from_numpy(np.ascontiguousarray(c_inter).ravel()).cuda()
    plan.step(c, steps)
    plan.sync_status()
    return c.cpu().numpy().reshape(n, batch)


@pytest.mark.parametrize("rewrite", [False, True])
@pytest.mark.parametrize("order,n,batch,l,kappa,dt", [
    (4, 6, 1, 1.0, 1.0, 1e-5),         # smallest pentadiagonal system, one system
    (4, 37, 131, 1.0, 1.0, 1e-6),       # ragged n (not a multiple of the unroll) and batch
    (4, 256, 300, 2 * np.pi, 0.3, 1e-3),  # stiff: sigma ~ 1.1e4
    (2, 3, 5, 1.0, 1.0, 1e-3),          # smallest tridiagonal system
    (2, 45, 257, 1.0, 1.0, 1e-4),
    (2, 1000, 129, 1.0, 2.0, 1e-3),     # stiff: sigma = 1e3
])
def test_cn1d_matches_oracle(order, n, batch, l, kappa, dt, rewrite):
    steps = 7
    c0 = synth.field(17 + n + batch, n, batch, -1.0, 1.0)  # (n, batch) = interleaved
    got = _run_gpu(order, c0, n, batch, l, kappa, dt, steps, rewrite)
    want = np.empty_like(c0)
    for s in range(batch):
        want[:, s] = oracle.cn1d_run(order, c0[:, s], l, kappa, dt, steps)
    tol = _tol(order, _sigma(order, n, l, kappa, dt), steps, np.max(np.abs(c0)))
    assert np.max(np.abs(got - want)) <= tol


def test_cn1d_rewrite_equals_constant_within_rounding():
    order, n, batch, l, kappa, dt, steps = 4, 128, 1000, 1.0, 1.0, 2e-7, 11
    c0 = synth.field(5, n, batch, -1.0, 1.0)
    a = _run_gpu(order, c0, n, batch, l, kappa, dt, steps, False)
    b = _run_gpu(order, c0, n, batch, l, kappa, dt, steps, True)
    assert np.max(np.abs(a - b)) <= _tol(order, _sigma(order, n, l, kappa, dt), steps, 1.0)


def test_cn_hyperdiffusion_exact_solution_on_device():
    # Sec. 4.2.4: A = 1, phi = 0, wave number 2, gamma = D = L = 1, T = 1e-4,
    # dt = 1e-8; the L2 error (Eq. myerr) falls as N^-2 (fitted -2.0162)
    T, dt, wave = 1e-4, 1e-8, 2
    k = 2 * np.pi * wave
    steps = int(round(T / dt))
    ns, errs = [16, 32, 64, 128], []
    for n in ns:
        x = np.arange(n) / n
        c0 = np.tile(np.cos(k * x)[:, None], (1, 3))  # three identical systems, as in Sec. 4.3
        got = _run_gpu(4, c0, n, 3, 1.0, 1.0, dt, steps, False)
        exact = np.exp(-k**4 * T) * np.cos(k * x)
        assert np.max(np.abs(got - got[:, :1])) == 0.0  # identical systems, identical bits
        errs.append(np.sqrt(np.mean((got[:, 0] - exact) ** 2)))
        if n <= 64:
            want = oracle.cn1d_run(4, np.cos(k * x), 1.0, 1.0, dt, steps)
            assert np.max(np.abs(got[:, 0] - want)) <= 1e-12
    slope = np.polyfit(np.log(ns), np.log(errs), 1)[0]
    assert abs(slope + 2.0) < 0.05, slope


def test_cn_diffusion_exact_solution_on_device():
    k, T, dt = 2 * np.pi * 3, 1e-3, 1e-6
    errs = []
    for n in (32, 64, 128, 256):
        x = np.arange(n) / n
        got = _run_gpu(2, np.cos(k * x)[:, None], n, 1, 1.0, 1.0, dt, int(round(T / dt)), False)
        errs.append(np.max(np.abs(got[:, 0] - np.exp(-k**2 * T) * np.cos(k * x))))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(orders - 2.0) < 0.05), orders


@pytest.mark.parametrize("order", [2, 4])
def test_cn1d_full_size_sampled(order):
    # the benchmark's size: 1024 unknowns x 65536 systems; sampled systems against the oracle
    n, batch, l, kappa = 1024, 65536, 1.0, 1.0
    dt = 1e-9 if order == 4 else 1e-5
    steps = 3
    g = torch.Generator().manual_seed(0)
    c0d = synth.uniform_torch(123, n * batch, -1.0, 1.0)
    c0 = c0d.cpu().reshape(n, batch)
    chx = _chx()
    for rewrite in (False, True):
        plan = chx.CN1DPlan(order, n, batch, l, kappa, dt, rewrite)
        c = c0d.clone()
        plan.step(c, steps)
        plan.sync_status()
        got = c.cpu().numpy().reshape(n, batch)
        del plan, c
        idx = torch.randperm(batch, generator=g)[:24].numpy()
        tol = _tol(order, _sigma(order, n, l, kappa, dt), steps, 1.0)
        for s in list(idx) + [0, batch - 1]:
            want = oracle.cn1d_run(order, c0[:, s].numpy(), l, kappa, dt, steps)
            assert np.max(np.abs(got[:, s] - want)) <= tol, (rewrite, s)
        torch.cuda.empty_cache()


def test_cn1d_zero_steps_and_bad_arguments():
    chx = _chx()
    c = torch.ones(10 * 4, dtype=torch.float64, device="cuda")
    plan = chx.CN1DPlan(4, 10, 4, 1.0, 1.0, 1e-4)
    plan.step(c, 0)
    assert torch.equal(c, torch.ones_like(c))
    for args in [(3, 10, 4, 1.0, 1.0, 1e-4), (4, 5, 4, 1.0, 1.0, 1e-4), (2, 2, 4, 1.0, 1.0, 1e-4),
                 (4, 10, 0, 1.0, 1.0, 1e-4), (4, 10, 4, 0.0, 1.0, 1e-4), (4, 10, 4, 1.0, -1.0, 1e-4),
                 (2, 10, 4, 1.0, 1.0, 0.0)]:
        with pytest.raises(chx.ChxError) as e:
            chx.CN1DPlan(*args)
        assert e.value.status == -1
    with pytest.raises(chx.ChxError):
        plan.step(c, -1)
