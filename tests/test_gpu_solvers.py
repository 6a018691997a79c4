"""GPU parity of the batched cyclic band solvers against the CPU oracle (through the C ABI)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda"


def _chx():
    import paper_2101_06550_gb300 as chx

    return chx


def _adi_coefs(sig):
    return [sig, -4 * sig, 1 + 6 * sig, -4 * sig, sig]


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# --------------------------------------------------------------------------- penta
@pytest.mark.parametrize("n", [5, 8, 37, 256])
@pytest.mark.parametrize("batch", [1, 33, 515])
def test_penta_uniform_f64(n, batch):
    chx = _chx()
    sig = 18.4
    f = synth.uniform(n + batch, n * batch, -1, 1)
    x = torch.from_numpy(f).to(DEV)
    plan = chx.PentaPlan(n, _adi_coefs(sig), batch, mode=chx.COEF_UNIFORM)
    plan.solve(x)
    ref = oracle.penta_cyclic_batch(*[np.full(n, c) for c in _adi_coefs(sig)], f, batch)
    assert _rel(x.cpu().numpy(), ref) <= 1e-12


@pytest.mark.parametrize("n", [6, 64, 333])
def test_penta_shared_f64_and_f32(n):
    chx = _chx()
    batch = 257
    co = synth.diag_dominant_penta(3, n, 1)
    f = synth.uniform(4, n * batch, -1, 1)
    ref = oracle.penta_cyclic_batch(*co, f, batch)
    x = torch.from_numpy(f).to(DEV)
    chx.PentaPlan(n, co, batch, mode=chx.COEF_SHARED).solve(x)
    assert _rel(x.cpu().numpy(), ref) <= 1e-13
    x32 = torch.from_numpy(f.astype(np.float32)).to(DEV)
    chx.PentaPlan(n, co, batch, mode=chx.COEF_SHARED, dtype=chx.F32).solve(x32)
    assert _rel(x32.cpu().numpy().astype(np.float64), ref) <= 1e-5


@pytest.mark.parametrize("n,batch", [(5, 7), (16, 100), (129, 300)])
def test_penta_per_system_f64(n, batch):
    chx = _chx()
    co = synth.diag_dominant_penta(8, n, batch)
    f = synth.uniform(9, n * batch, -1, 1)
    ref = oracle.penta_cyclic_batch(*co, f, batch)
    dco = [torch.from_numpy(c).to(DEV) for c in co]
    plan = chx.PentaPlan(n, dco, batch, mode=chx.COEF_PER_SYSTEM)
    x = torch.from_numpy(f).to(DEV)
    plan.solve(x)
    plan.sync_status()
    assert _rel(x.cpu().numpy(), ref) <= 1e-13
    # refactor with new coefficients ("Rewrite" mode) and solve again
    co2 = synth.diag_dominant_penta(10, n, batch)
    plan.refactor([torch.from_numpy(c).to(DEV) for c in co2])
    x2 = torch.from_numpy(f).to(DEV)
    plan.solve(x2)
    plan.sync_status()
    assert _rel(x2.cpu().numpy(), oracle.penta_cyclic_batch(*co2, f, batch)) <= 1e-13


def test_penta_per_system_f32():
    chx = _chx()
    n, batch = 48, 200
    co = synth.diag_dominant_penta(12, n, batch)
    f = synth.uniform(13, n * batch, -1, 1)
    ref = oracle.penta_cyclic_batch(*co, f, batch)
    plan = chx.PentaPlan(n, [torch.from_numpy(c).to(DEV) for c in co], batch, mode=chx.COEF_PER_SYSTEM, dtype=chx.F32)
    x = torch.from_numpy(f.astype(np.float32)).to(DEV)
    plan.solve(x)
    plan.sync_status()
    assert _rel(x.cpu().numpy().astype(np.float64), ref) <= 1e-5


@pytest.mark.parametrize("sig", [18.4, 7.05e3])
def test_penta_refine_f32_sweeps_fp64_residual(sig):
    chx = _chx()
    n, batch = 1024, 300
    f = synth.uniform(2, n * batch, -1, 1)
    ref = oracle.penta_cyclic_batch(*[np.full(n, c) for c in _adi_coefs(sig)], f, batch)
    plan = chx.PentaPlan(n, _adi_coefs(sig), batch, mode=chx.COEF_UNIFORM)
    x = torch.from_numpy(f).to(DEV)
    plan.solve(x, refine=True)
    got = x.cpu().numpy()
    # one refinement: error ~ (cond * eps32)^2, cond ~ 1 + 16 sig
    cond_eps = (1 + 16 * sig) * 6e-8
    assert _rel(got, ref) <= max(4 * cond_eps**2, 1e-12)
    # and it beats the unrefined FP32 solve
    x32 = torch.from_numpy(f.astype(np.float32)).to(DEV)
    chx.PentaPlan(n, _adi_coefs(sig), batch, mode=chx.COEF_UNIFORM, dtype=chx.F32).solve(x32)
    assert _rel(got, ref) < _rel(x32.cpu().numpy().astype(np.float64), ref)


def test_penta_full_size_sampled_and_residual():
    # the standalone-solver workload: N = 1024, batch 65536, constant ADI
    # coefficients a = gamma dt / dx^4 (gamma 0.01, dt 1e-3, dx = 2 pi / 1024)
    chx = _chx()
    n, batch = 1024, 65536
    sig = 0.01 * 1e-3 / (2 * np.pi / 1024) ** 4
    co = _adi_coefs(sig)
    f = synth.uniform_torch(1, n * batch, -1, 1, device=DEV)
    x = f.clone()
    chx.PentaPlan(n, co, batch, mode=chx.COEF_UNIFORM).solve(x)
    X = x.view(n, batch)
    F = f.view(n, batch)
    res = co[2] * X + co[1] * (torch.roll(X, 1, 0) + torch.roll(X, -1, 0)) + co[0] * (torch.roll(X, 2, 0) + torch.roll(X, -2, 0)) - F
    assert float(res.abs().max()) <= 1e-13 * (1 + 16 * sig)
    idx = np.array(synth.splitmix64(5, 64) % batch, dtype=np.int64)
    fs = F[:, idx].cpu().numpy()
    ref = oracle.penta_cyclic_batch(*[np.full(n, c) for c in co], fs.ravel(), len(idx)).reshape(n, -1)
    assert _rel(X[:, idx].cpu().numpy(), ref) <= 1e-11


def test_penta_per_system_full_size_sampled_and_residual():
    # the variable-coefficient ("Rewrite") workload at full size: N = 1024,
    # batch 65536, every system its own diagonally dominant random rows
    # (synth.diag_dominant_penta drawn on the device, seed 2): the residual of
    # every system, and 64 sampled systems against the oracle
    chx = _chx()
    n, batch = 1024, 65536
    cnt = n * batch
    a, b, d, e = (synth.uniform_torch(2, cnt, -1.0, 1.0, device=DEV, offset=k * cnt) for k in range(4))
    u = synth.uniform_torch(2, cnt, 0.0, 1.0, device=DEV, offset=4 * cnt)
    c = (1.5 + 0.5 * u) * (a.abs() + b.abs() + d.abs() + e.abs())
    del u
    f = synth.uniform_torch(9, cnt, -1.0, 1.0, device=DEV)
    plan = chx.PentaPlan(n, [a, b, c, d, e], batch, mode=chx.COEF_PER_SYSTEM)
    x = f.clone()
    plan.solve(x)
    plan.sync_status()
    A, B, C, D, E, X, F = (v.view(n, batch) for v in (a, b, c, d, e, x, f))
    # row i: a_i x_{i-2} + b_i x_{i-1} + c_i x_i + d_i x_{i+1} + e_i x_{i+2} = f_i (indices mod n)
    res = A * torch.roll(X, 2, 0) + B * torch.roll(X, 1, 0) + C * X + D * torch.roll(X, -1, 0) + E * torch.roll(X, -2, 0) - F
    scale = (A.abs() + B.abs() + C.abs() + D.abs() + E.abs()) * X.abs().max()
    assert float((res.abs() / scale).max()) <= 64 * 2.220446049250313e-16
    idx = np.array(synth.splitmix64(6, 64) % batch, dtype=np.int64)
    it = torch.from_numpy(idx).to(DEV)
    cols = [v.view(n, batch)[:, it].cpu().numpy().ravel() for v in (a, b, c, d, e, f)]
    ref = oracle.penta_cyclic_batch(*cols[:5], cols[5], len(idx)).reshape(n, -1)
    assert _rel(X[:, it].cpu().numpy(), ref) <= 1e-12


def test_penta_errors():
    chx = _chx()
    with pytest.raises(chx.ChxError) as e:
        chx.PentaPlan(8, [0.0] * 5, 4, mode=chx.COEF_UNIFORM)
    assert e.value.status == -2  # singular
    plan = chx.PentaPlan(8, _adi_coefs(1.0), 4, mode=chx.COEF_UNIFORM)
    with pytest.raises(chx.ChxError):
        plan.solve(torch.zeros(8 * 5, dtype=torch.float64, device=DEV))  # batch above the plan's
    # per-system singular systems are flagged on the device
    n, batch = 8, 3
    z = [torch.zeros(n * batch, dtype=torch.float64, device=DEV) for _ in range(5)]
    p2 = chx.PentaPlan(n, z, batch, mode=chx.COEF_PER_SYSTEM)
    with pytest.raises(chx.ChxError) as e:
        p2.sync_status()
    assert e.value.status == -2


# --------------------------------------------------------------------------- tri
@pytest.mark.parametrize("n", [3, 4, 17, 1024])
@pytest.mark.parametrize("mode", ["uniform", "shared", "per_system"])
def test_tri_f64(n, mode):
    chx = _chx()
    batch = 129
    f = synth.uniform(31, n * batch, -1, 1)
    if mode == "uniform":
        sig = 0.5 * 1e-3 / (1.0 / n) ** 2
        co = [-sig, 1 + 2 * sig, -sig]
        ref = oracle.tri_cyclic_batch(*[np.full(n, c) for c in co], f, batch)
        plan = chx.TriPlan(n, co, batch, mode=chx.COEF_UNIFORM)
    elif mode == "shared":
        co = synth.diag_dominant_tri(5, n, 1)
        ref = oracle.tri_cyclic_batch(*co, f, batch)
        plan = chx.TriPlan(n, co, batch, mode=chx.COEF_SHARED)
    else:
        co = synth.diag_dominant_tri(6, n, batch)
        ref = oracle.tri_cyclic_batch(*co, f, batch)
        plan = chx.TriPlan(n, [torch.from_numpy(c).to(DEV) for c in co], batch, mode=chx.COEF_PER_SYSTEM)
    x = torch.from_numpy(f).to(DEV)
    plan.solve(x)
    plan.sync_status()
    assert _rel(x.cpu().numpy(), ref) <= 1e-12


def test_tri_f32_and_full_size_residual():
    chx = _chx()
    n, batch = 1024, 65536
    sig = 1e-3 / (2 * (2 * np.pi / n) ** 2)
    co = [-sig, 1 + 2 * sig, -sig]
    f = synth.uniform_torch(7, n * batch, -1, 1, device=DEV)
    x = f.clone()
    chx.TriPlan(n, co, batch, mode=chx.COEF_UNIFORM).solve(x)
    X, F = x.view(n, batch), f.view(n, batch)
    res = co[1] * X + co[0] * (torch.roll(X, 1, 0) + torch.roll(X, -1, 0)) - F
    assert float(res.abs().max()) <= 1e-13 * (1 + 4 * sig)
    x32 = f.float()
    chx.TriPlan(n, co, batch, mode=chx.COEF_UNIFORM, dtype=chx.F32).solve(x32)
    assert float((x32.double() - x).abs().max() / x.abs().max()) <= 1e-4
