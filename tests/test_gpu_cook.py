"""GPU parity of the Cahn-Hilliard-Cook forcing (Sec. 7.7): the Philox4x64-10 +
Box-Muller deviates, the forced ADI step with given deviates, and whole runs."""
import numpy as np
import pytest

import oracle
import synth
from tests.test_gpu_ch import _rhs_norm, step_tolerance

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda"


def _chx():
    import paper_2101_06550_gb300 as chx

    return chx


def _forced_rhs_norm(cn, cp, rho, lx, ly, gamma, dt, sigma):
    return _rhs_norm(cn, cp, lx, ly, gamma, dt) + (2.0 / 3.0) * dt * float(
        np.max(np.abs(oracle.cook_forcing(rho, lx, ly, dt, sigma))))


@pytest.mark.parametrize("nx,ny,seed,sim,step", [(64, 64, 7, 0, 0), (37, 23, 2**63 + 5, 3, 12345),
                                                 (1, 1, 1, 1, 1), (512, 384, 2021, 11, 2**40)])
def test_noise_normals_match_oracle(nx, ny, seed, sim, step):
    chx = _chx()
    rho = torch.empty(2 * nx * ny, dtype=torch.float64, device=DEV)
    chx.noise_normals(rho, nx, ny, seed, sim, step)
    got = rho.cpu().numpy().reshape(2, ny, nx)
    want = oracle.noise_normals(nx, ny, seed, sim, step)
    # same uniforms (integer work); the transform runs in FP32 on the device and
    # in FP64 in the oracle: a few FP32 ulps of the radius sqrt(-2 ln u)
    rad = np.sqrt(want[0] ** 2 + want[1] ** 2)
    assert np.all(np.abs(got - want) <= 5e-7 * rad + 1e-300)
    if nx * ny > 1000:
        z = got.ravel()
        assert abs(z.mean()) < 5 / np.sqrt(z.size) and abs(z.var() - 1) < 5 * np.sqrt(2 / z.size)


@pytest.mark.parametrize("ny,nx,sigma,rest", [(64, 64, 1e-14, True), (80, 96, 1e-6, False), (48, 40, 1e-3, False)])
def test_step_noise_matches_oracle(ny, nx, sigma, rest):
    chx = _chx()
    lx, ly, gamma, dt = 2 * np.pi, 2 * np.pi * ny / nx, 0.01, 1e-3
    if rest:
        c0 = np.zeros((ny, nx))
        cm = c0.copy()
    else:
        c0 = synth.field(31, ny, nx, -0.3, 0.3)
        cm = c0 + 1e-3 * synth.field(32, ny, nx, -1, 1)
    rho = synth.field(33, 2 * ny, nx, -2.0, 2.0).reshape(2, ny, nx)  # any deviates: the step is linear in rho
    plan = chx.ChPlan(nx, ny, lx, ly, gamma, dt)
    cn = torch.from_numpy(c0).to(DEV)
    cp = torch.from_numpy(cm).to(DEV)
    plan.step_noise(cn, cp, plan.alloc_work(DEV), torch.from_numpy(rho.ravel()).to(DEV), sigma)
    plan.sync_status()
    want, want_prev = oracle.ch_cook_step(c0, cm, rho, lx, ly, gamma, dt, sigma)
    assert np.array_equal(cp.cpu().numpy(), want_prev)
    tol = 1e-11 * float(np.max(np.abs(want))) + 4 * 2.220446049250313e-16 * _forced_rhs_norm(
        c0, cm, rho, lx, ly, gamma, dt, sigma)
    assert np.max(np.abs(cn.cpu().numpy() - want)) <= tol


def test_step_noise_full_size_one_step():
    # the 2048^2 workload (gamma 0.005, dt 5e-4) with the paper's sigma = 1e-14
    chx = _chx()
    n, l, gamma, dt, sigma = 2048, 2 * np.pi, 0.005, 5e-4, 1e-14
    c0 = synth.field(3, n, n, -0.05, 0.05)
    cm = c0 + 1e-4 * synth.field(4, n, n, -1, 1)
    rho = oracle.noise_normals(n, n, 99, 0, 0)
    plan = chx.ChPlan(n, n, l, l, gamma, dt)
    cn = torch.from_numpy(c0).to(DEV)
    cp = torch.from_numpy(cm).to(DEV)
    plan.step_noise(cn, cp, plan.alloc_work(DEV), torch.from_numpy(rho.ravel()).to(DEV), sigma)
    want, _ = oracle.ch_cook_step(c0, cm, rho, l, l, gamma, dt, sigma)
    tol = step_tolerance(want, c0, cm, l, l, gamma, dt) + 4 * 2.220446049250313e-16 * (2 / 3) * dt * float(
        np.max(np.abs(oracle.cook_forcing(rho, l, l, dt, sigma))))
    assert np.max(np.abs(cn.cpu().numpy() - want)) <= tol


@pytest.mark.parametrize("nsteps", [1, 6, 7])
def test_cook_run_matches_oracle_from_rest(nsteps):
    chx = _chx()
    n, l, gamma, dt, sigma = 64, 2 * np.pi, 0.01, 0.1 * 2 * np.pi / 64, 1e-8
    zero = np.zeros((n, n))
    plan = chx.ChPlan(n, n, l, l, gamma, dt)
    cn = torch.zeros(n * n, dtype=torch.float64, device=DEV)
    cp = torch.zeros_like(cn)
    rho = torch.empty(2 * n * n, dtype=torch.float64, device=DEV)
    plan.cook_run(cn, cp, plan.alloc_work(DEV), rho, nsteps, sigma, seed=42, sim=3, step0=10)
    plan.sync_status()
    want, want_prev = oracle.ch_cook_run(zero, zero, l, l, gamma, dt, sigma, 42, 3, 10, nsteps)
    got = cn.cpu().numpy().reshape(n, n)
    # the run is driven by the deviates alone (C = 0 at the start), and the
    # device's deviates carry FP32 rounding (5e-7 relative, test above); the
    # response is linear in them at this amplitude
    assert np.max(np.abs(got - want)) <= 1e-6 * np.max(np.abs(want))
    assert np.max(np.abs(cp.cpu().numpy().reshape(n, n) - want_prev)) <= 1e-6 * np.max(np.abs(want_prev)) + 1e-300
    # mass stays zero to rounding
    assert abs(got.sum()) <= 1e-12 * np.abs(got).sum()
    # the last deviates are those of step step0 + nsteps - 1
    last = oracle.noise_normals(n, n, 42, 3, 10 + nsteps - 1)
    assert np.all(np.abs(rho.cpu().numpy().reshape(2, n, n) - last) <= 5e-7 * np.sqrt(last[0]**2 + last[1]**2))


@pytest.mark.parametrize("nx,ny,aspect", [(64, 64, 1.0), (70, 40, 1.0), (96, 33, 1.0), (63, 48, 1.0), (64, 48, 0.5)])
def test_cook_run_in_place_draw_matches_the_deviate_kernel(nx, ny, aspect):
    # For even nx the FP64 right-hand side draws each step's deviates itself
    # (tile by tile, with the west and south halo pairs); for odd nx the
    # standalone kernel draws them first.  Either way rho ends up bit-identical
    # to ch_noise_normals of the last step, and every step matches the oracle
    # driven by the standalone kernel's deviates.  70 and 40 leave ragged
    # tiles; 33 rows wrap the halo row of the last tile row; aspect != 1 makes
    # dy != dx (different forcing weights in x and y).
    chx = _chx()
    lx, gamma, dt, sigma, seed, sim, step0, nsteps = 2 * np.pi, 0.01, 1e-3, 1e-6, 5, 2, 4, 3
    ly = lx * ny / nx * aspect
    c0 = synth.field(81, ny, nx, -0.1, 0.1)
    plan = chx.ChPlan(nx, ny, lx, ly, gamma, dt)
    cn = torch.from_numpy(c0).to(DEV).reshape(-1)
    cp = cn.clone()
    rho = torch.empty(2 * nx * ny, dtype=torch.float64, device=DEV)
    plan.cook_run(cn, cp, plan.alloc_work(DEV), rho, nsteps, sigma, seed=seed, sim=sim, step0=step0)
    plan.sync_status()
    last = torch.empty_like(rho)
    chx.noise_normals(last, nx, ny, seed, sim, step0 + nsteps - 1)
    assert torch.equal(rho, last)
    c, p = c0, c0
    for k in range(nsteps):
        r = torch.empty_like(rho)
        chx.noise_normals(r, nx, ny, seed, sim, step0 + k)
        rk = r.cpu().numpy().reshape(2, ny, nx)
        tol_rhs = _forced_rhs_norm(c, p, rk, lx, ly, gamma, dt, sigma)
        c, p = oracle.ch_cook_step(c, p, rk, lx, ly, gamma, dt, sigma)
    tol = 1e-11 * float(np.max(np.abs(c))) * nsteps + 4 * 2.220446049250313e-16 * tol_rhs * nsteps
    assert np.max(np.abs(cn.cpu().numpy().reshape(ny, nx) - c)) <= tol


def test_cook_rejects_bad_arguments():
    chx = _chx()
    n = 32
    plan = chx.ChPlan(n, n, 1.0, 1.0, 0.01, 1e-3)
    cn = torch.zeros(n * n, dtype=torch.float64, device=DEV)
    cp = torch.zeros_like(cn)
    work = plan.alloc_work(DEV)
    rho = torch.zeros(2 * n * n, dtype=torch.float64, device=DEV)
    with pytest.raises(chx.ChxError) as e:
        plan.step_noise(cn, cp, work, rho, -1.0)
    assert e.value.status == -1
    both = torch.zeros(3 * n * n, dtype=torch.float64, device=DEV)
    with pytest.raises(chx.ChxError) as e:  # rho overlapping c_now
        plan.step_noise(both[:n * n], cp, work, both[n * n // 2:n * n // 2 + 2 * n * n], 1e-6)
    assert e.value.status == -1


def test_ensemble_cook_matches_single_plan_runs():
    # every slot of a forced ensemble group follows ch_cook_run with simulation
    # id = slot, through eager single steps and graph-replayed pairs alike
    chx = _chx()
    n, dx, dt, sigma, seed, step0 = 64, 2 * np.pi / 64, 1e-3, 1e-8, 9, 5
    gammas = [0.01, 0.02, 0.005]
    ics = [np.zeros((n, n)), synth.field(61, n, n, -0.1, 0.1), synth.field(62, n, n, -0.3, 0.3)]
    ens = chx.Ensemble(dt)
    gid = ens.group_create(n, n * dx, 0.01, 4)
    for s, (c0, g) in enumerate(zip(ics, gammas)):
        ens.load(gid, s, torch.from_numpy(c0).to(DEV), None, g)
    ens.set_active(gid, 3)
    ens.set_cook(gid, sigma, seed=seed, step0=step0)
    ens.step(1)  # eager
    ens.step(6)  # three graph pairs
    ens.sync_status()
    for s, (c0, g) in enumerate(zip(ics, gammas)):
        plan = chx.ChPlan(n, n, n * dx, n * dx, g, dt)
        cn = torch.from_numpy(c0).to(DEV)
        cp = cn.clone()
        rho = torch.empty(2 * n * n, dtype=torch.float64, device=DEV)
        plan.cook_run(cn, cp, plan.alloc_work(DEV), rho, 7, sigma, seed=seed, sim=s, step0=step0)
        got = torch.empty(n * n, dtype=torch.float64, device=DEV)
        ens.read(gid, s, got)
        want = cn.cpu().numpy().ravel()
        assert np.max(np.abs(got.cpu().numpy() - want)) <= 1e-11 * np.max(np.abs(want)), s
    # forcing off: the next steps are the plain ADI steps
    ens.set_cook(gid, 0.0)
    before = torch.empty((n, n), dtype=torch.float64, device=DEV)
    prev = torch.empty_like(before)
    ens.read(gid, 1, before, prev)
    ens.step(2)
    after = torch.empty((n, n), dtype=torch.float64, device=DEV)
    ens.read(gid, 1, after)
    plan = chx.ChPlan(n, n, n * dx, n * dx, gammas[1], dt)
    plan.step(before, prev, plan.alloc_work(DEV), 2)
    assert np.max(np.abs(after.cpu().numpy() - before.cpu().numpy())) <= 1e-11 * float(before.abs().max())


def test_cook_fp32_refine_matches_oracle_and_fp64():
    # the mixed-precision plan forms the forcing term in FP64 and adds it to its
    # double-float right-hand side: per step it stays within the FP32+refine
    # bound of the oracle, over a run within that bound of the FP64 run
    chx = _chx()
    n, l, gamma, dt, sigma = 96, 2 * np.pi, 0.01, 1e-3, 1e-8
    c0 = synth.field(71, n, n, -0.2, 0.2)
    rho = oracle.noise_normals(n, n, 4, 2, 0)
    p32 = chx.ChPlan(n, n, l, l, gamma, dt, chx.PREC_F32_REFINE)
    cn = torch.from_numpy(c0).to(DEV)
    cp = cn.clone()
    p32.step_noise(cn, cp, p32.alloc_work(DEV), torch.from_numpy(rho.ravel()).to(DEV), sigma)
    p32.sync_status()
    want, _ = oracle.ch_cook_step(c0, c0, rho, l, l, gamma, dt, sigma)
    assert np.max(np.abs(cn.cpu().numpy() - want)) <= 1e-6 * np.max(np.abs(want))
    outs = []
    for prec in (chx.PREC_F64, chx.PREC_F32_REFINE):
        plan = chx.ChPlan(n, n, l, l, gamma, dt, prec)
        a = torch.zeros(n * n, dtype=torch.float64, device=DEV)
        b = torch.zeros_like(a)
        scratch = torch.empty(2 * n * n, dtype=torch.float64, device=DEV)
        plan.cook_run(a, b, plan.alloc_work(DEV), scratch, 6, sigma, seed=3)
        outs.append(a.cpu().numpy())
    assert np.max(np.abs(outs[1] - outs[0])) <= 1e-6 * np.max(np.abs(outs[0]))
    # a mixed-precision ensemble group follows the mixed-precision plan slot by slot
    ens = chx.Ensemble(dt, chx.PREC_F32_REFINE)
    gid = ens.group_create(n, l, gamma, 2)
    ens.load(gid, 0, torch.zeros(n * n, dtype=torch.float64, device=DEV))
    ens.set_active(gid, 1)
    ens.set_cook(gid, sigma, seed=3)
    ens.step(6)
    got = torch.empty(n * n, dtype=torch.float64, device=DEV)
    ens.read(gid, 0, got)
    assert np.max(np.abs(got.cpu().numpy() - outs[1])) <= 1e-6 * np.max(np.abs(outs[1]))
