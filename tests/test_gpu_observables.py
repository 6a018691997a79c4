"""GPU parity of the coarsening observables (mass, F_h, s, k1; Secs. 2.4, 3.5.4)
for single fields and whole ensemble groups."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda"
EPS = np.finfo(np.float64).eps


def _chx():
    import paper_2101_06550_gb300 as chx

    return chx


def _check_obs(got, c, lx, ly, gamma):
    m, e, s, k1 = oracle.observables(c, lx, ly, gamma)
    n = c.size
    cell = lx * ly / n
    # fixed-order sums of n terms: within n eps of the sum of magnitudes
    assert abs(got[0] - m) <= n * EPS * np.abs(c).sum() * cell
    assert abs(got[1] - e) <= n * EPS * e
    assert got[2] == pytest.approx(s, rel=n * EPS)
    assert got[3] == pytest.approx(k1, rel=1e-12)


@pytest.mark.parametrize("ny,nx", [(64, 64), (80, 96), (45, 33), (2048, 2048)])
def test_observables_match_oracle(ny, nx):
    chx = _chx()
    lx, ly, gamma = 2 * np.pi, 2 * np.pi * ny / nx * 1.1, 0.01
    c = synth.field(12 + nx, ny, nx, -0.9, 0.9)
    plan = chx.ChPlan(nx, ny, lx, ly, gamma, 1e-3)
    out = torch.empty(4, dtype=torch.float64, device=DEV)
    ct = torch.from_numpy(c).to(DEV)
    for _ in range(2):  # the second call reuses the plan's scratch
        plan.observables(ct, out)
        plan.sync_status()
        _check_obs(out.cpu().numpy(), c, lx, ly, gamma)


def test_observables_of_a_developed_state():
    chx = _chx()
    n, l, gamma = 64, 2 * np.pi, 0.01
    dt = 0.1 * l / n
    c0 = synth.field(3, n, n, -0.1, 0.1)
    c, _ = oracle.ch_run(c0, c0, l, l, gamma, dt, 300)
    plan = chx.ChPlan(n, n, l, l, gamma, dt)
    out = torch.empty(4, dtype=torch.float64, device=DEV)
    plan.observables(torch.from_numpy(c).to(DEV), out)
    _check_obs(out.cpu().numpy(), c, l, l, gamma)


def test_ensemble_observables_per_slot():
    chx = _chx()
    n, dx, dt = 96, 2 * np.pi / 64, 1e-3
    ens = chx.Ensemble(dt)
    gid = ens.group_create(n, n * dx, 0.01, 6)
    gammas = [0.01, 0.02, 0.005, 0.013, 0.01]
    fields = [synth.field(70 + s, n, n, -0.5, 0.5) for s in range(5)]
    for s, (f, g) in enumerate(zip(fields, gammas)):
        ens.load(gid, s, torch.from_numpy(f).to(DEV), None, g)
    ens.set_active(gid, 5)
    out = torch.empty(4 * 5, dtype=torch.float64, device=DEV)
    ens.observables(gid, out)
    ens.sync_status()
    got = out.cpu().numpy().reshape(5, 4)
    for s in range(5):
        m, e, sv, _ = oracle.observables(fields[s], n * dx, n * dx, gammas[s])
        assert got[s, 0] == pytest.approx(m, abs=n * n * EPS * np.abs(fields[s]).sum() * dx * dx)
        assert got[s, 1] == pytest.approx(e, rel=n * n * EPS)
        assert got[s, 2] == pytest.approx(sv, rel=n * n * EPS)
        assert np.isnan(got[s, 3])
    # with k1: one batched transform over the active slots
    ens.observables(gid, out, with_k1=True)
    got = out.cpu().numpy().reshape(5, 4)
    for s in range(5):
        m, e, sv, k1 = oracle.observables(fields[s], n * dx, n * dx, gammas[s])
        assert got[s, 3] == pytest.approx(k1, rel=1e-12)
        assert got[s, 1] == pytest.approx(e, rel=n * n * EPS)
    # after steps the observables follow the slots' state
    ens.step(3)
    ens.observables(gid, out)
    cur = torch.empty(n * n, dtype=torch.float64, device=DEV)
    ens.read(gid, 2, cur)
    m, e, sv, _ = oracle.observables(cur.cpu().numpy().reshape(n, n), n * dx, n * dx, gammas[2])
    assert out[8:11].cpu().numpy() == pytest.approx([m, e, sv], rel=1e-11, abs=1e-12)


def test_observables_flag_nonfinite():
    chx = _chx()
    n = 32
    plan = chx.ChPlan(n, n, 1.0, 1.0, 0.01, 1e-3)
    c = torch.zeros(n * n, dtype=torch.float64, device=DEV)
    c[77] = float("nan")
    out = torch.empty(4, dtype=torch.float64, device=DEV)
    plan.observables(c, out)
    with pytest.raises(chx.ChxError) as e:
        plan.sync_status()
    assert e.value.status == -3
    plan.sync_status()  # the flag is cleared once read


def test_coarsening_run_on_device():
    # Sec. 3.5.4's run: 512^2, L = 2 pi, gamma = 0.01, dt = 0.1 dx, deep quench
    # C(x, 0) uniform in [-0.1, 0.1].  After the spinodal stage the domains
    # coarsen: s grows, k1 falls, F decreases and beta is positive.
    chx = _chx()
    n, l, gamma = 512, 2 * np.pi, 0.01
    dt = 0.1 * l / n
    plan = chx.ChPlan(n, n, l, l, gamma, dt)
    cn = torch.from_numpy(synth.field(1, n, n, -0.1, 0.1)).to(DEV).reshape(-1)
    cp = cn.clone()
    work = plan.alloc_work(DEV)
    out = torch.empty(4, dtype=torch.float64, device=DEV)
    every = 400
    t, rows = [], []
    for k in range(1, 21):
        plan.step(cn, cp, work, every)
        plan.observables(cn, out)
        t.append(k * every * dt)
        rows.append(out.cpu().numpy().copy())
    plan.sync_status()
    rows = np.array(rows)
    late = np.array(t) > 4
    assert np.all(np.diff(rows[late, 1]) < 0)      # F decreases
    assert rows[-1, 2] > rows[np.argmax(late), 2]  # s grows
    assert rows[-1, 3] < rows[np.argmax(late), 3]  # k1 falls
    assert abs(rows[-1, 0] - rows[0, 0]) <= 1e-9 * l * l  # mass
    beta = chx.coarsening_rate(np.array(t), rows[:, 1])
    assert np.all(beta[late] > 0)
    assert np.allclose(beta, oracle.coarsening_rate(np.array(t), rows[:, 1]), rtol=1e-9)


def test_coarsening_follows_the_one_third_law():
    # Sec. 3.5.4 (fig3:scaling): after a deep quench s(t) and 1/k1(t) grow as
    # t^(1/3) and F(t) decays as t^(-1/3).  On an 8 pi x 8 pi domain (2048^2,
    # gamma = 0.01, dt = 0.1 dx, C(x, 0) uniform in [-0.1, 0.1]) the domains
    # stay far from the box size up to t = 40; the fitted exponents over
    # t in [10, 40] are within 0.03 of 1/3 (a full run to t = 80 gives 0.335,
    # 0.330 and -0.338).
    chx = _chx()
    n, l, gamma = 2048, 8 * np.pi, 0.01
    dt = 0.1 * l / n
    plan = chx.ChPlan(n, n, l, l, gamma, dt)
    cn = torch.from_numpy(synth.field(1, n, n, -0.1, 0.1)).to(DEV).reshape(-1)
    cp = cn.clone()
    work = plan.alloc_work(DEV)
    out = torch.empty(4, dtype=torch.float64, device=DEV)
    every = int(round(2.0 / dt))
    t, rows = 0.0, []
    while t < 40.0:
        plan.step(cn, cp, work, every)
        t += every * dt
        plan.observables(cn, out)
        rows.append([t] + out.cpu().tolist())
    plan.sync_status()
    rows = np.array(rows)
    m = rows[:, 0] >= 10.0
    lt = np.log(rows[m, 0])
    assert abs(np.polyfit(lt, np.log(rows[m, 3]), 1)[0] - 1 / 3) < 0.03      # s
    assert abs(np.polyfit(lt, -np.log(rows[m, 4]), 1)[0] - 1 / 3) < 0.03     # 1/k1
    assert abs(np.polyfit(lt, np.log(rows[m, 2]), 1)[0] + 1 / 3) < 0.03      # F
