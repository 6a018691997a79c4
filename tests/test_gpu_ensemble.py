"""GPU tests of the ensemble runtime and the continuous-batching server."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda"
DX = 2 * np.pi / 64  # fixed spacing: L = n * DX


def _chx():
    import paper_2101_06550_gb300 as chx

    return chx


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _ic(seed, n):
    return synth.field(seed, n, n, -0.1, 0.1)


def _alone(n, gamma, dt, seed, steps, precision=0):
    chx = _chx()
    plan = chx.ChPlan(n, n, n * DX, n * DX, gamma, dt, precision)
    c = torch.from_numpy(_ic(seed, n)).to(DEV)
    p = c.clone()
    plan.step(c, p, plan.alloc_work(DEV), steps)
    return c.cpu().numpy()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("steps", [1, 6, 7])
def test_ensemble_matches_single_plans(precision, steps):
    chx = _chx()
    dt = 1e-3
    ens = chx.Ensemble(dt, precision)
    sims = [(64, 0.01, 1), (64, 0.02, 2), (96, 0.005, 3), (64, 0.01, 4), (128, 0.015, 5)]
    gids, slots = {}, []
    for n, g, s in sims:
        if n not in gids:
            gids[n] = ens.group_create(n, n * DX, 0.01, 4)
        gid = gids[n]
        slot = sum(1 for x in slots if x[0] == gid)
        ens.load(gid, slot, torch.from_numpy(_ic(s, n)).to(DEV), None, g)
        slots.append((gid, slot, n, g, s))
    for n, gid in gids.items():
        ens.set_active(gid, sum(1 for x in slots if x[0] == gid))
    ens.step(steps)
    tol = 1e-11 if precision == 0 else 1e-6
    for gid, slot, n, g, s in slots:
        out = torch.empty(n * n, dtype=torch.float64, device=DEV)
        ens.read(gid, slot, out)
        ref = _alone(n, g, dt, s, steps, precision)
        assert _rel(out.cpu().numpy().reshape(n, n), ref) <= tol, (n, g, s)
    ens.sync_status()


def test_ensemble_f32_refine_odd_rows_straddle_slots():
    # odd n: the fused x solve's two-row blocks straddle simulations (row 32 of
    # slot 0 with row 0 of slot 1 at n = 33), each row solved with its own
    # slot's operator; single segments of odd length in both directions
    chx = _chx()
    n, dt = 33, 1e-3
    gammas = [0.01, 0.02, 0.005]
    ens = chx.Ensemble(dt, chx.PREC_F32_REFINE)
    gid = ens.group_create(n, n * DX, 0.01, 3)
    for s, g in enumerate(gammas):
        ens.load(gid, s, torch.from_numpy(_ic(60 + s, n)).to(DEV), None, g)
    ens.set_active(gid, 3)
    ens.step(4)
    ens.sync_status()
    for s, g in enumerate(gammas):
        out = torch.empty(n * n, dtype=torch.float64, device=DEV)
        ens.read(gid, s, out)
        c0 = _ic(60 + s, n)
        ref, _ = oracle.ch_run(c0, c0, n * DX, n * DX, g, dt, 4)
        assert _rel(out.cpu().numpy().reshape(n, n), ref) <= 1e-6, (s, g)


@pytest.mark.parametrize("precision", [0, 1])
def test_ensemble_result_independent_of_the_mix(precision):
    # the same simulation alone and among others of other sizes and gammas gives
    # the same bits: FP32 + refinement ensembles step all groups with shared
    # persistent phase launches, whose work items never mix simulations
    chx = _chx()
    n, dt, steps = 64, 1e-3, 9
    target = torch.from_numpy(_ic(11, n)).to(DEV)
    ens1 = chx.Ensemble(dt, precision)
    g1 = ens1.group_create(n, n * DX, 0.01, 8)
    ens1.load(g1, 0, target, None, 0.013)
    ens1.set_active(g1, 1)
    ens1.step(steps)
    a = torch.empty(n * n, dtype=torch.float64, device=DEV)
    ens1.read(g1, 0, a)
    ens2 = chx.Ensemble(dt, precision)
    g2 = ens2.group_create(n, n * DX, 0.01, 8)
    g3 = ens2.group_create(96, 96 * DX, 0.01, 3)
    for s in range(6):
        if s == 3:
            ens2.load(g2, s, target, None, 0.013)
        else:
            ens2.load(g2, s, torch.from_numpy(_ic(50 + s, n)).to(DEV), None, 0.005 + 0.003 * s)
    for s in range(3):
        ens2.load(g3, s, torch.from_numpy(_ic(70 + s, 96)).to(DEV), None, 0.02)
    ens2.set_active(g2, 6)
    ens2.set_active(g3, 3)
    ens2.step(steps)
    b = torch.empty(n * n, dtype=torch.float64, device=DEV)
    ens2.read(g2, 3, b)
    ens1.sync_status()
    ens2.sync_status()
    assert torch.equal(a, b)


def test_ensemble_schedule_tuning_changes_no_result():
    # the packed schedule (group order, y strip width, blocks per SM) only moves
    # work items between blocks: a tuned ensemble and an untuned one agree bit
    # for bit, and the tuner leaves every simulation where it was
    chx = _chx()
    dt = 1e-3
    sizes = [(64, 4), (128, 2), (96, 3)]

    def make():
        ens = chx.Ensemble(dt, chx.PREC_F32_REFINE)
        gids = []
        for k, (n, cnt) in enumerate(sizes):
            g = ens.group_create(n, n * DX, 0.01, cnt)
            for s in range(cnt):
                ens.load(g, s, torch.from_numpy(_ic(100 + 10 * k + s, n)).to(DEV), None, 0.005 + 0.005 * s)
            ens.set_active(g, cnt)
            gids.append(g)
        return ens, gids

    e1, g1 = make()
    e2, g2 = make()
    e1.step(3)
    e2.step(3)
    sched = e2.tune_schedule(2)
    assert sched["order"] in (0, 1) and sched["points_per_item"] in (2048, 4096, 8192) and min(sched["blocks"]) >= 1
    info = e2.schedule_info()
    # right-hand-side items are pairs of vertically adjacent 32 x 32 tiles
    assert info["items"][0] == sum(cnt * ((n + 31) // 32) * (((n + 31) // 32 + 1) // 2) for n, cnt in sizes)
    e1.step(5)
    e2.step(5)
    for (n, cnt), a, b in zip(sizes, g1, g2):
        for s in range(cnt):
            x = torch.empty(n * n, dtype=torch.float64, device=DEV)
            y = torch.empty(n * n, dtype=torch.float64, device=DEV)
            e1.read(a, s, x)
            e2.read(b, s, y)
            assert torch.equal(x, y), (n, s)
    e1.sync_status()
    e2.sync_status()


def test_ensemble_matches_oracle_and_slot_move():
    chx = _chx()
    n, dt, g = 48, 1e-3, 0.01
    ens = chx.Ensemble(dt)
    gid = ens.group_create(n, n * DX, g, 3)
    c0, c1 = _ic(7, n), _ic(8, n)
    ens.load(gid, 0, torch.from_numpy(c0).to(DEV))
    ens.load(gid, 1, torch.from_numpy(c1).to(DEV))
    ens.set_active(gid, 2)
    ens.step(4)
    ens.move(gid, 1, 0)  # slot 1's simulation continues from slot 0
    ens.set_active(gid, 1)
    ens.step(3)
    out = torch.empty(n * n, dtype=torch.float64, device=DEV)
    ens.read(gid, 0, out)
    ref, _ = oracle.ch_run(c1, c1, n * DX, n * DX, g, dt, 7)
    assert _rel(out.cpu().numpy().reshape(n, n), ref) <= 1e-11


def test_ensemble_autotune_keeps_state_and_budget_admission():
    chx = _chx()
    n, dt = 128, 1e-3
    ens = chx.Ensemble(dt, hbm_budget=64 << 20)
    gid = ens.group_create(n, n * DX, 0.01, 4)
    for s in range(4):
        ens.load(gid, s, torch.from_numpy(_ic(20 + s, n)).to(DEV))
    ens.set_active(gid, 4)
    px, py = ens.autotune(gid, 2)
    assert n % px == 0 and n % py == 0
    ens.step(5)
    out = torch.empty(n * n, dtype=torch.float64, device=DEV)
    ens.read(gid, 2, out)
    ref = _alone(n, 0.01, dt, 22, 5)
    assert _rel(out.cpu().numpy().reshape(n, n), ref) <= 1e-11
    with pytest.raises(chx.ChxError) as e:
        ens.group_create(1024, 1024 * DX, 0.01, 16)  # far over the 64 MiB budget
    assert e.value.status == -4
    assert ens.bytes_used <= 64 << 20


@pytest.mark.parametrize("precision", [0, 1])
def test_server_continuous_batching_results_match_alone(precision):
    # FP64 and FP32 + refinement servers: requests overlap on the device, each
    # result matches the request run alone (single plan: 1e-11 in FP64, the
    # FP32 path's 1e-6 target), and a request served alone gives the same bits
    # as in the mix
    from paper_2101_06550_gb300 import serving

    dt = 1e-3
    reqs = serving.poisson_requests(12, rate=400.0, seed=3, n_min=32, n_max=128, steps_lo=10, steps_hi=60)
    mk = lambda r: torch.from_numpy(_ic(r.seed, r.n)).to(DEV)  # noqa: E731
    srv = serving.Server(dt, DX, precision=precision, capacity=4, chunk=16, make_ic=mk)
    stats = serving.serve(reqs, srv, time_limit=120)
    assert stats["completed"] == len(reqs)
    assert stats["p50_s"] <= stats["p99_s"]
    # requests overlapped on the device: more requests than ticks would allow one at a time
    assert srv.ticks < sum(-(-r.steps // 16) for r in reqs)
    tol = 1e-11 if precision == 0 else 1e-6
    for r in reqs:
        got = r.result.numpy().reshape(r.n, r.n)
        assert _rel(got, _alone(r.n, r.gamma, dt, r.seed, r.steps, precision)) <= tol, r
    r0 = reqs[5]
    solo = serving.Request(rid=0, n=r0.n, steps=r0.steps, gamma=r0.gamma, seed=r0.seed, arrival=0.0)
    srv2 = serving.Server(dt, DX, precision=precision, capacity=4, chunk=16, make_ic=mk)
    serving.serve([solo], srv2)
    assert torch.equal(solo.result, r0.result)


def test_server_fill_admission_and_time_bounded_ticks():
    # admission stops while the admitted grid points fill the GPU (a request is
    # still admitted when nothing runs), ticks are cut to about tick_ms, and
    # every result still matches its request run alone
    from paper_2101_06550_gb300 import serving

    dt = 1e-3
    reqs = serving.poisson_requests(10, rate=1000.0, seed=5, n_min=64, n_max=128, steps_lo=20, steps_hi=40)
    mk = lambda r: torch.from_numpy(_ic(r.seed, r.n)).to(DEV)  # noqa: E731
    fill = 2 * 128 * 128
    srv = serving.Server(dt, DX, precision=1, capacity=8, chunk=16, make_ic=mk, fill_points=fill, tick_ms=0.05)
    peak = [0]
    tick = srv.tick

    def watched(clock):
        peak[0] = max(peak[0], srv.active_points())
        return tick(clock)

    srv.tick = watched
    stats = serving.serve(reqs, srv, time_limit=120)
    assert stats["completed"] == len(reqs)
    assert 0 < peak[0] <= fill
    for r in reqs:
        got = r.result.numpy().reshape(r.n, r.n)
        assert _rel(got, _alone(r.n, r.gamma, dt, r.seed, r.steps, 1)) <= 1e-6, r
