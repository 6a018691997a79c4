"""GPU parity of the batched 1D Cahn-Hilliard step (Sec. 6.2.1) against the CPU oracle."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("n", [8, 33, 256])
@pytest.mark.parametrize("batch", [1, 100, 4097])
def test_ch1d_matches_oracle(n, batch):
    import paper_2101_06550_gb300 as chx

    l, gamma = 2 * np.pi, 0.01
    dt = 0.1 * l / n  # the thesis's dt = 0.1 dx
    c0 = synth.uniform(n + batch, n * batch, -0.1, 0.1)
    plan = chx.Ch1DPlan(n, batch, l, gamma, dt)
    c = torch.from_numpy(c0).cuda()
    plan.step(c, 7)
    ref = oracle.ch1d_run(c0, l, gamma, dt, 7, batch)
    assert _rel(c.cpu().numpy(), ref) <= 1e-11
    plan.sync_status()


def test_ch1d_full_batch_sampled_and_mass():
    # 2^20 simulations of N = 256 (Sec. 6.2.3): sampled systems against the
    # oracle, and every system's mass conserved
    import paper_2101_06550_gb300 as chx

    n, batch, l, gamma = 256, 1 << 20, 2 * np.pi, 0.01
    dt = 0.1 * l / n
    c = synth.uniform_torch(5, n * batch, -0.1, 0.1, device="cuda")
    c0 = c.clone()
    plan = chx.Ch1DPlan(n, batch, l, gamma, dt)
    plan.step(c, 3)
    C, C0 = c.view(n, batch), c0.view(n, batch)
    drift = (C.sum(0) - C0.sum(0)).abs().max().item()
    assert drift <= 1e-13 * C0.abs().sum(0).max().item()
    idx = np.array(synth.splitmix64(9, 48) % batch, dtype=np.int64)
    sub = C0[:, idx].cpu().numpy()
    ref = oracle.ch1d_run(sub.ravel(), l, gamma, dt, 3, len(idx)).reshape(n, -1)
    assert _rel(C[:, idx].cpu().numpy(), ref) <= 1e-11


def test_ch1d_rejects_bad_arguments():
    import paper_2101_06550_gb300 as chx

    with pytest.raises(chx.ChxError):
        chx.Ch1DPlan(4, 10, 1.0, 0.01, 1e-3)
    with pytest.raises(chx.ChxError):
        chx.Ch1DPlan(16, 10, 1.0, 0.01, 0.0)


def test_ch1d_convergence_study_on_device():
    # Table table5:converge1D rerun on the device: t = 20, whole steps until
    # t >= T, E_N by Eq. eq2:converge1D.  The printed E_N from N = 128 to 2048
    # and the observed orders from 128 to 1024 are reproduced.
    import decimal
    import os

    import paper_2101_06550_gb300 as chx

    rows = {}
    for ln in open(os.path.join(os.path.dirname(__file__), "golden", "table_converge1d.txt")):
        if ln.strip() and not ln.startswith("#"):
            n, e, o = ln.split()
            rows[int(n)] = (float(e), float(o), 0.5 * 10.0 ** decimal.Decimal(e).as_tuple().exponent)
    l, gamma, t_end, eps = 2 * np.pi, 0.01, 20.0, 1e-6
    res = {}
    for n in (64, 128, 256, 512, 1024, 2048):
        x = np.arange(n) * l / n
        dt = 0.1 * l / n
        c = torch.from_numpy(eps * np.cos(5 * x)).to("cuda")
        chx.Ch1DPlan(n, 1, l, gamma, dt).step(c, int(np.ceil(t_end / dt - 1e-9)))
        res[n] = c.cpu().numpy()
    e = {n: oracle.refinement_error_1d(res[n], res[n // 2]) for n in (128, 256, 512, 1024, 2048)}
    for n in (128, 256, 512, 1024, 2048):
        assert abs(e[n] - rows[n][0]) <= rows[n][2], (n, e[n], rows[n][0])
    for n in (128, 256, 512, 1024):
        assert abs(np.log2(e[n] / e[2 * n]) - rows[n][1]) <= 2e-4, (n, np.log2(e[n] / e[2 * n]), rows[n][1])
