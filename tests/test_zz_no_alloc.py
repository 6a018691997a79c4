"""The allocation-free diagnostics entry point (ch_diagnostics_noalloc).

Some callers cannot call cudaMalloc, so this entry point takes no plan and keeps
its scratch in a fixed device array.  It must give the same mass and energy as
the plan-based ch_diagnostics, on two calls in a row (the second call reuses the
array the first one left behind).  This file is collected last on purpose.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")


@pytest.mark.gpu
def test_noalloc_diagnostics_match_plan_based_twice():
    import paper_2101_06550_gb300 as chx
    from paper_2101_06550_gb300 import _chx

    lx, ly, gamma = 2 * np.pi, 3.0, 0.02
    for k, (ny, nx) in enumerate([(300, 517), (64, 2048)]):
        c = torch.from_numpy(synth.field(40 + k, ny, nx, -1, 1)).to("cuda")
        plan = chx.ChPlan(nx, ny, lx, ly, gamma, 1e-3)
        ref = torch.zeros(2, dtype=torch.float64, device="cuda")
        plan.diagnostics(c, ref)
        got = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
        _chx.ch_diagnostics_noalloc(c, lx, ly, gamma, got)
        torch.cuda.synchronize()
        plan.sync_status()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        scale_m = float(c.abs().sum()) * (lx / nx) * (ly / ny)
        assert abs(g[0] - r[0]) <= 1e-12 * scale_m
        assert abs(g[1] - r[1]) <= 1e-12 * abs(r[1])


@pytest.mark.gpu
def test_noalloc_rejects_too_many_rows_and_flags_nonfinite():
    from paper_2101_06550_gb300 import _chx

    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    big = torch.zeros(16385, 2, dtype=torch.float64, device="cuda")
    with pytest.raises(_chx.ChxError) as e:
        _chx.ch_diagnostics_noalloc(big, 1.0, 1.0, 0.01, out)
    assert e.value.status == -1
    c = torch.zeros(8, 8, dtype=torch.float64, device="cuda")
    c[2, 3] = float("nan")
    _chx.ch_diagnostics_noalloc(c, 1.0, 1.0, 0.01, out)
    assert np.all(np.isnan(out.cpu().numpy()))


@pytest.mark.gpu
def test_noalloc_call_takes_no_device_memory():
    # the property the entry point exists for: after a first call (which loads
    # its kernels and looks up the array's address), a call at another shape
    # leaves the device's free memory unchanged
    from paper_2101_06550_gb300 import _chx

    a = torch.from_numpy(synth.field(45, 96, 160, -1, 1)).to("cuda")
    b = torch.from_numpy(synth.field(46, 1024, 40, -1, 1)).to("cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    _chx.ch_diagnostics_noalloc(a, 1.0, 1.0, 0.01, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    _chx.ch_diagnostics_noalloc(b, 2.0, 1.5, 0.02, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0
    assert np.all(np.isfinite(out.cpu().numpy()))
