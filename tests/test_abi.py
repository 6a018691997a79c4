"""CPU-only checks of the C ABI library: it builds, loads and exports every declared symbol."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "chx.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b([a-z_][a-z0-9_]*)\s*\(", src)) - {"if", "sizeof"})


def test_header_names_match_binding():
    import paper_2101_06550_gb300 as chx

    assert sorted(chx.EXPORTS) == _declared()


def test_library_exports_all_declared_symbols():
    from paper_2101_06550_gb300 import build as b

    b.build()
    import ctypes

    lib = ctypes.CDLL(b.LIB)
    for name in _declared():
        assert hasattr(lib, name), name


def test_status_strings_without_gpu():
    import paper_2101_06550_gb300 as chx

    assert chx.status_string(0) == "CHX_OK"
    assert chx.status_string(-2) == "CHX_ESINGULAR"
    assert chx.version() >= 10000


def test_plan_create_rejects_bad_args_without_gpu():
    # argument validation happens before any CUDA call
    import paper_2101_06550_gb300 as chx

    with pytest.raises(chx.ChxError) as e:
        chx.ChPlan(4, 64, 1.0, 1.0, 0.01, 1e-3)
    assert e.value.status == -1
    with pytest.raises(chx.ChxError):
        chx.ChPlan(64, 64, 1.0, 1.0, 0.01, -1.0)


def test_coarsening_rate_host_entry_point_matches_oracle():
    # chx_coarsening_rate works on host arrays: no device is involved
    import numpy as np

    import oracle
    import synth

    chx = pytest.importorskip("paper_2101_06550_gb300")
    t = np.sort(synth.uniform(4, 40, 1.0, 2.0))
    F = np.exp(-t) + 2 + np.sin(3 * t)
    got = chx.coarsening_rate(t, F)
    want = oracle.coarsening_rate(t, F)
    # both take the quadratic-interpolant derivative; they differ only in rounding,
    # bounded by eps times the size of the three-point weights times |F|
    h = np.min(np.diff(t))
    bound = 64 * np.finfo(float).eps * (t / np.abs(F)) * (6 / h) * np.max(np.abs(F))
    assert np.all(np.abs(got - want) <= bound)
    for bad_t, bad_F in ((t[:2], F[:2]), (t[::-1].copy(), F), (t, np.where(np.arange(t.size) == 3, 0.0, F))):
        with pytest.raises(chx.ChxError):
            chx.coarsening_rate(bad_t, bad_F)
