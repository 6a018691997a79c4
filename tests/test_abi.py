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
