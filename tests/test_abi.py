"""The C-ABI library loads and exports every function include/corr.h declares (no GPU calls)."""
import os
import re

from paper_0906_1887_gb300 import build as corr_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(corr_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    import ctypes
    path = corr_build.build()
    lib = ctypes.CDLL(path)
    names = _declared("corr.h")
    assert "corr_xengine_run" in names and "corr_plan_create" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_0906_1887_gb300 import corr
    assert set(_declared("corr.h")) <= set(corr.SIGNATURES)


def test_host_only_calls():
    from paper_0906_1887_gb300 import corr
    import numpy as np
    text = open(os.path.join(ROOT, "include", "corr.h")).read()
    assert corr.version() == int(re.search(r"#define CORR_VERSION (\d+)", text).group(1))
    v = np.array([[3, -4], [10, 0]], dtype=np.int64)
    assert corr.average_host(v, 4).tolist() == [[0.75, -1.0], [2.5, 0.0]]


def test_binding_constants_match_header():
    # every CORR_* enum value of the header has the same value under its name in the binding
    from paper_0906_1887_gb300 import corr
    text = open(os.path.join(ROOT, "include", "corr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    consts = re.findall(r"\bCORR_([A-Z0-9_]+)\s*=\s*(-?\d+)", text)
    assert ("OPERANDS_PACKED_F8", "3") in consts
    for name, value in consts:
        assert getattr(corr, name) == int(value), name
