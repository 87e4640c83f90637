"""The C ABI library loads and exports every entry point include/ccm.h declares (no GPU)."""
import os
import re

import pytest

P = pytest.importorskip("paper_2504_00724_gb300")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(ccm_[A-Za-z0-9_]+)\s*\(", src, re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    lib = P.load_library()
    names = declared_functions()
    assert len(names) >= 20
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_error_strings_and_defaults():
    lib = P.lib()
    assert lib.ccm_strerror(0) == b"ok"
    assert b"elliptic" not in lib.ccm_strerror(-1)
    p = P.binding.default_params()
    assert p.nu1 == 3 and p.nu2 == 3 and abs(p.theta - 0.3) < 1e-15 and p.precision == 1


def test_null_arguments_rejected_without_gpu():
    lib = P.lib()
    assert lib.ccm_setup(None, None, None) == -1
    assert lib.ccm_apply(None, None, None, None, 1, None) == -1
    assert lib.ccm_solve(None, None, None, None, 1, None, None) == -1
    assert lib.ccm_query(None, None) == -1
    assert lib.ccm_group_create(None, 1, None, None) == -1
    assert lib.ccm_group_solve(None, None, None, None, None, None) == -1
    assert lib.ccm_group_query(None, None, None) == -1
    lib.ccm_group_free(None)


def test_binding_constants_match_header_and_bench():
    """Every CCM_* enum value of the header that the binding re-exports has the header's value,
    and every binding constant bench.py uses exists."""
    import re
    from pathlib import Path
    root = Path(__file__).resolve().parents[1]
    hdr = (root / "include" / "ccm.h").read_text()
    values = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(CCM_[A-Z0-9_]+)\s*=\s*(-?\d+)", hdr)}
    from paper_2504_00724_gb300 import binding as B
    exported = [n for n in dir(B) if n.startswith("CCM_")]
    assert exported
    for n in exported:
        if n in values:
            assert getattr(B, n) == values[n], n
    used = set(re.findall(r"binding\.(CCM_[A-Z0-9_]+)", (root / "bench.py").read_text()))
    for n in used:
        assert hasattr(B, n), n
