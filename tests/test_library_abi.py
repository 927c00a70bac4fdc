"""The C-ABI library builds for sm_103a, loads without a GPU and exports every declared entry point."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^MAGNUS_API\s+[\w\s\*]+?\b(\w+)\(", src, flags=re.M)
    return names


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("magnus_plan_create", "leja_expv", "magnus_propagate", "magnus_plan_destroy"):
        assert must in names


def test_library_loads_and_exports_every_symbol():
    from paper_1709_06483_gb300 import build, EXPORTS
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_symbols()
    assert sorted(names) == sorted(EXPORTS)
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings_without_gpu():
    import paper_1709_06483_gb300 as mg
    mg.build_lib = None
    lib = mg.load()
    assert lib.magnus_status_string(mg.ENOCONV) == b"MAGNUS_ENOCONV"
    assert lib.magnus_xxz_nnz(20) == 31981568 - 20 * (1 << 20)  # 2^20 + 19 * 2^19
