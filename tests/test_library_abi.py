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
    assert lib.magnus_status_string(mg.EDRIFT) == b"MAGNUS_EDRIFT"
    assert lib.magnus_xxz_nnz(20) == 31981568 - 20 * (1 << 20)  # 2^20 + 19 * 2^19


# C structs of the header and the binding's ctypes mirrors, field by field in declaration order
_STRUCTS = {
    "magnus_term": ("Term", ["kind", "nspins", "nnz", "rowptr", "col", "val", "J", "hz", "delta"]),
    "magnus_coeff": ("Coeff", ["a0", "nmodes", "_pad", "ac", "as", "om"]),
    "magnus_options": ("Options", ["tol_rel", "tol_abs", "rho_max", "m_max", "nvec", "ctas", "precision",
                                   "barrier_timeout_s", "test_skip_arrival", "interval", "fixed_sums", "row_layout", "plain_values", "_reserved",
                                   "norm_check"]),
    "magnus_stats": ("Stats", ["n_exp", "n_substeps", "n_matvec", "n_termapply", "max_m", "status", "m_log",
                               "m_log_cap", "kernel_ms", "grid", "block", "fixed_sums", "row_layout",
                               "norm_drift"]),
    "magnus_batch_item": ("BatchItem", ["dim", "nterms", "_pad", "terms", "coeffs"]),
    "magnus_batch_stats": ("BatchStats", ["n_exp", "n_substeps", "n_matvec", "n_termapply", "max_m", "status",
                                          "m_log", "m_log_cap_per_item", "graph_ms", "block", "cluster",
                                          "fixed_sums", "_pad"]),
}


def test_struct_layouts_match_the_header(tmp_path):
    """sizeof and every offsetof of the header's structs, from a C program compiled with gcc against
    include/magnus.h, equal those of the binding's ctypes structures."""
    import shutil
    import subprocess
    import paper_1709_06483_gb300 as mg
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "magnus.h"', "int main(void) {"]
    for cname, (_, fields) in _STRUCTS.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in fields:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        s, f, v = line.split()
        got[(s, f)] = int(v)
    for cname, (pyname, fields) in _STRUCTS.items():
        cls = getattr(mg, pyname)
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        pyfields = [f[0] for f in cls._fields_]
        assert len(pyfields) == len(fields), cname
        for cf, pf in zip(fields, pyfields):
            assert got[(cname, cf)] == getattr(cls, pf).offset, (cname, cf, pf)
