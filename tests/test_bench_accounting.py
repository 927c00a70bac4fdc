"""bench.py's algorithmic accounting and its reference-arm JSON line, on CPU.

The roofline fraction of the bench line divides the algorithmic bytes of one Leja iteration by the
kernel's time, so those bytes are pinned here to a count made independently: the stored entries of
the XXZ chain come from the oracle's CSR builders (checked against Kronecker products in
test_oracle_pins.py), and the per-entry and per-row sizes are those of the data layout (int32
columns, int64 row pointers, float64 values or 62-bit mantissas, int16 row exponents, complex128
vectors and their int64-pair fixed-point copies).
"""
import json
import subprocess
import sys

import numpy as np
import pytest

import bench
import magnus_inputs as mi
import oracle


def _chain_nnz(n):
    c = mi.xxz_chain(7, n, 0.01, 1)
    Hs = oracle.xxz_csr(n, c.J, c.hz, c.delta)
    Hd = oracle.field_x_csr(n)
    return c, int(Hs.rowptr[-1]), int(Hd.rowptr[-1])


@pytest.mark.parametrize("n", [4, 7, 10])
def test_chain_entry_counts(n):
    """H_s: the diagonal plus one entry per anti-parallel bond (half the rows per bond); the field:
    one entry per single-bit flip."""
    c, nnz_s, nnz_d = _chain_nnz(n)
    D = 2 ** n
    assert c.dim == D
    assert nnz_s == D + (n - 1) * D // 2
    assert nnz_d == n * D


def test_bytes_per_iteration_fixed_point_csr():
    """Cf4, 20 spins, fixed point, one substep per exponential and 7 Leja iterations per exponential
    (the substep inputs' copies are shared by 7 iterations)."""
    c = mi.workload2()
    D, n = c.dim, c.nspins
    nnz_s, nnz_d = D + (n - 1) * D // 2, n * D
    nbytes, flops = bench.algorithmic_per_iteration(c, "csr", "CF4", (nnz_s, nnz_d), fixed=True,
                                                    subs_per_it=1.0 / 7.0)
    matrix = nnz_s * (8 + 4) + nnz_d * 4 + (D + 1) * 8 + D * 2
    vectors = D * (16 + 16 + 32) + D * (16 + 16) + D * (16 + 16) / 7.0
    assert nbytes == int(matrix + vectors) == 331949210
    assert flops == 2 * 14 * D


def test_bytes_per_iteration_fp64_csr_and_matrix_free():
    c = mi.workload2()
    D, n = c.dim, c.nspins
    nnz = (D + (n - 1) * D // 2, n * D)
    nbytes, flops = bench.algorithmic_per_iteration(c, "csr", "CF4", nnz, fixed=False)
    assert nbytes == sum(nnz) * 12 + 2 * (D + 1) * 8 + 64 * D
    assert flops == 2 * (2 * sum(nnz) + 14 * D)
    nbytes, flops = bench.algorithmic_per_iteration(c, "mfree", "CF4", (0, 0), fixed=False)
    assert nbytes == 64 * D
    assert flops == 2 * D * ((4 + (n - 1) + 2 * n + 2) + 10)


def test_m4_applies_every_term_twice():
    c = mi.workload2()
    D, n = c.dim, c.nspins
    nnz = (D + (n - 1) * D // 2, n * D)
    b1, _ = bench.algorithmic_per_iteration(c, "csr", "CF4", nnz, fixed=False)
    b4, _ = bench.algorithmic_per_iteration(c, "csr", "M4", nnz, fixed=False)
    matrix = sum(nnz) * 12 + 2 * (D + 1) * 8
    assert b4 - b1 == matrix + 2 * 32 * D  # the second pass over the matrix, u_k written and read back


def test_reference_arm_json_line():
    """`bench.py --impl reference` times the FP64 CPU oracle and prints the contract's line."""
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                         cwd=bench.ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference"
    assert line["unit"] == "steps/s" and line["value"] > 0 and line["steps"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert np.isclose(line["e2e"]["value"], line["value"])


def test_clock_summary_of_sampled_records():
    """The clocks record of the bench line: median SM clock under load, the maximum, and every
    throttle reason seen Active in any sample (nvidia-smi csv,noheader,nounits rows)."""
    s = bench.ClockSampler(0)
    s.out = "\n".join([
        "0, 1965, 2070, 812.4, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2070, 2070, 990.1, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 1800, 2070, 1201.0, 0x0000000000000008, Active, Not Active, Not Active, Not Active",
        "garbage line",
    ])
    got = s.summary()
    assert got["sm_mhz"] == 1965.0 and got["sm_max_mhz"] == 2070.0 and got["samples"] == 3
    assert got["reasons"] == ["hw_slowdown", "sw_power_cap"]
    s.out = ""
    assert s.summary()["reasons"] == ["unavailable"]


def test_traffic_attaches_only_to_a_matching_capture(tmp_path, monkeypatch):
    """A 20-spin run's roofline takes its DRAM traffic from profiles/traffic.json only under the key
    of its storage, method, arithmetic and row layout, and only while the kernel sources hash to the
    capture's; the 10-spin chain never gets one."""
    class C:
        def __init__(self, n):
            self.nspins = n

    def rec(layout):
        return {"fixed_sums": 1, "row_layout": layout, "roofline": {"leja_iterations": 10, "traffic": None}}

    sha = bench.kernel_source_hash(bench.PERSISTENT_SOURCES)
    table = {"wl2_csr_M4_fixed_csr": {"kernel_sha": sha, "dram_bytes_per_iteration": 5},
             "wl2_mfree_CF4_fixed": {"kernel_sha": "0" * 16, "dram_bytes_per_iteration": 7}}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(table))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda files=bench.PERSISTENT_SOURCES: sha)
    r = rec("csr")
    bench.attach_traffic(r, C(20), "csr", "M4")
    assert r["roofline"]["traffic"] == 50 and r["roofline"]["traffic_key"] == "wl2_csr_M4_fixed_csr"
    r = rec(None)
    bench.attach_traffic(r, C(20), "mfree", "CF4")  # captured on other sources: no traffic
    assert r["roofline"]["traffic"] is None and r["roofline"]["traffic_key"] == "wl2_mfree_CF4_fixed"
    r = rec("csr")
    bench.attach_traffic(r, C(20), "csr", "CF4")  # no capture under this key
    assert r["roofline"]["traffic"] is None
    r = rec("csr")
    bench.attach_traffic(r, C(10), "csr", "M4")
    assert r["roofline"]["traffic"] is None and "traffic_key" not in r["roofline"]
