"""Benchmark: Magnus steps/s and Leja matvec GB/s, against the plain FP64 GPU path.

Headline workload (one Magnus step = one bench step): the open XXZ chain with 20 spins
(dim 2^20, 31,981,568 stored entries as complex128 CSR), J_i ~ U[0.5,1.5], h_i ~ U[-1,1],
drive cos(5t) on sum_i sigma^x_i, step h = 0.005 from t = 0, Leja tolerance 1e-10 (rel + abs),
method Cf4.  Synthetic inputs from magnus_inputs (seeded).  The CSR matrix (640 MB) is larger
than L2, so every Leja iteration streams it from HBM.  The value is the median of --repeats timed
regions of exactly --steps steps.

Beside it, in the same JSON line (one GPU only): the plain FP64 GPU path on the same chain and
steps (complex128 values multiplied in place, FP64 sums, Gershgorin enclosures), the speed-up over
it and the headline state's error against it; the headline path with Gershgorin enclosures; and a
short run of every other workload (10-spin chain CF4/M4, 20-spin M4 and matrix-free, the 13-spin
dense chain in three precisions with their errors, the 512-chain batch, the 16-spin adjoint).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: one process per GPU under torchrun; every rank propagates its own replica (the path
has no exchange step), value = all ranks' steps / max time; only the headline runs.
--impl reference times the FP64 CPU oracle (plain C, one host core) on the same workload, rank 0
only.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Magnus steps/s and Leja matvec GB/s vs plain FP64 GPU path at ≤1e-8 error"
SUMS_FIXED = ("exact int64 fixed point: the sum_i sx_i row sums and the H_s (or bond) products; FP64: "
              "the conversions back, the Leja update and the norms")
HBM_PEAK_FALLBACK = 6800.0
ROW_LAYOUT_NAMES = {0: None, 1: "staged", 2: "csr", 3: "sliced"}
SMS, FP64_FMA_PER_CLK, SM_MAX_MHZ = 152, 2, 2070.0
FP64_PEAK_TFLOPS = SMS * FP64_FMA_PER_CLK * 2 * SM_MAX_MHZ * 1e6 / 1e12  # 1.259 TFLOP/s derived


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def max_over_ranks(value, device="cpu"):
    """Maximum of a per-rank float over all ranks of the default process group (identity alone)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(units_per_rank, ms_max, world):
    """Whole-job throughput of independent replicas: all ranks' units / the slowest rank's time."""
    return world * units_per_rank / (ms_max / 1e3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# --------------------------------------------------------------------------- workload
def workload_terms(mg, c, storage):
    if storage == "csr":
        return [mg.build_xxz_csr(c.nspins, c.J, c.hz, c.delta), mg.build_field_x_csr(c.nspins)]
    if storage == "csr_real":  # float64 values: 12 B per stored entry
        return [mg.build_xxz_csr(c.nspins, c.J, c.hz, c.delta).as_real(), mg.build_field_x_csr(c.nspins).as_real()]
    return [mg.XXZTerm(c.nspins, c.J, c.hz, c.delta), mg.FieldXTerm(c.nspins)]


def drives(mg, c):
    return [mg.Drive.const(), mg.Drive(c.drive_a0, c.drive_ac, c.drive_as, c.drive_om)]


def algorithmic_per_iteration(c, storage, variant, nnz_terms, fixed=False, subs_per_it=0.0):
    """Bytes and FP64 work one Leja iteration needs (real-valued Hamiltonian, complex state).

    storage "csr_plain": the plain FP64 path (options.plain_values): complex128 values read in place
    (16 B + 4 B column per entry) and multiplied as complex numbers (4 FP64 instructions per entry).

    nnz_terms: stored entries of (H_s, sum_i sx_i) for CSR storage.  fixed: the fixed-point
    arithmetic of the linear generators: the pattern term sum_i sx_i (every stored value 1) is
    summed exactly in 64-bit integers, and (CSR) the products of H_s are 62-bit value mantissas
    times the fixed-point vector.

    Bytes, CSR: per stored entry 8 B value + 4 B column (the terms are real-valued: in complex
    storage the plan multiplies the real parts from a float64 copy it keeps; in fixed point the
    value is an 8 B mantissa), per row 8 B row pointer per term, plus per row 16 B read of w_{j-1},
    16 B write of w_j and 16 + 16 B read and write of p; matrix-free: the vector traffic only.  With
    fixed-point arithmetic the pattern term needs its columns only (4 B per entry, rows of one length
    need no row pointers), H_s adds a 2 B row exponent, and every row adds the 16 B write of the
    fixed-point copy of w_j and the 16 B read of that of w_{j-1}; the copy of each substep input
    costs 16 + 16 B per row once per substep (subs_per_it substeps per iteration).  M4 applies every
    term twice and writes and reads back u_k (2 x 32 B/row).

    FP64 work is counted in FMA-equivalent flops: every FP64 instruction the method needs (add,
    multiply or fused multiply-add) counts 2, because on GB300 each occupies one slot of the FP64
    pipe (2 per clock per SM, peak 152 x 2 x 2 x 2070 MHz = 1.259 TFLOP/s).  Per row: CSR needs 2
    instructions per stored entry of a term multiplied in FP64 (none in fixed point); the
    matrix-free XXZ row needs 4 for the
    diagonal, 2 per active bond ((n-1)/2 on average), 2 n for the field sum and 2 to weight it;
    both need 4 for the weighted combination (CSR) or none extra (matrix-free), 2 for the shift, 4
    for the Newton update of p and 4 for the two squared norms.  Fixed-point sums and products are
    integer work, outside the FP64 count: what stays FP64 is 14 instructions per row in both
    families.

    M6 applies every term 17 times per iteration (once per input vector of its five passes and the
    final one); its 23 intermediate vectors are each written once and read back once or twice:
    17 gathered inputs + 23 writes + 16 re-reads of 16 B per row on top of the Leja update, and 27
    combinations of the term values (2 instructions per term each) plus about 70 instructions of
    commutator arithmetic per row."""
    D = c.dim
    passes = {"M4": 2, "M6": 17}.get(variant, 1)
    fixed = fixed and variant != "M6"
    vec_bytes = 64 * D
    if fixed:
        vec_bytes += 32 * D + 32 * D * subs_per_it
    if variant == "M4":
        # u_k written and read back (2 x 32 B/row); in fixed point also their copies (2 x 32 B/row)
        vec_bytes += 2 * 16 * D * 2 * (2 if fixed else 1)
    if variant == "M6":
        vec_bytes += (17 + 23 + 16) * 16 * D
    if storage == "csr_plain":  # complex128 values multiplied in place: 16 B value + 4 B column, 4 FMAs
        nnz_s, nnz_c = nnz_terms
        mat = 20 * (nnz_s + nnz_c) + 2 * 8 * (D + 1)
        inst = passes * 4 * (nnz_s + nnz_c) + (4 + 2 + 4 + 4) * D + (8 * D if variant == "M4" else 0)
    elif storage in ("csr", "csr_real"):
        nnz_s, nnz_c = nnz_terms
        if fixed:
            mat = 12 * nnz_s + 4 * nnz_c + 8 * (D + 1) + 2 * D
            # FP64 left per row: linear 14; M4 24 (scaling the pattern term's sums, the weighted
            # u_k, the commutator difference and its weight, -i, shift, p, norms)
            inst = (24 if variant == "M4" else 14) * D
        else:
            mat = 12 * (nnz_s + nnz_c) + 2 * 8 * (D + 1)
            inst = passes * 2 * (nnz_s + nnz_c) + (4 + 2 + 4 + 4) * D + (8 * D if variant == "M4" else 0)
    elif fixed:
        # matrix-free in fixed point: bonds and field are integer work; FP64 keeps the diagonal (2),
        # adding it to the converted bond sum (2), weighting the field (2), p (4) and the norms (4);
        # M4 26 per row (the XXZ diagonal in both phases, the weighted u_k, the commutator, -i, shift)
        mat = 0
        inst = (26 if variant == "M4" else 2 + 2 + 2 + 4 + 4) * D
    else:
        n = c.nspins
        mat = 0
        inst = passes * D * (4 + (n - 1) + 2 * n + 2) + (2 + 4 + 4) * D + (8 * D if variant == "M4" else 0)
    if variant == "M6":
        inst += (27 * 2 * 2 + 70 - 4) * D  # combinations and commutator arithmetic (no separate weighting)
    return int(passes * mat + vec_bytes), int(2 * inst)


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 50 ms while the timed region runs (the
    default 20-spin region lasts about 0.15 s)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = [r.split(",") for r in (self.out or "").strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, name in enumerate(names):
                if r[5 + k].strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "samples": len(rows),
                "reasons": sorted(reasons)}


# sources whose change can change the persistent kernel's DRAM traffic (the kernel, its rows, and the
# plan set-up that chooses the matrices' layout and the kernel instantiation)
PERSISTENT_SOURCES = ("leja_persistent.cu", "rows.cuh", "csr_stage.cuh", "tcgen05.cuh", "persist_common.cuh",
                      "magnus_internal.cuh", "magnus_api.cu")
BATCH_SOURCES = ("batched.cu", "rows.cuh", "persist_common.cuh", "magnus_internal.cuh")
DENSE_TC_SOURCES = ("dense_persistent.cu", "dense_tc.cuh", "tcgen05.cuh", "persist_common.cuh", "magnus_internal.cuh")


def kernel_source_hash(files=PERSISTENT_SOURCES):
    """Hash of every source file a kernel is compiled from."""
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_1709_06483_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(workload_key, files=PERSISTENT_SOURCES):
    """DRAM bytes per Leja iteration from a committed ncu summary, if it matches this kernel source."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(p)).get(workload_key)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("kernel_sha") != kernel_source_hash(files):
        return None
    return rec.get("dram_bytes_per_iteration")


# --------------------------------------------------------------------------- our arm
def xxz_roofline(c, storage, variant, nnz_terms, st, kms, traffic_key=None):
    """Roofline of the persistent Leja kernel from its own CUDA-event duration (kms): algorithmic
    bytes and FMA-equivalent FP64 flops per Leja iteration (algorithmic_per_iteration) times the
    iterations; the larger of the HBM and FP64 times sets the bound."""
    nmv = st["n_matvec"]
    fixed = bool(st["fixed_sums"])
    bytes_it, flops_it = algorithmic_per_iteration(c, storage, variant, nnz_terms, fixed, st["n_substeps"] / nmv)
    gbs = bytes_it * nmv / (kms / 1e3) / 1e9
    tflops = flops_it * nmv / (kms / 1e3) / 1e12
    peaks = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", HBM_PEAK_FALLBACK))
    t_hbm, t_alu = bytes_it / (hbm_peak * 1e9), flops_it / (FP64_PEAK_TFLOPS * 1e12)
    traffic_it = profiled_traffic(traffic_key) if traffic_key else None
    if t_alu >= t_hbm:
        roof = {"bound": "alu", "achieved": round(tflops, 4), "peak": round(FP64_PEAK_TFLOPS, 4),
                "unit": "TFLOP/s", "frac": round(tflops / FP64_PEAK_TFLOPS, 4)}
    else:
        roof = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(gbs / hbm_peak, 4)}
    roof["traffic"] = None if traffic_it is None else int(traffic_it * nmv)
    roof.update({"kernel": "k_magnus_persistent", "launch_ms": round(kms, 3), "leja_iterations": nmv,
                 "algorithmic_bytes_per_iteration": bytes_it, "algorithmic_flops_per_iteration": flops_it,
                 "hbm_gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm_peak, 4),
                 "fp64_tflops": round(tflops, 4), "fp64_frac": round(tflops / FP64_PEAK_TFLOPS, 4),
                 "peak_source": ("hbm: MEASURED_PEAKS.json copy, of measured" if "hbm_gbs" in peaks else
                                 f"hbm: {HBM_PEAK_FALLBACK:.0f} GB/s, of fallback (no MEASURED_PEAKS.json)")
                                + "; fp64: 152 SMs x 2 FP64 instructions/clk x 2 flops x 2070 MHz (FMA-equivalent flops)"})
    return roof


def measure_xxz(mg, c, terms, storage, variant, steps, warmup, repeats, interval="lanczos", fixed=True, rows="auto",
                plain=False, world=1, local=0, keep_state=False, traffic_key=None):
    """Steps/s of magnus_propagate on chain c: `warmup` untimed steps, then `repeats` timed regions of
    exactly `steps` steps from the same psi0 and t0, each bracketed by a barrier and a device
    synchronisation, timed with CUDA events on the launching stream; clocks sampled over all of them.
    The roofline comes from the persistent kernel's own CUDA-event time of the median repeat."""
    import torch
    stream = torch.cuda.current_stream()
    nnz_terms = tuple(t.col.numel() for t in terms) if storage.startswith("csr") else (0, 0)
    plan = mg.Plan(c.dim, terms, drives(mg, c), interval=interval, fixed_sums=fixed, rows=rows,
                   plain_values=plain)
    psi0 = torch.from_numpy(c.psi0).cuda()
    psi = psi0.clone()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    if warmup:
        plan.propagate(psi, 0.0, c.h, warmup, variant)
    ms, sts = [], []
    with ClockSampler(local) as clk:
        for _ in range(max(1, repeats)):
            psi.copy_(psi0)
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = plan.propagate(psi, c.t0, c.h, steps, variant)
            e1.record(stream)
            barrier()
            ms.append(max_over_ranks(e0.elapsed_time(e1), "cuda"))
            sts.append(st)
    order = sorted(range(len(ms)), key=lambda i: ms[i])
    mid = order[len(order) // 2]
    rates = sorted(replica_rate(steps, m, world) for m in ms)
    st = sts[mid]
    rkey = "csr_plain" if plain else storage
    out = {"steps_per_s": round(replica_rate(steps, ms[mid], world), 3),
           "min": round(rates[0], 3), "max": round(rates[-1], 3), "repeats": len(ms), "steps": steps,
           "ms_per_step": round(ms[mid] / steps, 4), "leja_iterations": st["n_matvec"], "max_degree": st["max_m"],
           "us_per_leja_iteration": round(st["kernel_ms"] * 1e3 / max(1, st["n_matvec"]), 2),
           "fixed_sums": st["fixed_sums"], "row_layout": ROW_LAYOUT_NAMES.get(st["row_layout"]), "grid": st["grid"],
           "norm_drift": st["norm_drift"],
           "roofline": xxz_roofline(c, rkey, variant, nnz_terms, st, st["kernel_ms"], traffic_key),
           "clocks": clk.summary()}
    if keep_state:
        out["_psi"] = psi.clone()
        out["_plan"] = plan
    else:
        plan.close()
    return out


def run_ours(args):
    import torch

    import magnus_inputs as mi
    import paper_1709_06483_gb300 as mg

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    mg.load()
    c = mi.workload1() if args.workload == "xxz10" else mi.workload2()
    variant, storage = args.variant, args.storage
    stream = torch.cuda.current_stream()
    terms = workload_terms(mg, c, storage)
    nnz_terms = tuple(t.col.numel() for t in terms) if storage.startswith("csr") else (0, 0)
    nnz_total = sum(nnz_terms) if storage.startswith("csr") else None
    fixed = bool(args.fixed_sums)
    head = measure_xxz(mg, c, terms, storage, variant, args.steps, args.warmup, args.repeats, args.interval, fixed,
                       args.rows, False, world, local, keep_state=True)
    attach_traffic(head, c, storage, variant)
    plan, psi_head = head.pop("_plan"), head.pop("_psi")
    value = head["steps_per_s"]
    psi = torch.empty_like(psi_head)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # end-to-end through the public API with host buffers: every step copies its input state from
    # pinned host memory, runs one Magnus step (magnus_propagate, which returns when the step is
    # done) and copies the result back to pinned host memory.  Two device state buffers: the next
    # step's input copy and the previous step's result copy run on a copy stream while the current
    # step computes.  Every step restarts from the same host state (independent one-step problems).
    host_in = torch.from_numpy(c.psi0).pin_memory()
    host_out = [torch.empty_like(host_in).pin_memory() for _ in range(2)]
    bufs = [psi, torch.empty_like(psi)]
    cstream = torch.cuda.Stream()
    ready = [torch.cuda.Event() for _ in range(2)]  # input of the step on bufs[i] copied
    done = [torch.cuda.Event() for _ in range(2)]   # step on bufs[i] finished
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(cstream)
    with torch.cuda.stream(cstream):
        bufs[0].copy_(host_in, non_blocking=True)
        ready[0].record(cstream)
    for n in range(e2e_steps):
        i = n % 2
        stream.wait_event(ready[i])
        if n + 1 < e2e_steps:  # after the previous result's read of bufs[1 - i] (same copy stream)
            with torch.cuda.stream(cstream):
                bufs[1 - i].copy_(host_in, non_blocking=True)
                ready[1 - i].record(cstream)
        plan.propagate(bufs[i], c.t0 + n * c.h, c.h, 1, variant)
        done[i].record(stream)
        cstream.wait_event(done[i])
        with torch.cuda.stream(cstream):
            host_out[i].copy_(bufs[i], non_blocking=True)
    cstream.wait_stream(stream)
    e1.record(cstream)
    barrier()
    cstream.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), "cuda")
    e2e = {"value": round(world * e2e_steps / (e2e_ms / 1e3), 3), "unit": "steps/s",
           "h2d_bytes_per_step": host_in.numel() * 16, "d2h_bytes_per_step": host_out[0].numel() * 16,
           "steps": e2e_steps, "copies": "double-buffered: next input H2D and previous result D2H on a copy "
           "stream during the current step; each step an independent one-step problem from the same host state"}
    plan.close()

    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+i64" if head["fixed_sums"] else "f64",
        "data": "synthetic",
        "config": {"workload": f"xxz_chain_{c.nspins}spins_{storage}_{variant.lower()}", "spins": c.nspins, "dim": c.dim,
                   "nnz": nnz_total, "h": c.h, "t0": c.t0, "variant": variant, "storage": storage,
                   "interval": args.interval, "row_layout": head["row_layout"],
                   "sums": SUMS_FIXED if head["fixed_sums"] else "FP64",
                   "leja_tol": 1e-10, "l2": "inputs larger than L2: the 640 MB CSR is streamed every iteration"
                   if storage.startswith("csr") else "matrix-free; 4 state vectors of 16 MB stay L2-resident",
                   "parallelism": f"replicas x{world}"},
        "timing": {"repeats": head["repeats"], "steps_per_repeat": args.steps, "value": "median of the repeats",
                   "min": head["min"], "max": head["max"]},
        "matvec_gbs": head["roofline"]["hbm_gbs"],
        "leja": {"iterations": head["leja_iterations"], "max_degree": head["max_degree"],
                 "us_per_iteration": head["us_per_leja_iteration"],
                 "norm_drift": head["norm_drift"],
                 "norm_drift_how": "largest | ||p|| - ||v|| | / ||v|| over the substeps (the a posteriori check's "
                                   "quantity; 0 up to rounding and the Leja tolerance)"},
        "roofline": head["roofline"],
        "e2e": e2e,
        "gpu_launches": 2 * head["repeats"],
        "gpu_launches_detail": "timed regions: k_exp_setup + k_magnus_persistent per magnus_propagate call, "
                               "one call per repeat",
        "clocks": head["clocks"],
    }
    if world == 1 and not args.headline_only:
        # the metric's comparison: the plain FP64 GPU path on the same chain, steps and start state
        # (complex128 values multiplied in place, FP64 sums, Gershgorin enclosures, rows from global
        # memory), and the state error of the headline path against it
        try:
            plain = measure_xxz(mg, c, workload_terms(mg, c, "csr"), "csr", variant, args.steps, 1,
                                min(3, args.repeats), "gershgorin", False, "csr", True, world, local,
                                keep_state=True, traffic_key=f"wl2_csr_plain_{variant}")
            plain.pop("_plan").close()
            pp = plain.pop("_psi")
            err = float(torch.linalg.norm(psi_head - pp) / torch.linalg.norm(pp))
            rig = measure_xxz(mg, c, terms, storage, variant, args.steps, 1, 1, "gershgorin", fixed,
                              args.rows, False, world, local)
            line["vs_plain_fp64"] = {
                "plain_fp64": {k: plain[k] for k in ("steps_per_s", "min", "max", "repeats", "leja_iterations",
                                                     "us_per_leja_iteration", "roofline")},
                "plain_how": "complex128 CSR values multiplied in place (options.plain_values), FP64 sums, "
                             "Gershgorin enclosures, rows read from global memory",
                "speedup": round(value / plain["steps_per_s"], 3),
                "state_error": err, "state_error_bound": 1e-8,
                "state_error_how": f"relative 2-norm of the headline path's state after the {args.steps} timed "
                                   "steps against the plain FP64 GPU path's, same psi0 and t0",
                "gershgorin_enclosures": {k: rig[k] for k in ("steps_per_s", "leja_iterations",
                                                              "us_per_leja_iteration")},
                "gershgorin_how": "the headline path with rigorous Gershgorin enclosures instead of Lanczos"}
        except Exception as exc:  # noqa: BLE001 - the headline line is still printed
            line["vs_plain_fp64"] = {"error": repr(exc)[:300]}
        line["workloads"] = run_all_workloads(args, mg, mi, local)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(variant, args.cpu_steps, args.interval)
        if "workloads" in line:
            for name, rec in workload_cpu_baselines().items():
                if name in line["workloads"]:
                    line["workloads"][name]["cpu_oracle"] = rec
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# --------------------------------------------------------------------------- every workload
def attach_traffic(rec, c, storage, variant):
    """The roofline's `traffic` of a 20-spin run: DRAM bytes per Leja iteration from the committed ncu
    capture of the same workload, storage, method and row layout (profiles/traffic.json, valid only
    for the sources it was taken on) times the run's Leja iterations; None without such a capture."""
    if c.nspins != 20:
        return
    key = f"wl2_{storage}_{variant}" + ("_fixed" if rec["fixed_sums"] else "") + (
        f"_{rec['row_layout']}" if rec["row_layout"] else "")
    t = profiled_traffic(key)
    rec["roofline"]["traffic"] = None if t is None else int(t * rec["roofline"]["leja_iterations"])
    rec["roofline"]["traffic_key"] = key


def wl_xxz(mg, mi, c, storage, variant, steps, repeats, interval, local, label):
    terms = workload_terms(mg, c, storage)
    r = measure_xxz(mg, c, terms, storage, variant, steps, 3, repeats, interval, True, "auto", False, 1, local)
    attach_traffic(r, c, storage, variant)
    r["workload"] = label
    return r


def run_all_workloads(args, mg, mi, local):
    """One short run of every workload of the benchmark configs, each with its own roofline: the
    10-spin chain (CF4 and M4, latency-bound), the 20-spin chain with M4 and matrix-free, the 13-spin
    dense chain in three precisions with their state errors, the 512-chain batch and the 16-spin
    adjoint gradient.  Each entry is independent; a failure is recorded and the rest still run."""
    out = {}
    jobs = [
        ("cfg1_xxz10_csr_cf4", lambda: wl_xxz(mg, mi, mi.workload1(), "csr", "CF4", 100, 5, args.interval, local,
                                               "10-spin XXZ chain, CSR, CF4, h = 0.01, t in [0, 1] (100 steps)")),
        ("cfg1_xxz10_csr_m4", lambda: wl_xxz(mg, mi, mi.workload1(), "csr", "M4", 100, 5, args.interval, local,
                                              "10-spin XXZ chain, CSR, M4, h = 0.01, t in [0, 1] (100 steps)")),
        ("cfg2_xxz20_csr_m4", lambda: wl_xxz(mg, mi, mi.workload2(), "csr", "M4", 100, 3, args.interval, local,
                                              "20-spin XXZ chain, CSR, M4, h = 0.005, 100 steps")),
        ("cfg2_xxz20_mfree_cf4", lambda: wl_xxz(mg, mi, mi.workload2(), "mfree", "CF4", 100, 3, args.interval,
                                                 local, "20-spin XXZ chain, matrix-free, CF4, h = 0.005, 100 steps")),
        ("cfg3_dense13", lambda: dense_workload(mg, mi, local, nvec=64, nspins=13, rate_steps=(2, 4, 100),
                                                err_states=4, err_steps=100)),
        ("cfg3_dense13_m4_tensor", lambda: dense_workload(mg, mi, local, nvec=64, nspins=13, rate_steps=(2, 0, 50),
                                                          err_states=4, err_steps=50, variant="M4",
                                                          modes=("fp64", "tensor_sliced"))),
        ("cfg4_batch512", lambda: batch_workload(mg, mi, local, steps=100, storage="csr", fixed=True)),
        ("cfg5_adjoint16", lambda: adjoint_workload(mg, mi, local, nsteps=1000)),
    ]
    for name, fn in jobs:
        t = time.perf_counter()
        try:
            out[name] = fn()
        except Exception as exc:  # noqa: BLE001
            out[name] = {"error": repr(exc)[:300]}
        out[name]["wall_s"] = round(time.perf_counter() - t, 2)
    return out


# --------------------------------------------------------------------------- dense workload
def dense_workload(mg, mi, local, nvec=64, nspins=13, rate_steps=(2, 4, 100), err_states=4, err_steps=100,
                   variant="CF4", warmup=1, modes=("fp64", "fp32_split", "tensor_sliced")):
    """Long-range chain with dense H_s and dense sum sx (dim 2^nspins), nvec states, h = 0.01: the
    plain FP64 path, the FP32-split path and the tensor-core sliced path.  Rates from nvec states
    over rate_steps[i] steps (FP64, split, tensor); state errors of the reduced-precision paths
    against the FP64 GPU path on the first err_states states over err_steps steps (the states do not
    interact: every state column has its own scales and stop test)."""
    import torch
    c = mi.workload3(nvec=nvec, nspins=nspins)
    Hs = mg.build_longrange_dense(c.nspins, c.hz, 1.5, c.delta)
    Hd = mg.build_field_x_dense(c.nspins)
    stream = torch.cuda.current_stream()
    prec_of = {"fp64": mg.FP64, "fp32_split": mg.FP32_SPLIT, "tensor_sliced": mg.TENSOR_SLICED}
    D = c.dim
    psi_all = torch.from_numpy(c.psi0).cuda()
    res, finals = {}, {}
    for i, prec in enumerate(("fp64", "fp32_split", "tensor_sliced")):
        if prec not in modes:
            continue
        nsteps = rate_steps[i]
        plan = mg.Plan(D, [mg.DenseTerm(Hs), mg.DenseTerm(Hd)], drives(mg, c), nvec=nvec, precision=prec_of[prec])
        psi = psi_all.clone()
        if warmup:
            plan.propagate(psi, 0.0, c.h, 1, variant)
        psi.copy_(psi_all)
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            s0.record(stream)
            st = plan.propagate(psi, 0.0, c.h, nsteps, variant)
            s1.record(stream)
            torch.cuda.synchronize()
        ms = s0.elapsed_time(s1)
        nmv = st["n_matvec"] / nvec  # Leja iterations (all vectors advance together)
        # per Leja iteration: each dense term read once (16 B/element) + nvec vectors x 64 B/row;
        # FP64 work: 2 FMAs per H element per vector per term (real H x complex state)
        bytes_it = 2 * 16 * D * D + nvec * 64 * D
        fma_it = 2 * 2 * D * D * nvec
        kms = st["kernel_ms"]
        r = {"steps_per_s": round(nsteps / (ms / 1e3), 4), "steps": nsteps, "ms_per_step": round(ms / nsteps, 3),
             "leja_iterations": nmv, "kernel_ms": round(kms, 3),
             "matvec_gbs": round(bytes_it * nmv / (kms / 1e3) / 1e9, 2),
             "fp64_equiv_tflops": round(2 * fma_it * nmv / (kms / 1e3) / 1e12, 4), "clocks": clk.summary()}
        if prec == "tensor_sliced":
            # issued bf16 MMA work (tcgen05): 10 digit pairs x 2 flops x D^2 x 128 columns per dense term
            # and product phase; phases per Leja iteration: 1 (linear generators), 2 for M4 (u_k = H_k w,
            # then the one commutator pair of the two dense terms)
            phases = 2 if variant == "M4" else 1
            r["product_phases_per_iteration"] = phases
            r["bf16_tflops_issued"] = round(phases * 10 * 2 * D * D * 128 * 2 * nmv / (kms / 1e3) / 1e12, 2)
        if prec == "fp64":
            r["roofline"] = {"bound": "alu", "achieved": r["fp64_equiv_tflops"], "peak": round(FP64_PEAK_TFLOPS, 4),
                             "unit": "TFLOP/s", "frac": round(r["fp64_equiv_tflops"] / FP64_PEAK_TFLOPS, 4)}
        res[prec] = r
        if prec != "fp64" and nsteps >= err_steps:
            finals[prec] = psi[:err_states].clone()
        plan.close()
    # state errors: the first err_states states over err_steps steps against the FP64 GPU path
    errs = {}
    want = [p for p in ("fp32_split", "tensor_sliced") if p in modes]
    if "fp64" in modes and err_states > 0 and want:
        plan = mg.Plan(D, [mg.DenseTerm(Hs), mg.DenseTerm(Hd)], drives(mg, c), nvec=err_states)
        ref = psi_all[:err_states].clone()
        plan.propagate(ref, 0.0, c.h, err_steps, variant)
        plan.close()
        for prec in want:
            got = finals.get(prec)
            if got is None:
                plan = mg.Plan(D, [mg.DenseTerm(Hs), mg.DenseTerm(Hd)], drives(mg, c), nvec=err_states,
                               precision=prec_of[prec])
                got = psi_all[:err_states].clone()
                plan.propagate(got, 0.0, c.h, err_steps, variant)
                plan.close()
            e = torch.linalg.norm(got - ref, dim=1) / torch.linalg.norm(ref, dim=1)
            errs[prec] = float(e.max())
    peaks = measured_peaks()
    bf16_peak = float(peaks.get("bf16_tflops", 1900.0))
    if "tensor_sliced" in res:
        ts = res["tensor_sliced"]
        # DRAM bytes per Leja iteration from the 12-spin capture (dim 4096) of the same method, scaled
        # by (dim / 4096)^2: the traffic is the digits of the dense terms, read once per product phase
        # (one per Leja iteration for linear generators, two for M4)
        t12 = profiled_traffic("dense_tc_12spins_64states" + ("_m4" if variant == "M4" else ""), DENSE_TC_SOURCES)
        ts["roofline"] = {"bound": "tensor", "kernel": "k_dense_persistent (tcgen05 digit products)",
                          "achieved": ts["bf16_tflops_issued"], "peak": bf16_peak, "unit": "TFLOP/s",
                          "frac": round(ts["bf16_tflops_issued"] / bf16_peak, 4),
                          "traffic": None if t12 is None or nvec != 64 else int(t12 * (D / 4096) ** 2),
                          "traffic_unit": "DRAM bytes per Leja iteration (12-spin ncu capture scaled by (dim/4096)^2)",
                          "peak_source": ("MEASURED_PEAKS.json bf16_tflops (burst), of measured"
                                          if "bf16_tflops" in peaks else
                                          "1900 TFLOP/s bf16 burst, of fallback (no MEASURED_PEAKS.json)"),
                          "work": "10 bf16 digit-pair products x 2 flops x dim^2 x 128 columns per dense term per "
                                  "product phase (1 per Leja iteration, 2 for M4)"}
    f64 = res.get("fp64")
    return {"workload": f"long-range chain, {nspins} spins, dense H_s and sum sx (2 x {16 * D * D / 1e9:.2f} GB "
                        f"complex128), {nvec} states, {variant}, h = 0.01",
            "paths": res,
            "speedup_vs_fp64": ({k: round(res[k]["steps_per_s"] / f64["steps_per_s"], 3) for k in res if k != "fp64"}
                                if f64 else None),
            "state_error_vs_fp64": errs,
            "state_error_how": f"max over states 0..{err_states - 1} of the relative 2-norm error after {err_steps} "
                               f"steps against the FP64 GPU path",
            "state_error_bound": 1e-8}


def run_dense13(args):
    """The dense workload alone (one JSON line); the line's value is the fastest path's rate."""
    import torch

    import magnus_inputs as mi
    import paper_1709_06483_gb300 as mg

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    mg.load()
    modes = tuple(m for m in args.dense_prec.split(",") if m)
    r = dense_workload(mg, mi, local, nvec=args.states, nspins=args.spins,
                       rate_steps=(min(args.steps, 4), min(args.steps, 10), args.steps), err_states=min(4, args.states),
                       err_steps=args.steps, variant=args.variant, warmup=args.warmup, modes=modes)
    paths = r["paths"]
    best = paths.get("tensor_sliced") or paths.get("fp32_split") or paths.get("fp64")
    line = {
        "metric": METRIC, "value": best["steps_per_s"], "unit": "steps/s", "n_gpus": world,
        "steps": best["steps"], "warmup": args.warmup, "ms_per_step": best["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16-digits(f64-equivalent)" if "tensor_sliced" in paths else "f64", "data": "synthetic",
        "config": {"workload": f"longrange_chain_{args.spins}spins_dense_{args.states}states_{args.variant.lower()}",
                   "spins": args.spins, "states": args.states, "variant": args.variant,
                   "l2": "inputs larger than L2: two dense terms of 16 dim^2 bytes"},
        "roofline": best.get("roofline"), "gpu_launches": 2, **{k: v for k, v in r.items() if k != "workload"},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- batched workload
def batch_workload(mg, mi, local, steps=100, storage="csr", fixed=True, variant="CF4", warmup=1, sample_every=32,
                   config=None):
    """512 independent XXZ chains of 8-14 spins (dims 256..16384), per-chain drive A cos(w t), Cf4,
    h = 0.01, one persistent launch under a replayed CUDA graph.  A step advances every chain by one
    Magnus step.  Compared with one plan and launch per chain on every sample_every-th chain."""
    import torch
    chains = mi.workload4()
    probs = []
    nnz_s = nnz_c = 0  # stored entries of H_s and of sum_i sx_i over all chains
    for c in chains:
        terms = workload_terms(mg, c, storage)
        if storage.startswith("csr"):
            nnz_s += terms[0].col.numel()
            nnz_c += terms[1].col.numel()
        probs.append((c.dim, terms, drives(mg, c)))
    nnz = nnz_s + nnz_c
    # config (CTA size, cluster size) fixes the launch shape; None lets the batch's autotuner choose
    B = mg.Batch(probs, fixed_sums=fixed, **({"ctas": -(config[0] + 65536 * config[1])} if config else {}))
    psi0 = [torch.from_numpy(c.psi0).cuda() for c in chains]
    psis = [p.clone() for p in psi0]
    B.propagate(psis, 0.0, 0.01, warmup or 1, variant)  # autotune + warm-up
    for p, q in zip(psis, psi0):
        p.copy_(q)
    B.propagate(psis, 0.0, 0.01, steps, variant)         # captures the graph for these steps
    for p, q in zip(psis, psi0):
        p.copy_(q)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t = time.perf_counter()
        st = B.propagate(psis, 0.0, 0.01, steps, variant)  # replay
        wall = time.perf_counter() - t
    gms = st["graph_ms"]
    rows = sum(c.dim for c in chains)
    fixed = bool(st["fixed_sums"])
    # as algorithmic_per_iteration: with fixed sums the field term needs its columns only and the
    # vectors add the fixed-point copies (32 B per row, and 32 B per row once per substep)
    vec = 64 * rows + ((32 + 32 * st["n_substeps"] / st["n_matvec"]) * rows if fixed else 0)
    if fixed:  # H_s mantissas + columns, its row pointers and exponents; the field's columns only
        mat = 12 * nnz_s + 4 * nnz_c + sum(8 * (c.dim + 1) + 2 * c.dim for c in chains)
    else:  # real values: complex-stored ones are multiplied from the batch's float64 copy
        mat = 12 * nnz + sum(2 * 8 * (c.dim + 1) for c in chains)
    bytes_it = mat + vec if storage.startswith("csr") else vec
    # Leja iterations differ per chain; algorithmic bytes weighted by each chain's iterations are
    # approximated with the mean iteration count per chain
    iters_per_chain = st["n_matvec"] / len(chains)
    gbs = bytes_it * iters_per_chain / (gms / 1e3) / 1e9
    if fixed:  # fixed-point sums and products: 14 FP64 instructions per row remain in both families
        inst_it = 14 * rows
    elif storage.startswith("csr"):
        inst_it = 2 * nnz + 14 * rows
    else:
        inst_it = sum(c.dim * (4 + (c.nspins - 1) + 2 * c.nspins + 2) + 10 * c.dim for c in chains)
    tflops = 2 * inst_it * iters_per_chain / (gms / 1e3) / 1e12
    peaks = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", HBM_PEAK_FALLBACK))
    # one plan and one persistent launch per chain for comparison (same arithmetic), on a sample of
    # the chains (sizes drawn independently, so the sample is unbiased), extrapolated by the count
    seq_steps = min(steps, 20)
    sample = chains[::sample_every]
    seq_ms = 0.0
    for c in sample:
        q = mg.Plan(c.dim, workload_terms(mg, c, storage), drives(mg, c), fixed_sums=fixed)
        x = torch.from_numpy(c.psi0).cuda()
        q.propagate(x, 0.0, 0.01, 1, variant)
        torch.cuda.synchronize()
        t = time.perf_counter()
        q.propagate(x, 0.0, 0.01, seq_steps, variant)
        torch.cuda.synchronize()
        seq_ms += (time.perf_counter() - t) * 1e3
        q.close()
    share = len(sample) / len(chains)
    seq_rate = seq_steps / (seq_ms / share / 1e3)
    batch_rate = steps / (gms / 1e3)
    # DRAM bytes per step from the committed capture of this launch shape, if it matches the sources
    tkey = f"batch512_{storage}_{variant}_{st['block']}x{st['cluster']}" + ("_fixed" if fixed else "")
    t_step = profiled_traffic(tkey, BATCH_SOURCES)
    B.close()
    return {
        "workload": f"512 XXZ chains of 8-14 spins, {storage}, {variant}, h = 0.01, {steps} steps per graph replay",
        "steps_per_s": round(batch_rate, 3), "steps": steps, "ms_per_step": round(gms / steps, 4),
        "unit": "steps/s (all 512 chains per step)", "chain_steps_per_s": round(len(chains) * batch_rate, 1),
        "chains": len(chains), "rows": rows, "nnz": nnz, "cta_size": st["block"], "cluster_size": st["cluster"],
        "fixed_sums": int(fixed), "leja_iterations": st["n_matvec"], "matvec_gbs": round(gbs, 1),
        "per_chain_plans": {"steps_per_s": round(seq_rate, 3), "how": f"one plan and launch per chain (same "
                            f"arithmetic), {len(sample)} of 512 chains x {seq_steps} steps, wall time scaled by the "
                            f"chain count (x {1 / share:.0f})"},
        "speedup_vs_per_chain_plans": round(batch_rate / seq_rate, 2),
        # the larger of the FP64 and HBM times per iteration sets the bound, as for the single chain
        "roofline": dict(({"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                           "frac": round(gbs / hbm_peak, 4)}
                          if gbs / hbm_peak > tflops / FP64_PEAK_TFLOPS else
                          {"bound": "alu", "achieved": round(tflops, 4), "peak": round(FP64_PEAK_TFLOPS, 4),
                           "unit": "TFLOP/s", "frac": round(tflops / FP64_PEAK_TFLOPS, 4)}),
                         kernel="k_batched", hbm_gbs=round(gbs, 1), hbm_frac=round(gbs / hbm_peak, 4),
                         fp64_tflops=round(tflops, 4), fp64_frac=round(tflops / FP64_PEAK_TFLOPS, 4),
                         traffic=None if t_step is None else int(t_step * steps),
                         traffic_key=tkey, note="graph time includes the batch's setup launch"),
        "wall_ms": round(wall * 1e3, 2), "clocks": clk.summary(),
        "gpu_launches_detail": "graph: k_exp_setup_batch + k_batched (plus two memsets)"}


def run_batch512(args):
    import torch

    import magnus_inputs as mi
    import paper_1709_06483_gb300 as mg

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    mg.load()
    cfg = tuple(int(x) for x in args.batch_config.split("x")) if args.batch_config else None
    r = batch_workload(mg, mi, local, steps=args.steps, storage=args.storage, fixed=bool(args.fixed_sums),
                       variant=args.variant, warmup=args.warmup, sample_every=16, config=cfg)
    line = {
        "metric": METRIC, "value": r["steps_per_s"], "unit": r["unit"], "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+i64" if r["fixed_sums"] else "f64", "data": "synthetic",
        "config": {"workload": f"batch_512_xxz_chains_8to14spins_{args.storage}_{args.variant.lower()}",
                   "chains": r["chains"], "rows": r["rows"], "nnz": r["nnz"], "h": 0.01, "variant": args.variant,
                   "cta_size": r["cta_size"], "cluster_size": r["cluster_size"],
                   "sums": SUMS_FIXED if r["fixed_sums"] else "FP64"},
        "gpu_launches": 2, **{k: v for k, v in r.items() if k not in ("workload", "unit", "steps")},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- adjoint workload
def adjoint_workload(mg, mi, local, nsteps=1000, fd_coefs=(0, 31)):
    """Optimal-control gradient: 16-spin chain (matrix-free), f(t) = sum_{k=1}^{32} c_k sin(k pi t / T),
    T = 10, nsteps Cf4 steps of 0.01, F = |<phi|psi(T)>|^2, dF/dc by the adjoint with checkpoints every
    16 steps; timed against one forward propagation, and checked against central differences of F
    for the coefficients fd_coefs."""
    import torch
    c = mi.workload5()
    n, om, ck = c.nspins, c.drive_om, c.drive_as

    def plan_for(coefs):
        return mg.Plan(c.dim, [mg.XXZTerm(n, c.J, c.hz, c.delta), mg.FieldXTerm(n)],
                       [mg.Drive.const(), mg.Drive(0.0, np.zeros(om.size), coefs, om)])

    plan = plan_for(ck)
    psi0, phi = torch.from_numpy(c.psi0).cuda(), torch.from_numpy(c.phi).cuda()
    plan.adjoint_grad(psi0, phi, 0.0, c.h, min(nsteps, 32), "CF4", kd=1, ckpt_every=16)  # warm-up
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t = time.perf_counter()
        F, grad, st = plan.adjoint_grad(psi0, phi, 0.0, c.h, nsteps, "CF4", kd=1, ckpt_every=16)
        t_grad = time.perf_counter() - t
    psi = psi0.clone()
    torch.cuda.synchronize()
    t = time.perf_counter()
    plan.propagate(psi, 0.0, c.h, nsteps, "CF4")
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t
    plan.close()

    def fid(coefs):
        q = plan_for(coefs)
        x = psi0.clone()
        q.propagate(x, 0.0, c.h, nsteps, "CF4")
        q.close()
        return abs(torch.vdot(phi, x).item()) ** 2

    errs = []
    for k in fd_coefs:
        up, dn = ck.copy(), ck.copy()
        up[k] += 1e-5
        dn[k] -= 1e-5
        fd = (fid(up) - fid(dn)) / 2e-5
        errs.append(abs(grad[1 + om.size + k] - fd))
    return {
        "workload": f"16-spin chain (matrix-free), 32 sine modes, T = 10, {nsteps} Cf4 steps of 0.01, checkpoints "
                    "every 16 steps, gradient of |<phi|psi(T)>|^2 by the adjoint",
        "steps_per_s": round(nsteps / t_grad, 2), "unit": "adjoint steps/s (forward + gradient)", "steps": nsteps,
        "ms_per_step": round(t_grad * 1e3 / nsteps, 4), "F": F, "gradient_time_s": round(t_grad, 4),
        "forward_time_s": round(t_fwd, 4), "gradient_over_forward": round(t_grad / t_fwd, 3),
        "max_abs_err_vs_central_differences": max(errs), "fd_coefficients": list(fd_coefs),
        # the plain alternative: central differences need 2 forward propagations per parameter
        "speedup_vs_central_differences": round(2 * grad.size * t_fwd / t_grad, 2), "parameters": int(grad.size),
        "clocks": clk.summary(),
        "gpu_launches_detail": "about 4 per exponential (recompute, augmented Leja, dot, costate)"}


def run_adjoint16(args):
    import torch

    import magnus_inputs as mi
    import paper_1709_06483_gb300 as mg

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    mg.load()
    nsteps = args.steps if args.steps != 100 else 1000
    r = adjoint_workload(mg, mi, local, nsteps=nsteps)
    line = {
        "metric": METRIC, "value": r["steps_per_s"], "unit": r["unit"], "n_gpus": world, "steps": nsteps,
        "warmup": 1, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "adjoint_xxz_16spins_32modes_cf4", "spins": 16, "modes": 32, "T": 10.0, "h": 0.01,
                   "checkpoint_every": 16},
        "gpu_launches": "about 4 per exponential", **{k: v for k, v in r.items() if k not in ("workload", "unit", "steps")},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- the matvec alone
def run_spmv20(args):
    """The generator matvec in isolation (magnus_apply): y = (H_s + H_d) x on the 20-spin chain,
    one state; --steps applications timed with CUDA events after --warmup.

    FP64 arithmetic (--fixed-sums 0), algorithmic bytes per application: CSR 12 B per stored entry
    (8 B real value -- a plan keeps complex-stored real values as a float64 copy -- + 4 B column)
    + 2 x 8 B row pointers per row + 16 B read of x (each element once) + 16 B write of y per row;
    matrix-free 32 B per row.  Bound by the FP64 pipe: FMA-equivalent flops as in the Leja
    iteration, without the shift, update and norms.

    Fixed point (default): 12 B per H_s entry (62-bit value mantissa + column), 4 B per entry of the
    pattern term sum_i sx_i (column only), 8 B of row pointer and 2 B of row exponent per row, and
    80 B per row of vectors: x read twice (max |x|, then the copy Z = trunc(x 2^s)), Z written and
    read once, y written.  About 6 FP64 instructions per row remain (the weighted conversions back
    to FP64), so the bound is HBM."""
    import torch

    import magnus_inputs as mi
    import paper_1709_06483_gb300 as mg

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    mg.load()
    c = mi.workload2()
    terms = workload_terms(mg, c, args.storage)
    fixed = bool(args.fixed_sums)
    plan = mg.Plan(c.dim, terms, drives(mg, c), fixed_sums=fixed)
    x = torch.from_numpy(c.psi0).cuda()
    y = torch.empty_like(x)
    beta = np.array([1.0, 1.0])
    for _ in range(max(args.warmup, 3)):
        plan.apply(beta, x, y)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            plan.apply(beta, x, y)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    D, n = c.dim, c.nspins
    if args.storage.startswith("csr"):
        nnz_s, nnz_d = (t.col.numel() for t in terms)
        if fixed:
            nbytes = 12 * nnz_s + 4 * nnz_d + 8 * (D + 1) + 2 * D + 80 * D
            inst = 6 * D
        else:
            nbytes = 12 * (nnz_s + nnz_d) + 2 * 8 * (D + 1) + 32 * D  # real values: the plan's float64 copy
            inst = 2 * (nnz_s + nnz_d) + 4 * D
    else:
        nbytes = 80 * D if fixed else 32 * D
        inst = D * 8 if fixed else D * (4 + (n - 1) + 2 * n + 2)
    gbs = nbytes / (ms / 1e3) / 1e9
    tflops = 2 * inst / (ms / 1e3) / 1e12
    peaks = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", HBM_PEAK_FALLBACK))
    if fixed:  # the FP64 pipe holds only the conversions back: HBM bytes are the bound
        roof = {"bound": "hbm", "achieved": round(gbs, 1), "peak": round(hbm_peak, 1), "unit": "GB/s",
                "frac": round(gbs / hbm_peak, 4), "fp64_tflops": round(tflops, 4),
                "fp64_frac": round(tflops / FP64_PEAK_TFLOPS, 4)}
    else:
        roof = {"bound": "alu", "achieved": round(tflops, 4), "peak": round(FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s",
                "frac": round(tflops / FP64_PEAK_TFLOPS, 4), "hbm_gbs": round(gbs, 1),
                "hbm_frac": round(gbs / hbm_peak, 4)}
    roof.update({"kernel": "k_apply", "traffic": None, "algorithmic_bytes": nbytes})
    line = {
        "metric": METRIC, "value": round(gbs, 1), "unit": "GB/s (generator matvec alone)", "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": round(ms, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+i64" if fixed else "f64", "data": "synthetic",
        "config": {"workload": f"matvec_xxz_chain_20spins_{args.storage}", "spins": n, "dim": D, "states": 1,
                   "sums": SUMS_FIXED if fixed else "FP64",
                   "l2": "inputs larger than L2" if args.storage.startswith("csr") else "matrix-free, L2-resident"},
        "roofline": roof,
        "gpu_launches": args.steps * (3 if fixed else 1), "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- oracle arm
def oracle_problem(c, interval="gershgorin"):
    import oracle
    Hs = oracle.xxz_csr(c.nspins, c.J, c.hz, c.delta)
    Hd = oracle.field_x_csr(c.nspins)
    f = oracle.Coeff(c.drive_a0, c.drive_ac, c.drive_as, c.drive_om)
    return oracle.Problem([Hs, Hd], [oracle.Coeff.const(), f], interval=interval)


def _oracle_timing(steps, variant, interval, threaded, workload="xxz20", count=1):
    """Run oracle/cpu_timing.py in a process of its own (no CUDA context) and return its record."""
    env = dict(os.environ)
    if threaded:
        env["OMP_NUM_THREADS"] = str(os.cpu_count() or 1)
    cmd = [sys.executable, "-m", "oracle.cpu_timing", "--steps", str(steps), "--variant", variant,
           "--interval", interval, "--workload", workload, "--count", str(count)] + (["--threaded"] if threaded else [])
    out = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-500:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def cpu_baseline(variant, nsteps, interval="gershgorin"):
    """The FP64 CPU oracle as it stands (plain C) on the first nsteps steps of the 20-spin chain, timed
    on the host cores: the single-threaded checker (the line's value) and the OpenMP build of the
    same source on every core (its element-wise loops spread over threads, identical bits), the
    analogue of the paper's multi-core CPU runs."""
    one = _oracle_timing(nsteps, variant, interval, False)
    rec = {"value": round(one["steps"] / one["seconds"], 4), "unit": "steps/s", "cores": 1, "kind": "oracle",
           "sample": f"first {nsteps} of the 200 {variant} steps of the 20-spin chain (full state, full matrix), "
                     f"{interval} enclosures, single-threaded",
           "host": one["host"], "nproc": one["nproc"]}
    try:
        allc = _oracle_timing(nsteps, variant, interval, True)
        rec["all_cores"] = {"value": round(allc["steps"] / allc["seconds"], 4), "unit": "steps/s",
                            "cores": allc["threads"], "kind": "oracle (OpenMP build of the same source)",
                            "sample": f"the same {nsteps} steps on {allc['threads']} threads"}
    except Exception as exc:  # noqa: BLE001 - e.g. no OpenMP runtime on the host
        rec["all_cores"] = {"unavailable": repr(exc)[:200]}
    return rec


def workload_cpu_baselines():
    """The FP64 CPU oracle on a bounded sample of each of the other workloads (a few seconds each),
    single-threaded and on every core, in the unit of the workload's GPU rate: the 10-spin chain
    whole (100 Cf4 steps); the dense chain one state for one step (scaled to 64 states); the batch
    the first 32 chains for 10 steps (scaled by rows to all 512); the adjoint the first 20 of its
    1000 steps (forward and gradient)."""
    specs = {
        "cfg1_xxz10_csr_cf4": ("xxz10", 100, 1, "steps/s",
                               lambda r: r["steps"] / r["seconds"], "all 100 CF4 steps of the 10-spin chain"),
        "cfg3_dense13": ("dense13", 1, 1, "steps/s (64 states)",
                         lambda r: r["steps"] / (r["seconds"] * 64 / r["states"]),
                         "1 CF4 step of 1 of the 64 states, scaled to 64 states"),
        "cfg4_batch512": ("batch512", 10, 32, "steps/s (all 512 chains per step)",
                          lambda r: r["steps"] / (r["seconds"] * r["rows_all"] / r["rows"]),
                          "10 CF4 steps of the first 32 chains, scaled by rows to all 512"),
        "cfg5_adjoint16": ("adjoint16", 20, 1, "adjoint steps/s (forward + gradient)",
                           lambda r: r["steps"] / r["seconds"], "the first 20 of the 1000 CF4 steps, forward and gradient"),
    }
    out = {}
    for name, (wl, steps, count, unit, rate, sample) in specs.items():
        try:
            one = _oracle_timing(steps, "CF4", "gershgorin", False, wl, count)
            rec = {"value": round(rate(one), 6), "unit": unit, "cores": 1, "kind": "oracle", "sample": sample,
                   "seconds": round(one["seconds"], 3)}
            try:
                allc = _oracle_timing(steps, "CF4", "gershgorin", True, wl, count)
                rec["all_cores"] = {"value": round(rate(allc), 6), "unit": unit, "cores": allc["threads"],
                                    "kind": "oracle (OpenMP build of the same source)",
                                    "seconds": round(allc["seconds"], 3)}
            except Exception as exc:  # noqa: BLE001
                rec["all_cores"] = {"unavailable": repr(exc)[:200]}
            out[name] = rec
        except Exception as exc:  # noqa: BLE001 - the rest still runs
            out[name] = {"error": repr(exc)[:200]}
    return out


def run_reference(args):
    import magnus_inputs as mi
    rank, world, _ = dist_env()
    if rank != 0:
        return
    c = mi.workload2()
    P = oracle_problem(c, args.interval)
    psi = c.psi0.copy()
    if args.warmup:
        P.propagate(psi, c.t0, c.h, min(args.warmup, 1), args.variant)
    t = time.perf_counter()
    P.propagate(c.psi0, c.t0, c.h, args.steps, args.variant)
    dt = time.perf_counter() - t
    value = args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"xxz_chain_20spins_{args.storage}_{args.variant.lower()}", "spins": c.nspins,
                   "dim": c.dim, "h": c.h, "variant": args.variant, "interval": args.interval},
        "cpu_baseline": {"value": round(value, 4), "unit": "steps/s", "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} {args.variant} steps of the 20-spin chain, plain C FP64 oracle"},
        "e2e": {"value": round(value, 4), "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--variant", choices=["CF4", "M4", "CF4_3", "M2", "M6"], default="CF4")
    ap.add_argument("--storage", choices=["csr", "csr_real", "mfree"], default="csr")
    ap.add_argument("--dense-prec", default="fp64,fp32_split,tensor_sliced",
                    help="dense workload: comma list of fp64, fp32_split, tensor_sliced")
    ap.add_argument("--interval", choices=["gershgorin", "lanczos"], default="lanczos",
                    help="spectral enclosure of each term (20-spin workload)")
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--fixed-sums", type=int, choices=[0, 1], default=1,
                    help="xxz20: pattern-term sums in fixed point (1) or FP64 (0)")
    ap.add_argument("--rows", choices=["auto", "sliced", "csr", "staged"], default="auto",
                    help="layout of the fixed-point CSR rows (options.row_layout)")
    ap.add_argument("--repeats", type=int, default=5,
                    help="timed regions of --steps steps each (the value is their median)")
    ap.add_argument("--headline-only", action="store_true",
                    help="xxz20: skip the plain-FP64 comparison and the other workloads")
    ap.add_argument("--cpu-steps", type=int, default=16,
                    help="steps of the CPU oracle sample (about 12 s on one Grace core)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-config", default="", help="batch512 only: CTAxCLUSTER (e.g. 1024x1) instead of the "
                    "autotuner's choice")
    ap.add_argument("--spins", type=int, default=13, help="dense13 only: chain length (profiling smaller cases)")
    ap.add_argument("--states", type=int, default=64, help="dense13 only: states sharing H")
    ap.add_argument("--workload", choices=["xxz20", "xxz10", "dense13", "batch512", "adjoint16", "spmv20"],
                    default="xxz20", help="xxz20: the headline 20-spin chain (xxz10: the 10-spin chain in its "
                    "place); dense13: 13-spin dense chain, 64 states, FP64 vs split")
    args = ap.parse_args()
    if args.workload == "dense13" and args.impl == "ours":
        run_dense13(args)
        return
    if args.workload == "batch512" and args.impl == "ours":
        run_batch512(args)
        return
    if args.workload == "adjoint16" and args.impl == "ours":
        run_adjoint16(args)
        return
    if args.workload == "spmv20" and args.impl == "ours":
        run_spmv20(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
