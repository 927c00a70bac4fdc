"""Benchmark: Magnus steps/s and Leja matvec GB/s of the plain FP64 GPU path.

Workload (one Magnus step = one bench step): the open XXZ chain with 20 spins
(dim 2^20, 31,981,568 stored entries as complex128 CSR), J_i ~ U[0.5,1.5],
h_i ~ U[-1,1], drive cos(5t) on sum_i sigma^x_i, step h = 0.005 from t = 0, Leja
tolerance 1e-10 (rel + abs), method Cf4.  Synthetic inputs from magnus_inputs
(seeded).  The CSR matrix (640 MB) is larger than L2, so every Leja iteration
streams it from HBM.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: one process per GPU under torchrun; every rank propagates its own
replica (the path has no exchange step), value = all ranks' steps / max time.
--impl reference times the FP64 CPU oracle (plain C, one host core) on the same
workload, rank 0 only.
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
    if storage in ("csr", "csr_real"):
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
PERSISTENT_SOURCES = ("leja_persistent.cu", "rows.cuh", "persist_common.cuh", "magnus_internal.cuh", "magnus_api.cu")
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
    c = mi.workload2()
    variant, storage = args.variant, args.storage
    stream = torch.cuda.current_stream()
    terms = workload_terms(mg, c, storage)
    nnz_terms = tuple(t.col.numel() for t in terms) if storage.startswith("csr") else (0, 0)
    nnz_total = sum(nnz_terms) if storage.startswith("csr") else None
    plan = mg.Plan(c.dim, terms, drives(mg, c), interval=args.interval, fixed_sums=bool(args.fixed_sums))
    psi0 = torch.from_numpy(c.psi0).cuda()
    psi = psi0.clone()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # warm-up: W steps
    if args.warmup:
        plan.propagate(psi, 0.0, c.h, args.warmup, variant)
    psi.copy_(psi0)
    barrier()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        start.record(stream)
        st = plan.propagate(psi, c.t0, c.h, args.steps, variant)
        end.record(stream)
        barrier()
    ms = max_over_ranks(start.elapsed_time(end), "cuda")
    value = replica_rate(args.steps, ms, world)

    # roofline of the persistent Leja kernel, from its own CUDA-event duration
    nmv = st["n_matvec"]
    fixed = bool(st["fixed_sums"])
    bytes_it, flops_it = algorithmic_per_iteration(c, storage, variant, nnz_terms, fixed, st["n_substeps"] / nmv)
    kms = st["kernel_ms"]
    gbs = bytes_it * nmv / (kms / 1e3) / 1e9
    tflops = flops_it * nmv / (kms / 1e3) / 1e12
    peaks = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", HBM_PEAK_FALLBACK))
    t_hbm, t_alu = bytes_it / (hbm_peak * 1e9), flops_it / (FP64_PEAK_TFLOPS * 1e12)
    key = f"wl2_{storage}_{variant}" + ("_fixed" if fixed else "")
    traffic_it = profiled_traffic(key)
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

    # end-to-end through the public API with host buffers: every step copies its input state from
    # pinned host memory, runs one Magnus step (magnus_propagate, which returns when the step is
    # done) and copies the result back to pinned host memory.  Two device state buffers: the next
    # step's input copy and the previous step's result copy run on a copy stream while the current
    # step computes.
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
    e2e_ms = e0.elapsed_time(e1)
    e2e = {"value": round(world * e2e_steps / (e2e_ms / 1e3), 3), "unit": "steps/s",
           "h2d_bytes_per_step": host_in.numel() * 16, "d2h_bytes_per_step": host_out[0].numel() * 16,
           "steps": e2e_steps, "copies": "double-buffered: next input H2D and previous result D2H on a copy "
           "stream during the current step"}

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+i64" if fixed else "f64", "data": "synthetic",
        "config": {"workload": f"xxz_chain_20spins_{storage}_{variant.lower()}", "spins": c.nspins, "dim": c.dim,
                   "nnz": nnz_total, "h": c.h, "t0": c.t0, "variant": variant, "storage": storage,
                   "interval": args.interval,
                   "sums": SUMS_FIXED if fixed else "FP64",
                   "leja_tol": 1e-10, "l2": "inputs larger than L2: the 640 MB CSR is streamed every iteration"
                   if storage.startswith("csr") else "matrix-free; 4 state vectors of 16 MB stay L2-resident",
                   "parallelism": f"replicas x{world}"},
        "matvec_gbs": round(gbs, 1),
        "leja": {"iterations": nmv, "max_degree": st["max_m"], "exponentials": st["n_exp"]},
        "roofline": roof,
        "e2e": e2e,
        "gpu_launches": 2,
        "gpu_launches_detail": "timed region: k_exp_setup + k_magnus_persistent (one persistent launch per call)",
        "clocks": clk.summary(),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(c, variant, args.cpu_steps, args.interval)
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        torch.distributed.destroy_process_group()


# --------------------------------------------------------------------------- dense workload
def run_dense13(args):
    """13-spin long-range chain, dense H_s and dense sum sx (dim 8192, 2 x 1.07 GB complex128), 64
    states, Cf4, h = 0.01: the plain FP64 path, the FP32-split path and the tensor-core sliced path
    on the same states; each reduced-precision path's state error against the FP64 GPU result is
    stated.  The line's value is the sliced path's rate."""
    import torch

    import magnus_inputs as mi
    import paper_1709_06483_gb300 as mg

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    mg.load()
    c = mi.workload3(nvec=args.states, nspins=args.spins)
    Hs = mg.build_longrange_dense(c.nspins, c.hz, 1.5, c.delta)
    Hd = mg.build_field_x_dense(c.nspins)
    stream = torch.cuda.current_stream()
    res = {}
    modes = {"fp64": mg.FP64, "fp32_split": mg.FP32_SPLIT, "tensor_sliced": mg.TENSOR_SLICED}
    wanted = [m for m in args.dense_prec.split(",") if m]
    for prec, mode in modes.items():
        if prec not in wanted:
            continue
        plan = mg.Plan(c.dim, [mg.DenseTerm(Hs), mg.DenseTerm(Hd)], drives(mg, c), nvec=args.states,
                       precision=mode)
        psi0 = torch.from_numpy(c.psi0).cuda()
        psi = psi0.clone()
        if args.warmup:
            plan.propagate(psi, 0.0, c.h, 1, args.variant)
        psi.copy_(psi0)
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            s0.record(stream)
            st = plan.propagate(psi, 0.0, c.h, args.steps, args.variant)
            s1.record(stream)
            torch.cuda.synchronize()
        ms = s0.elapsed_time(s1)
        res[prec] = {"ms": ms, "st": st, "psi": psi.clone(), "clk": clk.summary()}
        plan.close()
    D, nv = c.dim, args.states
    out = {}
    for prec, r in res.items():
        nmv = r["st"]["n_matvec"] / nv  # Leja iterations (all vectors advance together)
        # per Leja iteration: each dense term read once (16 B/element) + 64 vectors x 64 B/row;
        # FP64 work: 2 FMAs per H element per vector per term (real H x complex state)
        bytes_it = 2 * 16 * D * D + nv * 64 * D
        fma_it = 2 * 2 * D * D * nv
        kms = r["st"]["kernel_ms"]
        out[prec] = {"steps_per_s": round(args.steps / (r["ms"] / 1e3), 4), "ms_per_step": round(r["ms"] / args.steps, 3),
                     "leja_iterations": nmv, "kernel_ms": round(kms, 3),
                     "matvec_gbs": round(bytes_it * nmv / (kms / 1e3) / 1e9, 2),
                     "fp64_equiv_tflops": round(2 * fma_it * nmv / (kms / 1e3) / 1e12, 4), "clocks": r["clk"]}
        if prec == "tensor_sliced":
            # issued bf16 MMA work (tcgen05, Cf4): 10 digit pairs x 2 flops x D^2 x 128 columns per dense term
            out[prec]["bf16_tflops_issued"] = round(10 * 2 * D * D * 128 * 2 * nmv / (kms / 1e3) / 1e12, 2)
    errs = {}
    if "fp64" in res:
        a = res["fp64"]["psi"].cpu().numpy()
        for prec in ("fp32_split", "tensor_sliced"):
            if prec in res:
                b = res[prec]["psi"].cpu().numpy()
                errs[prec] = float(np.max(np.linalg.norm(a - b, axis=1) / np.linalg.norm(a, axis=1)))
    f64 = out.get("fp64")
    best = out.get("tensor_sliced") or out.get("fp32_split") or f64
    peaks = measured_peaks()
    bf16_peak = float(peaks.get("bf16_tflops", 1900.0))
    if "tensor_sliced" in out:
        # the dominant kernel of the timed path: k_dense_persistent<..., 3>, its tensor-core work
        ts = out["tensor_sliced"]
        # DRAM bytes per Leja iteration from the 12-spin capture (dim 4096), scaled by (dim / 4096)^2:
        # the traffic is the digits of the dense terms, read once per iteration
        t12 = profiled_traffic("dense_tc_12spins_64states", DENSE_TC_SOURCES)
        roof = {"bound": "tensor", "kernel": "k_dense_persistent (tcgen05 digit products)",
                "achieved": ts["bf16_tflops_issued"], "peak": bf16_peak, "unit": "TFLOP/s",
                "frac": round(ts["bf16_tflops_issued"] / bf16_peak, 4),
                "traffic": None if t12 is None or nv != 64 else int(t12 * (D / 4096) ** 2),
                "traffic_unit": "DRAM bytes per Leja iteration (12-spin ncu capture scaled by (dim/4096)^2)",
                "peak_source": ("MEASURED_PEAKS.json bf16_tflops (burst), of measured" if "bf16_tflops" in peaks
                                else "1900 TFLOP/s bf16 burst, of fallback (no MEASURED_PEAKS.json)"),
                "work": "10 bf16 digit-pair products x 2 flops x dim^2 x 128 columns per dense term per Leja iteration"}
    else:
        roof = {"bound": "alu", "kernel": "k_dense_persistent (FP64 path)",
                "achieved": f64["fp64_equiv_tflops"], "peak": round(FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s",
                "frac": round(f64["fp64_equiv_tflops"] / FP64_PEAK_TFLOPS, 4), "traffic": None}
    line = {
        "metric": METRIC, "value": best["steps_per_s"], "unit": "steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": best["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16-digits(f64-equivalent)" if "tensor_sliced" in out else "f64",
        "data": "synthetic",
        "config": {"workload": f"longrange_chain_{c.nspins}spins_dense_{nv}states_cf4", "spins": c.nspins, "dim": D,
                   "states": nv, "h": c.h, "variant": args.variant,
                   "l2": f"inputs larger than L2: 2 x {16 * D * D / 1e9:.2f} GB dense terms"},
        "paths": out,
        "speedup_vs_fp64": {k: round(out[k]["steps_per_s"] / f64["steps_per_s"], 3) for k in errs} if f64 else None,
        "state_error_vs_fp64": errs,
        "roofline": roof,
        "gpu_launches": 2,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- batched workload
def run_batch512(args):
    """512 independent XXZ chains of 8-14 spins (dims 256..16384, CSR terms), per-chain drive
    A cos(w t), Cf4, h = 0.01, one persistent launch under a replayed CUDA graph.  A step advances
    every chain by one Magnus step."""
    import torch

    import magnus_inputs as mi
    import paper_1709_06483_gb300 as mg

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    mg.load()
    chains = mi.workload4()
    probs = []
    nnz_s = nnz_c = 0  # stored entries of H_s and of sum_i sx_i over all chains
    for c in chains:
        terms = workload_terms(mg, c, args.storage)
        if args.storage.startswith("csr"):
            nnz_s += terms[0].col.numel()
            nnz_c += terms[1].col.numel()
        probs.append((c.dim, terms, drives(mg, c)))
    nnz = nnz_s + nnz_c
    B = mg.Batch(probs, fixed_sums=bool(args.fixed_sums))
    psi0 = [torch.from_numpy(c.psi0).cuda() for c in chains]
    psis = [p.clone() for p in psi0]
    B.propagate(psis, 0.0, 0.01, args.warmup or 1, args.variant)  # autotune + warm-up
    for p, q in zip(psis, psi0):
        p.copy_(q)
    B.propagate(psis, 0.0, 0.01, args.steps, args.variant)         # captures the graph for these steps
    for p, q in zip(psis, psi0):
        p.copy_(q)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    with ClockSampler(local) as clk:
        t = time.perf_counter()
        st = B.propagate(psis, 0.0, 0.01, args.steps, args.variant)  # replay
        wall = time.perf_counter() - t
    gms = st["graph_ms"]
    rows = sum(c.dim for c in chains)
    fixed = bool(st["fixed_sums"])
    vb = 12  # real values: complex-stored ones are multiplied from the batch's float64 copy
    # as algorithmic_per_iteration: with fixed sums the field term needs its columns only and the
    # vectors add the fixed-point copies (32 B per row, and 32 B per row once per substep)
    vec = 64 * rows + ((32 + 32 * st["n_substeps"] / st["n_matvec"]) * rows if fixed else 0)
    if fixed:  # H_s mantissas + columns, its row pointers and exponents; the field's columns only
        mat = 12 * nnz_s + 4 * nnz_c + sum(8 * (c.dim + 1) + 2 * c.dim for c in chains)
    else:
        mat = vb * nnz + sum(2 * 8 * (c.dim + 1) for c in chains)
    bytes_it = mat + vec if args.storage.startswith("csr") else vec
    # Leja iterations differ per chain; algorithmic bytes weighted by each chain's iterations are
    # approximated with the mean iteration count per chain
    iters_per_chain = st["n_matvec"] / len(chains)
    gbs = bytes_it * iters_per_chain / (gms / 1e3) / 1e9
    if fixed:  # fixed-point sums and products: 14 FP64 instructions per row remain in both families
        inst_it = 14 * rows
    elif args.storage.startswith("csr"):
        inst_it = 2 * nnz + 14 * rows
    else:
        inst_it = sum(c.dim * (4 + (c.nspins - 1) + 2 * c.nspins + 2) + 10 * c.dim for c in chains)
    tflops = 2 * inst_it * iters_per_chain / (gms / 1e3) / 1e12
    peaks = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", HBM_PEAK_FALLBACK))
    # the plain FP64 GPU path for comparison: one plan and one persistent launch per chain, on a
    # sample of every 16th chain (the sizes are drawn independently, so the sample is unbiased),
    # extrapolated by the chain count
    seq_steps = min(args.steps, 20)
    sample = chains[::16]
    seq_ms = 0.0
    for c in sample:
        q = mg.Plan(c.dim, workload_terms(mg, c, args.storage), drives(mg, c), fixed_sums=bool(args.fixed_sums))
        x = torch.from_numpy(c.psi0).cuda()
        q.propagate(x, 0.0, 0.01, 1, args.variant)
        torch.cuda.synchronize()
        t = time.perf_counter()
        q.propagate(x, 0.0, 0.01, seq_steps, args.variant)
        torch.cuda.synchronize()
        seq_ms += (time.perf_counter() - t) * 1e3
        q.close()
    share = len(sample) / len(chains)
    seq_rate = seq_steps / (seq_ms / share / 1e3)
    batch_rate = args.steps / (gms / 1e3)
    line = {
        "metric": METRIC, "value": round(args.steps / (gms / 1e3), 3), "unit": "steps/s (all 512 chains per step)",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(gms / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+i64" if fixed else "f64",
        "data": "synthetic",
        "config": {"workload": f"batch_512_xxz_chains_8to14spins_{args.storage}_{args.variant.lower()}",
                   "chains": len(chains), "rows": rows, "nnz": nnz, "h": 0.01, "variant": args.variant,
                   "cta_size": st["block"], "cluster_size": st["cluster"],
                   "sums": SUMS_FIXED if fixed else "FP64"},
        "chain_steps_per_s": round(len(chains) * args.steps / (gms / 1e3), 1),
        "per_chain_plans": {"steps_per_s": round(seq_rate, 3), "how": f"one plan and launch per chain (same "
                            f"arithmetic), {len(sample)} of 512 chains x {seq_steps} steps, wall time scaled by the "
                            f"chain count (x {1 / share:.0f})"},
        "speedup_vs_per_chain_plans": round(batch_rate / seq_rate, 2),
        "leja_iterations": st["n_matvec"], "matvec_gbs": round(gbs, 1),
        # the larger of the FP64 and HBM times per iteration sets the bound, as for the single chain:
        # FMA-equivalent flops and bytes per iteration as in algorithmic_per_iteration, summed over
        # the chains
        "roofline": dict(({"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                           "frac": round(gbs / hbm_peak, 4)}
                          if gbs / hbm_peak > tflops / FP64_PEAK_TFLOPS else
                          {"bound": "alu", "achieved": round(tflops, 4), "peak": round(FP64_PEAK_TFLOPS, 4),
                           "unit": "TFLOP/s", "frac": round(tflops / FP64_PEAK_TFLOPS, 4)}),
                         kernel="k_batched", hbm_gbs=round(gbs, 1), hbm_frac=round(gbs / hbm_peak, 4),
                         fp64_tflops=round(tflops, 4), fp64_frac=round(tflops / FP64_PEAK_TFLOPS, 4),
                         traffic=None, note="graph time includes the batch's setup launch"),
        "wall_ms": round(wall * 1e3, 2), "gpu_launches": 2,
        "gpu_launches_detail": "graph: k_exp_setup_batch + k_batched (plus two memsets)", "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    B.close()


# --------------------------------------------------------------------------- adjoint workload
def run_adjoint16(args):
    """Optimal-control gradient: 16-spin chain (matrix-free), f(t) = sum_{k=1}^{32} c_k sin(k pi t / T),
    T = 10, 1000 Cf4 steps of 0.01, F = |<phi|psi(T)>|^2, dF/dc by the adjoint with checkpoints every
    16 steps; timed against one forward propagation, and checked against central differences of F for
    two coefficients."""
    import torch

    import magnus_inputs as mi
    import paper_1709_06483_gb300 as mg

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    mg.load()
    c = mi.workload5()
    n, om, ck = c.nspins, c.drive_om, c.drive_as

    def plan_for(coefs):
        return mg.Plan(c.dim, [mg.XXZTerm(n, c.J, c.hz, c.delta), mg.FieldXTerm(n)],
                       [mg.Drive.const(), mg.Drive(0.0, np.zeros(om.size), coefs, om)])

    plan = plan_for(ck)
    psi0, phi = torch.from_numpy(c.psi0).cuda(), torch.from_numpy(c.phi).cuda()
    nsteps = args.steps if args.steps != 100 else c.nsteps
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
    t_fwd = time.perf_counter() - t

    def fid(coefs):
        q = plan_for(coefs)
        x = psi0.clone()
        q.propagate(x, 0.0, c.h, nsteps, "CF4")
        q.close()
        return abs(torch.vdot(phi, x).item()) ** 2

    errs = []
    for k in (0, 31):
        up, dn = ck.copy(), ck.copy()
        up[k] += 1e-5
        dn[k] -= 1e-5
        fd = (fid(up) - fid(dn)) / 2e-5
        errs.append(abs(grad[1 + om.size + k] - fd))
    line = {
        "metric": METRIC, "value": round(nsteps / t_grad, 2), "unit": "adjoint steps/s (forward + gradient)",
        "n_gpus": world, "steps": nsteps, "warmup": 1, "ms_per_step": round(t_grad * 1e3 / nsteps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "adjoint_xxz_16spins_32modes_cf4", "spins": n, "dim": c.dim, "modes": int(om.size),
                   "T": 10.0, "h": c.h, "checkpoint_every": 16},
        "F": F, "gradient_time_s": round(t_grad, 4), "forward_time_s": round(t_fwd, 4),
        "gradient_over_forward": round(t_grad / t_fwd, 3), "max_abs_err_vs_central_differences": max(errs),
        # the plain FP64 GPU alternative: central differences need 2 forward propagations per parameter
        "speedup_vs_central_differences": round(2 * grad.size * t_fwd / t_grad, 2),
        "parameters": int(grad.size),
        "gpu_launches": "about 4 per exponential (recompute, augmented Leja, dot, costate)", "clocks": clk.summary(),
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


def cpu_baseline(c, variant, nsteps, interval="gershgorin"):
    """The FP64 CPU oracle as it stands (plain C, single thread) on the first nsteps steps."""
    P = oracle_problem(c, interval)
    t = time.perf_counter()
    P.propagate(c.psi0, c.t0, c.h, nsteps, variant)
    dt = time.perf_counter() - t
    return {"value": round(nsteps / dt, 4), "unit": "steps/s", "cores": 1, "kind": "oracle",
            "sample": f"first {nsteps} of the 200 {variant} steps of the 20-spin chain (full state, full matrix)",
            "host": os.uname().machine, "nproc": os.cpu_count()}


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
    ap.add_argument("--cpu-steps", type=int, default=16,
                    help="steps of the CPU oracle sample (about 12 s on one Grace core)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--spins", type=int, default=13, help="dense13 only: chain length (profiling smaller cases)")
    ap.add_argument("--states", type=int, default=64, help="dense13 only: states sharing H")
    ap.add_argument("--workload", choices=["xxz20", "dense13", "batch512", "adjoint16", "spmv20"], default="xxz20",
                    help="xxz20: the headline 20-spin chain; dense13: 13-spin dense chain, 64 states, FP64 vs split")
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
