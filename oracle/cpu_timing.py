"""Time the FP64 CPU oracle on the bench's workloads -- TEST INFRASTRUCTURE, run only by bench.py's
CPU-baseline legs, in a process of its own (no CUDA context, no torch).

    python -m oracle.cpu_timing [--workload xxz20|xxz10|dense13|batch512|adjoint16] --steps S
                                [--threaded] [--variant CF4] [--interval gershgorin] [--count K]

xxz20 / xxz10: the 20-spin (10-spin) open XXZ chain of the seeded inputs, its first S Magnus steps.
dense13: the long-range chain with dense H_s and dense sum sx, the first K of its 64 states, S steps.
batch512: the first K of the 512 chains, S steps each.  adjoint16: the 16-spin chain with 32 drive
modes, F and its gradient by the adjoint over the first S of its 1000 steps.  The matrices come from
the oracle's own builders.  Prints one JSON line: the wall time, the work done (steps, and the rows
or states or chains it covered) and the threads used.  --threaded loads the OpenMP build of the same
source (element-wise loops spread over OMP_NUM_THREADS threads, identical bits); without it, the
single-threaded checker.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--threaded", action="store_true")
    ap.add_argument("--variant", default="CF4")
    ap.add_argument("--interval", default="gershgorin")
    ap.add_argument("--workload", default="xxz20", choices=["xxz20", "xxz10", "dense13", "batch512", "adjoint16"])
    ap.add_argument("--count", type=int, default=1, help="dense13: states; batch512: chains")
    args = ap.parse_args()

    import numpy as np

    import magnus_inputs as mi
    import oracle

    th = args.threaded
    rec = {"workload": args.workload, "steps": args.steps, "variant": args.variant}

    def chain_problem(c):
        Hs = oracle.xxz_csr(c.nspins, c.J, c.hz, c.delta)
        Hd = oracle.field_x_csr(c.nspins)
        f = oracle.Coeff(c.drive_a0, c.drive_ac, c.drive_as, c.drive_om)
        return oracle.Problem([Hs, Hd], [oracle.Coeff.const(), f], interval=args.interval, threaded=th)

    if args.workload in ("xxz20", "xxz10"):
        c = mi.workload2() if args.workload == "xxz20" else mi.workload1()
        P = chain_problem(c)
        t = time.perf_counter()
        P.propagate(c.psi0, c.t0, c.h, args.steps, args.variant)
        dt = time.perf_counter() - t
    elif args.workload == "dense13":
        c = mi.workload3(nvec=64, nspins=13)
        f = oracle.Coeff(c.drive_a0, c.drive_ac, c.drive_as, c.drive_om)
        P = oracle.Problem([oracle.longrange_dense(c.nspins, c.hz, 1.5, c.delta), oracle.field_x_dense(c.nspins)],
                           [oracle.Coeff.const(), f], interval=args.interval, threaded=th)
        t = time.perf_counter()
        for v in range(args.count):
            P.propagate(c.psi0[v], 0.0, c.h, args.steps, args.variant)
        dt = time.perf_counter() - t
        rec["states"] = args.count
    elif args.workload == "batch512":
        chains = mi.workload4()[: args.count]
        dt = 0.0
        for c in chains:
            P = chain_problem(c)  # plan-time work (Gershgorin) outside the timed region
            t = time.perf_counter()
            P.propagate(c.psi0, 0.0, c.h, args.steps, args.variant)
            dt += time.perf_counter() - t
        rec["chains"] = len(chains)
        rec["rows"] = int(sum(c.dim for c in chains))
        rec["rows_all"] = int(sum(c.dim for c in mi.workload4()))
    else:  # adjoint16
        c = mi.workload5()
        Hs = oracle.xxz_csr(c.nspins, c.J, c.hz, c.delta)
        Hd = oracle.field_x_csr(c.nspins)
        f = oracle.Coeff(0.0, np.zeros(c.drive_om.size), c.drive_as, c.drive_om)
        P = oracle.Problem([Hs, Hd], [oracle.Coeff.const(), f], interval=args.interval, threaded=th)
        t = time.perf_counter()
        P.adjoint_grad(c.psi0, c.phi, 0.0, c.h, args.steps, "CF4", kd=1)
        dt = time.perf_counter() - t
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)) if th else 1
    rec.update({"seconds": dt, "threads": threads, "host": os.uname().machine, "nproc": os.cpu_count()})
    print(json.dumps(rec), flush=True)


if __name__ == "__main__":
    main()
