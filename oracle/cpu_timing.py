"""Time the FP64 CPU oracle on the 20-spin chain -- TEST INFRASTRUCTURE, run only by bench.py's
CPU-baseline leg, in a process of its own (no CUDA context, no torch).

    python -m oracle.cpu_timing --steps S [--threaded] [--variant CF4] [--interval gershgorin]

Builds the 20-spin open XXZ chain of the seeded inputs (CSR terms from the oracle's own builders),
propagates its first S Magnus steps and prints one JSON line: the wall time, the steps and the
threads used.  --threaded loads the OpenMP build of the same source (element-wise loops spread over
OMP_NUM_THREADS threads, identical bits); without it, the single-threaded checker.
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
    args = ap.parse_args()

    import magnus_inputs as mi
    import oracle

    c = mi.workload2()
    Hs = oracle.xxz_csr(c.nspins, c.J, c.hz, c.delta)
    Hd = oracle.field_x_csr(c.nspins)
    f = oracle.Coeff(c.drive_a0, c.drive_ac, c.drive_as, c.drive_om)
    P = oracle.Problem([Hs, Hd], [oracle.Coeff.const(), f], interval=args.interval, threaded=args.threaded)
    t = time.perf_counter()
    P.propagate(c.psi0, c.t0, c.h, args.steps, args.variant)
    dt = time.perf_counter() - t
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)) if args.threaded else 1
    print(json.dumps({"seconds": dt, "steps": args.steps, "threads": threads, "variant": args.variant,
                      "host": os.uname().machine, "nproc": os.cpu_count()}), flush=True)


if __name__ == "__main__":
    main()
