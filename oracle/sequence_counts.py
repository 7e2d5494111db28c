"""Write the oracle's iteration counts for the benchmark sequence (128^3, 20 systems).

Runs only the CPU oracle (about 15 minutes on one core per mode). The counts let the
benchmark's CPU legs extrapolate per-iteration oracle timings to solves per second.
Usage: python -m oracle.sequence_counts [deflation|sc|plain] [systems]
"""
import json
import os
import sys
import time

import oracle
import workloads as wl

MODES = {"plain": oracle.PLAIN, "deflation": oracle.DEFLATION, "sc": oracle.SUBSPACE_CORRECTION}


def main():
    mode = sys.argv[1] if len(sys.argv) > 1 else "deflation"
    systems = int(sys.argv[2]) if len(sys.argv) > 2 else 20
    p = wl.config_c2()
    t0 = time.perf_counter()
    res, aux = oracle.run_sequence(p, systems, MODES[mode], 16, tol=1e-8)
    out = {"workload": "fv7_128cube_16balls_1e5_dt1e-3", "mode": mode, "m": 16, "tol": 1e-8,
           "iterations": [r["iters"] for r in res], "relres": [r["relres"] for r in res],
           "seconds": time.perf_counter() - t0}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", f"fv7_128cube_{mode}_counts.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
