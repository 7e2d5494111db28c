"""Write the oracle's iteration counts for the benchmark sequences (CPU oracle only).

The counts let the benchmark's CPU legs extrapolate per-iteration oracle timings to solves
per second, with the oracle's own number of iterations per solve.

    python -m oracle.sequence_counts [deflation|sc|plain] [systems]         # 128^3, 20 systems
    python -m oracle.sequence_counts --c5 [deflation|sc|plain] [systems]    # 256^3, forward + adjoint

The 128^3 sequence takes about 15 minutes on one core per mode. The 256^3 one (1e6
inclusions, W from m = 32 samples of system 1, every forward solve followed by its adjoint
A lambda = 2 (x_t - x_target) warm-started from the previous lambda) runs the OpenMP build of
the oracle, whose results are those of the serial build, for the first few systems (about
half an hour for two systems on 8 cores).
"""
import json
import os
import sys
import time

import numpy as np

import oracle
import workloads as wl

MODES = {"plain": oracle.PLAIN, "deflation": oracle.DEFLATION, "sc": oracle.SUBSPACE_CORRECTION}
DATA = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")


def c2_counts(mode, systems):
    p = wl.config_c2()
    t0 = time.perf_counter()
    res, aux = oracle.run_sequence(p, systems, MODES[mode], 16, tol=1e-8)
    out = {"workload": "fv7_128cube_16balls_1e5_dt1e-3", "mode": mode, "m": 16, "tol": 1e-8,
           "iterations": [r["iters"] for r in res], "relres": [r["relres"] for r in res],
           "seconds": time.perf_counter() - t0}
    return out, os.path.join(DATA, f"fv7_128cube_{mode}_counts.json")


def c5_counts(mode, systems, m=32, tol=1e-8):
    """The 256^3 sequence with adjoints: system 1 plain (m samples when W is used), W = Q of the
    sampled errors (theta = inf), then systems 2.. in the mode; after every forward solve the
    adjoint solve of the same matrix and mode. x_target as in the benchmark."""
    p = wl.config_c5()
    xt = np.random.default_rng(20220316 + 7).standard_normal(p.n) * float(np.abs(p.source).max()) * 1e-3
    with oracle.using(oracle.openmp_lib()):
        ic = oracle.IC0(p)
        x = np.zeros(p.n)
        lam = np.zeros(p.n)
        aux = None
        fwd, adj, rel_f, rel_a = [], [], [], []
        t0 = time.perf_counter()
        for t in range(systems):
            b = x / p.dt + p.source
            if t == 0 or mode == "plain":
                sm = m if (t == 0 and mode != "plain") else 0
                o = oracle.System(p, ic).solve(b, x, tol=tol, sample_m=sm, history=False)
                if t == 0 and mode != "plain":
                    aux, info = oracle.build_w(p, o["x"], o["samples"], o["sample_iter"])
            else:
                o = oracle.System(p, ic, MODES[mode], aux).solve(b, x, tol=tol, history=False)
            x = o["x"]
            fwd.append(o["iters"])
            rel_f.append(o["relres"])
            g = 2.0 * x - 2.0 * xt
            sys_a = oracle.System(p, ic) if (t == 0 or mode == "plain") else oracle.System(p, ic, MODES[mode], aux)
            oa = sys_a.solve(g, lam, tol=tol, history=False)
            lam = oa["x"]
            adj.append(oa["iters"])
            rel_a.append(oa["relres"])
            print(json.dumps({"system": t + 1, "forward": fwd[-1], "adjoint": adj[-1],
                              "seconds": time.perf_counter() - t0}), flush=True)
    out = {"workload": "fv7_256cube_64balls_1e6_dt1e-3", "mode": mode, "m": m, "tol": tol,
           "iterations": fwd, "adjoint_iterations": adj, "relres": rel_f, "adjoint_relres": rel_a,
           "seconds": time.perf_counter() - t0, "threads": int(oracle.openmp_lib().orc_threads())}
    return out, os.path.join(DATA, f"fv7_256cube_{mode}_counts.json")


def main():
    args = sys.argv[1:]
    c5 = "--c5" in args
    args = [a for a in args if a != "--c5"]
    mode = args[0] if args else "deflation"
    if c5:
        out, path = c5_counts(mode, int(args[1]) if len(args) > 1 else 2)
    else:
        out, path = c2_counts(mode, int(args[1]) if len(args) > 1 else 20)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
