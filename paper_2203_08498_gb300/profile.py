"""Per-kernel timing of one PCG iteration, outside any CUDA graph (for ncu and for users).

python -m paper_2203_08498_gb300.profile --grid 96 --mode deflation --m 16 --reps 5 [--precision fp32] [--recipe c5]
python -m paper_2203_08498_gb300.profile --grid 256 --recipe c5 --mode plain --precision fp32 --pair --reps 3

Builds the heterogeneous-diffusion matrix of the given grid, factors it, installs an
orthonormal W of m columns (random, seeded: the per-iteration cost does not depend on W's
values) and runs reps iterations with esd_profile_iterations, which launches each kernel of
the iteration body directly on the stream with CUDA events between them (FP64 kernels, or
with --precision fp32 the FP32 inner kernels of the refinement form). With --pair (plain FP32)
it runs the paired kernels of esd_solve_pair instead (esd_profile_pair_iterations) on the
source and a seeded random second right-hand side. Prints one JSON line with the average
milliseconds per kernel.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np


def main(argv=None):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch

    import paper_2203_08498_gb300 as esd
    import workloads as wl

    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, default=96)
    ap.add_argument("--mode", default="deflation", choices=["plain", "deflation", "sc"])
    ap.add_argument("--m", type=int, default=16)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--precond", default="ic0", choices=["ic0", "none"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--recipe", default="c2", choices=["c2", "c5"],
                    help="c2: 16 balls of 1e5 (radius 4-8 cells at 128^3); c5: 64 balls of 1e6 (8-16 at 256^3)")
    ap.add_argument("--pair", action="store_true", help="the paired kernels of two systems (plain FP32)")
    a = ap.parse_args(argv)
    if a.pair and (a.mode != "plain" or a.precision != "fp32" or a.precond != "ic0"):
        ap.error("--pair runs plain FP32 PCG with IC(0)")
    if a.recipe == "c5":
        r = a.grid / 256.0
        p = wl.config_c5(N=a.grid, rmin=8 * r, rmax=16 * r)
    else:
        r = a.grid / 128.0
        p = wl.config_c2(N=a.grid, rmin=4 * r, rmax=8 * r)
    dev = torch.device("cuda:0")
    A = esd.Matrix.from_problem(p)
    pre = esd.PRECOND_IC0 if a.precond == "ic0" else esd.PRECOND_NONE
    if pre == esd.PRECOND_IC0:
        A.factor_ic0()
    prec = esd.FP64 if a.precision == "fp64" else esd.FP32_REFINE
    S = esd.Solver(A, precond=pre, maxit_cap=a.reps + 10, sample_cap=0, precision=prec)
    mode = {"plain": esd.PLAIN, "deflation": esd.DEFLATION, "sc": esd.SUBSPACE_CORRECTION}[a.mode]
    if mode != esd.PLAIN:
        W, _ = np.linalg.qr(np.random.default_rng(0).standard_normal((p.n, a.m)))
        S.set_W(np.asfortranarray(W))
    S.set_mode(mode)
    b = torch.from_numpy(p.source).to(dev)
    x = torch.zeros(p.n, dtype=torch.float64, device=dev)
    if a.pair:
        S2 = esd.Solver(A, precond=pre, maxit_cap=a.reps + 10, sample_cap=0, precision=prec)
        b2 = torch.from_numpy(wl.random_rhs(p.n, wl.SEED_BASE + 11)).to(dev)
        prof = S.profile_pair_iterations(S2, b, x, b2, torch.zeros_like(x), reps=a.reps)
    else:
        prof = S.profile_iterations(b, x, reps=a.reps)
    print(json.dumps({"grid": a.grid, "recipe": a.recipe, "n": p.n, "nnz": p.nnz, "mode": a.mode, "m": a.m,
                      "precision": a.precision, "pair": a.pair, "kernels_ms": prof}), flush=True)


if __name__ == "__main__":
    main()
