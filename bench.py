#!/usr/bin/env python3
"""Benchmark of the hot path.

Headline (default, --config c5): 3D 7-point finite-volume diffusion on a 256^3 grid
(n = 16,777,216, nnz = 117,047,296), background coefficient 1 and 64 seeded balls of radius
8-16 cells with coefficient 1e6, Dirichlet boundaries, 8-colour ordering; a backward-Euler
sequence b_t = x_{t-1}/dt + Gaussian source (dt = 1e-3, x_0 = 0), every forward solve followed
by its adjoint A lambda = 2 (x_t - x_target); the precision form (FP32 inner IC(0)-PCG inside
FP64 iterative refinement) to a true FP64 residual of 1e-8; W from m = 32 error vectors
sampled (method A) during system 1.

One step = one system of the sequence: the right-hand side on the device, the forward solve,
the adjoint right-hand side and the adjoint solve. x, lambda and W carry over from step to
step; the first warm-up step is system 1 (sampling and the W build). value = solves per
second (forward and adjoint solves, all ranks). The mode is the fastest correct one on this
workload (plain: on this 7-point operator the W terms cost more per iteration than the
iterations they save, Eq. ganma); deflation and subspace correction with the same W, and
plain FP64 PCG resumed until its true residual meets the tolerance, are timed beside it on
two more systems of the same sequence. Inputs are resident in HBM when the timed region
starts; the working set is larger than L2, so no flush is needed between steps.

Other workloads (--config): c2 = the 128^3 sequence of 20 systems in FP64 (one step = the
whole sequence), c3 = 192^3 27-point anisotropic log-normal Q1 FE, 10 systems to 1e-10 in
the precision form with deflation m = 24, c4 = 128^3 log-normal exp(theta) diffusion, one
optimisation step through the autograd API, c1 = the 64 x 64 five-system sequence.

--impl reference times the CPU oracle (the FP64 C restatement of the method) on the same
workload: a bounded number of iterations per step, extrapolated to solves per second with
the oracle's own iteration counts.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "time-to-1e-8 per system & solves/sec; HBM GB/s vs plain FP64 PCG on GB300"
UNIT = "solves/s"
L2_BYTES = 129e6


# Per workload: grid, systems per step, sampled columns m, tolerance, mode, precision and
# whether every forward solve is followed by its adjoint solve.
CONFIGS = {
    # 64 x 64 5-point, 4 squares of 1e3, red-black: tiny, L2-resident, latency-bound
    "c1": dict(grid=64, systems=5, m=8, tol=1e-8, mode="deflation", precision="fp64", adjoint=False,
               mtilde=None, inner_tol=0.1),
    # 128^3 7-point, 16 balls of 1e5, FP64: timed in plain mode, the fastest correct FP64 mode
    # on this workload; deflation and SC (m = 16) are timed beside it on the same sequence
    "c2": dict(grid=128, systems=20, m=16, tol=1e-8, mode="plain", precision="fp64", adjoint=False,
               mtilde=None, inner_tol=0.1),
    # 192^3 27-point anisotropic log-normal FE: the precision form to 1e-10
    "c3": dict(grid=192, systems=10, m=24, tol=1e-10, mode="deflation", precision="fp32", adjoint=False,
               mtilde=None, inner_tol=0.1),
    # 128^3 log-normal exp(theta): one optimisation step = theta update + forward + adjoint
    "c4": dict(grid=128, systems=1, m=16, tol=1e-8, mode="deflation", precision="fp64", adjoint=True,
               mtilde=None, inner_tol=0.1),
    # 256^3 7-point, 64 balls of 1e6: precision form, each forward solve with its adjoint
    "c5": dict(grid=256, systems=50, m=32, tol=1e-8, mode="plain", precision="fp32", adjoint=True,
               mtilde=None, inner_tol=0.1),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="esdcg", choices=["esdcg", "reference"])
    ap.add_argument("--config", default="c5", choices=sorted(CONFIGS))
    ap.add_argument("--mode", default=None, choices=["plain", "deflation", "sc"])
    ap.add_argument("--grid", type=int, default=None)
    ap.add_argument("--systems", type=int, default=None)
    ap.add_argument("--m", type=int, default=None)
    ap.add_argument("--tol", type=float, default=None)
    ap.add_argument("--precision", default=None, choices=["fp64", "fp32"],
                    help="fp32: FP32 inner PCG inside FP64 iterative refinement")
    ap.add_argument("--mtilde", type=int, default=None,
                    help="keep the Ritz vectors of the k smallest Ritz values of the sampled W (theta filter)")
    ap.add_argument("--inner-tol", dest="inner_tol", type=float, default=None,
                    help="residual reduction of each FP32 inner solve in the refinement form")
    ap.add_argument("--no-extras", action="store_true", help="skip e2e, comparison modes and CPU baseline")
    ap.add_argument("--no-pair", dest="no_pair", action="store_true",
                    help="c5: solve each forward system and its adjoint one after the other instead of "
                         "pairing the adjoint of system t with the forward solve of system t + 1")
    a = ap.parse_args()
    for k, v in CONFIGS[a.config].items():
        if getattr(a, k, None) is None:
            setattr(a, k, v)
    return a


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


_WORKLOADS = {}


def workload(args):
    """The config's problem (C4 also returns theta and x_target); built once per process."""
    key = (args.config, args.grid)
    if key not in _WORKLOADS:
        _WORKLOADS[key] = _make_workload(args)
    return _WORKLOADS[key]


def _make_workload(args):
    import workloads as wl
    r = args.grid / {"c1": 64.0, "c2": 128.0, "c3": 192.0, "c4": 128.0, "c5": 256.0}[args.config]
    if args.config == "c1":
        return wl.config_c1()
    if args.config == "c2":
        return wl.config_c2() if args.grid == 128 else wl.config_c2(N=args.grid, rmin=4 * r, rmax=8 * r)
    if args.config == "c3":
        return wl.config_c3(N=args.grid)
    if args.config == "c5":
        return wl.config_c5(N=args.grid, rmin=8 * r, rmax=16 * r)
    return wl.config_c4(N=args.grid)


def workload_name(args, p):
    base = {
        "c1": "fv5_64x64_4squares_1e3_redblack_dt1e-2",
        "c2": f"fv7_{args.grid}cube_16balls_1e5_dt1e-3",
        "c3": f"fe27_{args.grid}cube_aniso1e-3_lognormal_s2_dt1e-3",
        "c4": f"fv7_{args.grid}cube_exp_theta_smooth4_steady",
        "c5": f"fv7_{args.grid}cube_64balls_1e6_dt1e-3",
    }[args.config]
    what = ("one optimisation step: theta update (device assembly, IC(0), AW/E refresh), forward solve "
            "and adjoint solve through the autograd API" if args.config == "c4" else
            f"{args.systems}-system backward-Euler sequence" + (", each solve followed by its adjoint"
                                                                 if args.adjoint else ""))
    prec = "FP64" if args.precision == "fp64" else "FP32 inner PCG in FP64 refinement"
    return (f"{base}: {what}, IC(0)-PCG to {args.tol:g} ({prec}), W from m={args.m} sampled error "
            f"vectors, {args.mode}")


def level_stats(p):
    """Rows and strict-lower / strict-upper entries per colour (for per-kernel bytes)."""
    A = p.scipy().tocoo()
    col_of = np.searchsorted(p.colour_ptr, np.arange(p.n), side="right") - 1
    rows = np.diff(p.colour_ptr)
    low = np.bincount(col_of[A.row[A.col < A.row]], minlength=p.ncolours)
    up = np.bincount(col_of[A.row[A.col > A.row]], minlength=p.ncolours)
    return rows, low, up


# ---------------------------------------------------------------- clocks

class Clocks:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    def __init__(self, gpu_index):
        self.proc = None
        self.lines = []
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(gpu_index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- GPU arm

def max_over_ranks(value, device):
    """The largest of every rank's value (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def launch_count(info, mode_is, m, fp32, its, outer):
    """Kernels of this library launched by solves with these inner iteration counts and
    refinement steps (from the launch sequences of the iteration and refinement graphs)."""
    nf = info["fwd_levels"] - 1
    nb = max(info["bwd_levels"] - 1, 1)
    body = 2 + nf + nb
    defl = 1 if mode_is == "deflation" else 0
    start = 1 + 2 * defl + 1 + nf + nb  # residual0, projection, update, sweeps
    end = 2 * defl + 1                   # correction, finish
    total = 0
    for k, o in zip(its, outer):
        if fp32:
            total += 2 + o * (start + end + 2)  # residual, final; per step prep, start, end, residual
        else:
            total += start + end + 1               # + true residual
        total += body * k
    return total


def pair_launch_count(info, its, outer, paired):
    """Kernels launched by one esd_solve_pair: per refinement step both systems' prep, start,
    finish and residual and the three loop conditions; one body per paired iteration and
    one per iteration that either system ran alone."""
    nf = info["fwd_levels"] - 1
    nb = max(info["bwd_levels"] - 1, 1)
    body = 2 + nf + nb
    start = 1 + 1 + nf + nb
    end = 1
    o = max(outer)
    return 5 + o * (2 * (start + end + 2) + 6) + body * (sum(its) - paired)


def gpu_arm(args):
    import torch
    import paper_2203_08498_gb300 as esd

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    if args.config == "c4":
        return c4_arm(args, esd, torch, dev, ws, rank)
    if args.config == "c5":
        return system_arm(args, esd, torch, dev, ws, rank)
    p = workload(args)
    n, nnz = p.n, p.nnz
    modes_map = {"plain": esd.PLAIN, "deflation": esd.DEFLATION, "sc": esd.SUBSPACE_CORRECTION}
    mode = modes_map[args.mode]
    fp32 = args.precision == "fp32"
    A = esd.Matrix.from_problem(p)
    A.factor_ic0()
    S = esd.Solver(A, maxit_cap=20000, sample_cap=max(args.m, 2),
                   precision=esd.FP32_REFINE if fp32 else esd.FP64)
    src = torch.from_numpy(p.source).to(dev)
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    b = torch.empty_like(x)
    inv_dt = 1.0 / p.dt
    info = A.info()
    if args.adjoint:
        # loss ||x - x_t||^2 per system: the adjoint right-hand side 2 x - 2 x_t is formed by
        # the library's rhs kernel (inv_dt = 2, s = -2 x_t)
        xt = np.random.default_rng(20220316 + 7).standard_normal(n) * float(np.abs(p.source).max()) * 1e-3
        neg2xt = torch.from_numpy(-2.0 * xt).to(dev)
        lam = torch.zeros_like(x)
        g = torch.empty_like(x)

    def sequence(md, S=S):
        A.factor_ic0()
        x.zero_()
        its, outer, adj, stats = [], [], [], {}
        for t in range(args.systems):
            S.backward_euler_rhs(x, src, inv_dt, b)
            if t == 0:
                S.set_mode(esd.PLAIN)
                st, it, rr = S.solve(b, x, args.tol, 20000, args.m if md != esd.PLAIN else 0)
                stats["cond"] = S.estimate_cond()
                if md != esd.PLAIN:
                    stats["m_kept"] = S.sample_and_build_W()
                    S.set_mode(md)
            else:
                st, it, rr = S.solve(b, x, args.tol, 20000, 0)
            if st != esd.OK:
                raise RuntimeError(f"solve {t} returned {st}")
            its.append(it)
            outer.append(S.last_solve_info()["outer_steps"])
            if args.adjoint:
                S.backward_euler_rhs(x, neg2xt, 2.0, g)
                lam.zero_()
                st, ita, rr = S.solve(g, lam, args.tol, 20000, 0)
                if st != esd.OK:
                    raise RuntimeError(f"adjoint solve {t} returned {st}")
                adj.append(ita)
                outer.append(S.last_solve_info()["outer_steps"])
        return its, stats, adj, outer

    def timed(md, steps, warm, S=S):
        for _ in range(warm):
            sequence(md, S)
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record()
        out = []
        for _ in range(steps):
            out.append(sequence(md, S))
        e1.record()
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        ms = max_over_ranks(e0.elapsed_time(e1), dev)
        return ms, wall, out

    clocks = Clocks(local)
    ms, wall, runs = timed(mode, args.steps, args.warmup)
    clk = clocks.stop()
    its, stats, adj, outer = runs[-1]
    solves_per_step = args.systems * (2 if args.adjoint else 1)
    value = solves_per_step * args.steps * ws / (ms / 1e3)
    ms_step = ms / args.steps

    launches = 0
    for it_list, st_, adj_list, outer_list in runs:
        all_its = []
        for t in range(len(it_list)):
            all_its.append(it_list[t])
            if args.adjoint:
                all_its.append(adj_list[t])
        launches += info["fwd_levels"] + 1 + (2 if fp32 else 0)  # factorisation (+ FP32 copies)
        launches += len(all_its) + (len(adj_list) if args.adjoint else 0)  # right-hand sides
        launches += launch_count(info, args.mode, args.m, fp32, all_its, outer_list)
        launches += 1  # condition estimate
        if mode != esd.PLAIN:
            launches += (1 + 8 + args.m) * (2 if fp32 else 1) + (3 if fp32 else 0)  # W build (+ FP32 pass)

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if not fp32 else "f32 inner, f64 refinement", "data": "synthetic",
        "config": {"workload": workload_name(args, p), "config": args.config, "grid": args.grid, "n": n,
                   "nnz": nnz, "systems": args.systems, "m": args.m, "mode": args.mode, "tol": args.tol,
                   "precision": args.precision, "adjoint": args.adjoint,
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "l2": "inputs larger than L2 (matrix, factor and vectors > 129 MB)"},
        "gpu_launches": launches,
        "clocks": clk,
        "iterations": its,
        "time_to_tol_ms_per_system": ms_step / solves_per_step,
        "cond_estimate_system1": {"lmin": stats["cond"][0], "lmax": stats["cond"][1],
                                  "kappa": stats["cond"][2]},
    }
    if args.adjoint:
        result["adjoint_iterations"] = adj
    if fp32:
        result["refinement_steps"] = outer
    if rank != 0 or args.no_extras:
        return result, None

    # roofline of the dominant kernel: live per-kernel CUDA-event times of the same kernels
    S.set_mode(mode)
    xs = x.clone()
    prof = S.profile_iterations(b, xs, reps=20)
    peaks = read_peaks()
    result["roofline"], result["kernel_times_ms"] = roofline(prof, p, args, mode, esd, peaks, A.layout())

    modes = None
    if args.config == "c2" and not fp32:
        # per-iteration time in each mode through the graphs (from the timed sequences)
        modes = {}
        for name, md in modes_map.items():
            if md == mode:
                its_m, ms_m = its, ms_step
            else:
                ms_m, _, r = timed(md, 1, 1)
                its_m = r[-1][0]
            modes[name] = {"iterations": its_m, "ms_per_sequence": ms_m,
                           "solves_per_s": args.systems / (ms_m / 1e3),
                           "mean_iters_2_to_T": float(np.mean(its_m[1:]))}
        result["modes"] = modes
        # the W build alone (errors of the sampled solve, CholeskyQR2, AW, E, E^-1, Ritz values):
        # solves/s with and without it
        S.set_mode(esd.PLAIN)
        xw = torch.zeros_like(x)
        S.solve(b, xw, args.tol, 20000, args.m)
        torch.cuda.synchronize()
        tw = time.perf_counter()
        S.sample_and_build_W()
        torch.cuda.synchronize()
        w_ms = (time.perf_counter() - tw) * 1e3
        S.set_mode(mode)
        result["w_build"] = {"ms": w_ms, "solves_per_s_without_w_build":
                             args.systems / ((ms_step - w_ms) / 1e3)}
        # the precision form on the same sequence: FP32 inner PCG (resumed, inner_tol 0.1) inside
        # FP64 refinement to the same tolerance, against plain FP64 PCG
        S32 = esd.Solver(A, maxit_cap=20000, sample_cap=max(args.m, 2), precision=esd.FP32_REFINE)
        fp64_plain_ms = modes["plain"]["ms_per_sequence"]
        pf = {"fp64_plain_ms_per_system": fp64_plain_ms / args.systems}
        for name, md in modes_map.items():
            ms_m, _, r = timed(md, 1, 1, S=S32)
            its_m = r[-1][0]
            pf[f"fp32_{name}"] = {"ms_per_system": ms_m / args.systems, "iterations": its_m,
                                  "speedup_vs_fp64_plain": fp64_plain_ms / ms_m}
        result["precision_form"] = pf
        # time per iteration and model bandwidth per mode (single solves of system 2)
        result["iteration"] = iteration_roofline(S, esd, p, args, x, b, src, peaks)
        # gamma of Eq. ganma: time per accelerated iteration over time per plain one, against
        # the paper's byte model (T_sciccg / T_iccg), and the sequence speedups over plain
        it_t = {k: v["ms_per_iter"] for k, v in result["iteration"].items()}
        nnz_av = p.nnz / p.n
        result["gamma"] = {"model": (116 + 16 * args.m + 24 * nnz_av) / (100 + 24 * nnz_av),
                           "measured_deflation": it_t["deflation"] / it_t["plain"],
                           "measured_sc": it_t["sc"] / it_t["plain"],
                           "sequence_speedup_vs_plain": {k: modes["plain"]["ms_per_sequence"] / modes[k]["ms_per_sequence"]
                                                         for k in ("deflation", "sc")}}
        # end to end through the C ABI with host buffers
        result["e2e"] = e2e(esd, p, args, torch)
        # the condition estimate of Algorithm PCG-con and the cost of its fused power product
        result["power_method"] = power_method_report(esd, A, p, args, b, torch, peaks)
        # sampling method A against method B (Table sampling B): W from each, deflated solves
        result["sampling_a_vs_b"] = sampling_comparison(esd, A, p, args, b, torch)
        # IC orderings: multicolour against the paper's block-Jacobi IC and natural order
        result["ic_orderings"] = ordering_comparison(esd, p, args, torch, b.device)
    elif args.config == "c1":
        # latency-bound: per-iteration time of each mode through the solve graph against the
        # sum of its kernels launched one by one
        lat = {}
        for name, md in modes_map.items():
            S.set_mode(md)
            x0 = torch.zeros_like(x)
            S.solve(b, x0, args.tol, 20000, 0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            its_sum = 0
            for _ in range(20):
                x0.zero_()
                st, it, rr = S.solve(b, x0, args.tol, 20000, 0)
                its_sum += it
            torch.cuda.synchronize()
            per_it = (time.perf_counter() - t0) / its_sum
            kern = S.profile_iterations(b, torch.zeros_like(x), reps=20)
            lat[name] = {"iters": its_sum // 20, "us_per_iteration_graph": per_it * 1e6,
                         "us_per_iteration_kernels_one_by_one": sum(t for _, t in kern) * 1e3,
                         "kernels": len(kern)}
        result["latency"] = lat
        result["e2e"] = {"value": None, "unit": UNIT, "h2d_bytes_per_step": None, "d2h_bytes_per_step": None,
                         "note": "end-to-end host-buffer timing is taken on the headline 128^3 sequence only"}
    else:
        # comparator: plain FP64 PCG on the same sequence (one timed pass)
        S64 = S if not fp32 else esd.Solver(A, maxit_cap=20000, sample_cap=max(args.m, 2))
        ms64, _, r64 = timed(esd.PLAIN, 1, 0, S=S64)
        result["fp64_plain"] = {"ms_per_step": ms64, "iterations": r64[-1][0],
                                "ms_per_solve": ms64 / solves_per_step,
                                "speedup_of_this_run": ms64 / ms_step}
        if fp32:
            # the precision form without the accelerator: FP32 inner plain PCG, FP64 refinement
            ms32, _, r32 = timed(esd.PLAIN, 1, 0, S=S)
            result["fp32_plain"] = {"ms_per_step": ms32, "iterations": r32[-1][0],
                                    "ms_per_solve": ms32 / solves_per_step,
                                    "speedup_vs_fp64_plain": ms64 / ms32}
        result["e2e"] = {"value": None, "unit": UNIT, "h2d_bytes_per_step": None, "d2h_bytes_per_step": None,
                         "note": "end-to-end host-buffer timing is taken on the headline 128^3 sequence only"}
    return result, modes


def build_w(S, args):
    """W from the sampled solve: all m columns (theta = inf), or with --mtilde k the Ritz
    vectors of the k smallest Ritz values (theta between the k-th and (k+1)-th, Eq. bk)."""
    kept = S.sample_and_build_W()
    if args.mtilde and args.mtilde < kept:
        r = np.sort(S.ritz_values())
        kept = S.sample_and_build_W(0.5 * (r[args.mtilde - 1] + r[args.mtilde]))
    return kept


def system_arm(args, esd, torch, dev, ws, rank):
    """One step = one forward solve and one adjoint solve of the backward-Euler sequence:
    b_t = x_{t-1}/dt + s on the device, the forward solve in the configured mode, and the
    adjoint A lambda = 2 (x - x_target) (warm-started from the previous lambda). Unpaired
    (--no-pair, and every mode but plain FP32): system t's forward solve, then its adjoint.
    Paired (plain FP32, the default): the adjoint of system t - 1 and the forward solve of
    system t need only x_{t-1}, so one esd_solve_pair runs both. x, lambda and W carry over
    from step to step; the first warm-up step is system 1 (the sampling solve and the W
    build; paired, its adjoint goes with system 2), so the timed steps are later systems of
    the same sequence (continuing past its 50 systems when more steps are asked for). After
    the timed steps, two more steps are solved once more, system by system in every mode and
    by plain FP64 PCG from the same right-hand sides and starts, timed per solve; the FP64
    comparator is resumed (esd_solve again from its own x) until its true residual
    ||b - A x|| / ||b|| recomputed in FP64 meets the tolerance."""
    p = workload(args)
    n = p.n
    modes_map = {"plain": esd.PLAIN, "deflation": esd.DEFLATION, "sc": esd.SUBSPACE_CORRECTION}
    mode = modes_map[args.mode]
    fp32 = args.precision == "fp32"
    A = esd.Matrix.from_problem(p)
    A.factor_ic0()
    S = esd.Solver(A, maxit_cap=20000, sample_cap=max(args.m, 2), precision=esd.FP32_REFINE if fp32 else esd.FP64,
                   inner_tol=args.inner_tol)
    paired = fp32 and mode == esd.PLAIN and not args.no_pair
    # the adjoint's solver of a pair (same matrix and factor, its own vectors and state)
    Sa = esd.Solver(A, maxit_cap=20000, sample_cap=0, precision=esd.FP32_REFINE, inner_tol=args.inner_tol) \
        if paired else None
    src = torch.from_numpy(p.source).to(dev)
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    b = torch.empty_like(x)
    xt = np.random.default_rng(20220316 + 7).standard_normal(n) * float(np.abs(p.source).max()) * 1e-3
    neg2xt = torch.from_numpy(-2.0 * xt).to(dev)
    lam = torch.zeros_like(x)
    g = torch.empty_like(x)
    inv_dt = 1.0 / p.dt
    info = A.info()
    state = {"t": 0, "kept": 0, "cond": None}
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def one_system(marks=None, save=None):
        """Forward and adjoint solve of the next system; marks: 3 events (start, after the
        forward solve, after the adjoint); save: dict receiving copies of b, x_{t-1}, g and
        lambda_{t-1} (outside any timed region)."""
        t = state["t"]
        state["t"] += 1
        if marks:
            marks[0].record()
        S.backward_euler_rhs(x, src, inv_dt, b)
        if save is not None:
            save.update(b=b.clone(), x0=x.clone())
        if t == 0:
            # system 1 samples m iterates in any mode, so that W exists for the accelerated
            # modes (this one, or the ones compared beside it)
            S.set_mode(esd.PLAIN)
            st, it, rr = S.solve(b, x, args.tol, 20000, args.m)
            state["cond"] = S.estimate_cond()
            state["kept"] = build_w(S, args)
            S.set_mode(mode)
        else:
            st, it, rr = S.solve(b, x, args.tol, 20000, 0)
        fwd = S.last_solve_info()
        if st != esd.OK:
            raise RuntimeError(f"solve of system {t + 1} returned {st}")
        if marks:
            marks[1].record()
        S.backward_euler_rhs(x, neg2xt, 2.0, g)
        if save is not None:
            save.update(g=g.clone(), lam0=lam.clone())
        st, ita, rr = S.solve(g, lam, args.tol, 20000, 0)
        adj = S.last_solve_info()
        if st != esd.OK:
            raise RuntimeError(f"adjoint solve of system {t + 1} returned {st}")
        if marks:
            marks[2].record()
        return {"system": t + 1, "iters": it, "adjoint_iters": ita, "outer": fwd["outer_steps"],
                "adjoint_outer": adj["outer_steps"], "true_relres": fwd["true_relres"],
                "adjoint_true_relres": adj["true_relres"], "restarts": fwd["restarts"] + adj["restarts"]}

    def first_forward():
        """System 1 alone (paired steps): the sampling solve and the W build."""
        state["t"] += 1
        S.backward_euler_rhs(x, src, inv_dt, b)
        S.set_mode(esd.PLAIN)
        st, it, rr = S.solve(b, x, args.tol, 20000, args.m)
        if st != esd.OK:
            raise RuntimeError(f"solve of system 1 returned {st}")
        state["cond"] = S.estimate_cond()
        state["kept"] = build_w(S, args)
        S.set_mode(mode)

    def one_pair(marks=None, save=None):
        """The forward solve of system t + 1 and the adjoint of system t, both from x_t, in one
        esd_solve_pair; marks and save as one_system's (marks[1] = marks[2]: one call)."""
        t = state["t"]
        state["t"] += 1
        if marks:
            marks[0].record()
        S.backward_euler_rhs(x, src, inv_dt, b)
        S.backward_euler_rhs(x, neg2xt, 2.0, g)
        if save is not None:
            save.update(b=b.clone(), x0=x.clone(), g=g.clone(), lam0=lam.clone())
        st, (it, _), (ita, _), npair = S.solve_pair(Sa, b, x, g, lam, args.tol, 20000)
        if st != esd.OK:
            raise RuntimeError(f"pair solve of system {t + 1} (adjoint of system {t}) returned {st}")
        if marks:
            marks[1].record()
            marks[2].record()
        fwd, adj = S.last_solve_info(), Sa.last_solve_info()
        return {"system": t + 1, "adjoint_of": t, "iters": it, "adjoint_iters": ita, "paired": npair,
                "outer": fwd["outer_steps"], "adjoint_outer": adj["outer_steps"],
                "true_relres": fwd["true_relres"], "adjoint_true_relres": adj["true_relres"],
                "restarts": fwd["restarts"] + adj["restarts"]}

    def step(marks=None, save=None):
        if not paired:
            return one_system(marks, save)
        if state["t"] == 0:
            first_forward()
        return one_pair(marks, save)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(dev.index if dev.index is not None else 0)
    marks = [[ev(), ev(), ev()] for _ in range(args.steps)]
    t0 = time.perf_counter()
    rows = [step(marks[k]) for k in range(args.steps)]
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    ms = max_over_ranks(marks[0][0].elapsed_time(marks[-1][2]), dev)
    fwd_ms = [mk[0].elapsed_time(mk[1]) for mk in marks]
    adj_ms = [mk[1].elapsed_time(mk[2]) for mk in marks]
    value = 2 * args.steps * ws / (ms / 1e3)
    ms_step = ms / args.steps

    launches = 0
    for r in rows:
        launches += 2  # right-hand sides
        if paired:
            launches += pair_launch_count(info, [r["iters"], r["adjoint_iters"]], [r["outer"], r["adjoint_outer"]],
                                          r["paired"])
        else:
            launches += launch_count(info, args.mode, args.m, fp32, [r["iters"], r["adjoint_iters"]],
                                     [r["outer"], r["adjoint_outer"]])
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if not fp32 else "f32 inner, f64 refinement", "data": "synthetic",
        "config": {"workload": workload_name(args, p), "config": args.config, "grid": args.grid, "n": n,
                   "nnz": p.nnz, "systems_in_sequence": args.systems,
                   "step": ("the forward solve of system t + 1 with the adjoint of system t, paired "
                            "(esd_solve_pair)" if paired else
                            "one system of the sequence: forward solve + adjoint solve"),
                   "m": args.m, "m_kept": state["kept"], "mode": args.mode, "tol": args.tol,
                   "precision": args.precision, "inner_tol": args.inner_tol if fp32 else None,
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "l2": "inputs larger than L2 (matrix, factor, W and vectors > 129 MB)"},
        "gpu_launches": launches,
        "clocks": clk,
        "wall_s_timed": wall,
        "time_to_tol_ms_per_system": ({"pair": float(np.mean(fwd_ms)), "per_solve": ms_step / 2} if paired else
                                      {"forward": float(np.mean(fwd_ms)), "adjoint": float(np.mean(adj_ms)),
                                       "per_solve": ms_step / 2}),
        "systems": [r["system"] for r in rows],
        "paired_iterations": [r["paired"] for r in rows] if paired else None,
        "iterations": [r["iters"] for r in rows],
        "adjoint_iterations": [r["adjoint_iters"] for r in rows],
        "refinement_steps": [r["outer"] for r in rows] if fp32 else None,
        "true_relres_max": max(max(r["true_relres"], r["adjoint_true_relres"]) for r in rows),
        "cond_estimate_system1": {"lmin": state["cond"][0], "lmax": state["cond"][1], "kappa": state["cond"][2]}
        if state["cond"] else None,
    }
    if rank != 0 or args.no_extras:
        return result, None

    # roofline of the dominant kernel from live per-kernel times of the same kernels
    S.set_mode(mode)
    peaks = read_peaks()
    if paired:
        # the kernels of the timed steps: the paired launches (b and g of the last step)
        prof = S.profile_pair_iterations(Sa, b, x.clone(), g, lam.clone(), reps=10)
        result["roofline"], result["kernel_times_ms"] = roofline(prof, p, args, mode, esd, peaks, A.layout(),
                                                                 pair=True)
        result["kernel_times_ms_unpaired"] = dict(S.profile_iterations(b, x.clone(), reps=10))
    else:
        prof = S.profile_iterations(b, x.clone(), reps=10)
        result["roofline"], result["kernel_times_ms"] = roofline(prof, p, args, mode, esd, peaks, A.layout())

    # the next two systems: this mode (advancing the sequence), then from the same b_t and
    # x_{t-1} (and g_t, lambda_{t-1}) the other modes of this precision form with the same W,
    # and plain FP64 PCG resumed until its true residual meets the tolerance
    S64 = esd.Solver(A, maxit_cap=20000, sample_cap=0)
    S64.solve(b, x.clone(), args.tol, 20000, 0)  # graph capture
    others = [k for k in ("plain", "deflation", "sc") if k != args.mode]
    for name in others:  # graph capture of the other modes
        S.set_mode(modes_map[name])
        S.solve(b, x.clone(), args.tol, 20000, 0)
    S.set_mode(mode)

    def timed_solve(solver, bv, x0):
        xv = x0.clone()
        e0, e1 = ev(), ev()
        torch.cuda.synchronize()
        e0.record()
        st, its, rr = solver.solve(bv, xv, args.tol, 20000, 0)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), its, solver.last_solve_info()

    cmp_rows = []
    for _ in range(2):
        saved = {}
        mk = [ev(), ev(), ev()]
        r = step(mk, save=saved)
        torch.cuda.synchronize()
        row = {"system": r["system"], "this": {"iters": r["iters"], "adjoint_iters": r["adjoint_iters"],
                                               "true_relres": r["true_relres"],
                                               "adjoint_true_relres": r["adjoint_true_relres"]}}
        if paired:
            row["adjoint_of"] = r["adjoint_of"]
            row["this"].update(pair_ms=mk[0].elapsed_time(mk[1]), paired=r["paired"])
            # the same two solves one after the other (esd_solve), same mode and precision
            fms, fit, finfo = timed_solve(S, saved["b"], saved["x0"])
            ams, ait, ainfo = timed_solve(S, saved["g"], saved["lam0"])
            row["plain_unpaired"] = {"forward_ms": fms, "adjoint_ms": ams, "iters": fit, "adjoint_iters": ait,
                                     "true_relres": max(finfo["true_relres"], ainfo["true_relres"])}
        else:
            row["this"].update(forward_ms=mk[0].elapsed_time(mk[1]), adjoint_ms=mk[1].elapsed_time(mk[2]))
        for name in others:
            S.set_mode(modes_map[name])
            fms, fit, finfo = timed_solve(S, saved["b"], saved["x0"])
            ams, ait, ainfo = timed_solve(S, saved["g"], saved["lam0"])
            row[name] = {"forward_ms": fms, "adjoint_ms": ams, "iters": fit, "adjoint_iters": ait,
                         "true_relres": max(finfo["true_relres"], ainfo["true_relres"])}
        S.set_mode(mode)
        for name, bv, x0 in (("forward", saved["b"], saved["x0"]), ("adjoint", saved["g"], saved["lam0"])):
            xv = x0.clone()
            e0, e1 = ev(), ev()
            torch.cuda.synchronize()
            e0.record()
            st, its, rr = S64.solve(bv, xv, args.tol, 20000, 0)
            first_true = S64.true_relres()
            resumed = 0
            while S64.true_relres() > args.tol and resumed < 10:
                st, it2, rr = S64.solve(bv, xv, args.tol, 20000, 0)
                its += it2
                resumed += 1
            e1.record()
            torch.cuda.synchronize()
            row["fp64_plain_" + name] = {"ms": e0.elapsed_time(e1), "iters": its, "resumed": resumed,
                                         "true_relres_first_stop": first_true, "true_relres": S64.true_relres()}
        cmp_rows.append(row)
    pair_ms = lambda c: c["pair_ms"] if "pair_ms" in c else c["forward_ms"] + c["adjoint_ms"]  # noqa: E731
    this_ms = float(np.mean([pair_ms(c["this"]) for c in cmp_rows]))
    f64_ms = float(np.mean([c["fp64_plain_forward"]["ms"] + c["fp64_plain_adjoint"]["ms"] for c in cmp_rows]))
    result["vs_fp64_plain"] = {"systems": cmp_rows, "ms_per_system_this": this_ms / 2,
                               "ms_per_system_fp64_plain_to_true_tol": f64_ms / 2,
                               "speedup_vs_fp64_plain": f64_ms / this_ms}
    # every mode of this precision form on the same systems (W from m samples of system 1)
    modes_out = {args.mode: {"ms_per_solve": this_ms / 2,
                             "iters_per_solve": float(np.mean([(c["this"]["iters"] + c["this"]["adjoint_iters"]) / 2
                                                               for c in cmp_rows]))}}
    for name in others + (["plain_unpaired"] if paired else []):
        ms_o = float(np.mean([c[name]["forward_ms"] + c[name]["adjoint_ms"] for c in cmp_rows]))
        modes_out[name] = {"ms_per_solve": ms_o / 2,
                           "iters_per_solve": float(np.mean([(c[name]["iters"] + c[name]["adjoint_iters"]) / 2
                                                             for c in cmp_rows]))}
    base = modes_out["plain"]
    for name, v in modes_out.items():
        v["speedup_vs_fp64_plain"] = (f64_ms / 2) / v["ms_per_solve"]
        v["ms_per_iter"] = v["ms_per_solve"] / v["iters_per_solve"]
        if name != "plain":
            # Eq. ganma: an accelerated mode wins when its iteration cut exceeds its cost ratio
            v["gamma_measured"] = v["ms_per_iter"] / base["ms_per_iter"]
            v["iteration_ratio"] = v["iters_per_solve"] / base["iters_per_solve"]
    result["modes"] = {"m_kept": state["kept"], "by_mode": modes_out,
                       "fastest": min(modes_out, key=lambda k: modes_out[k]["ms_per_solve"])}
    # HBM GB/s per iteration on the paper's byte model: this form against plain FP64
    s_in = 4 if fp32 else 8
    m_eff = state["kept"] if mode != esd.PLAIN else 0
    lay = A.layout() if mode == esd.PLAIN else None
    mat = matrix_bytes(p, s_in, lay, 0) + (matrix_bytes(p, s_in, lay, 1) + matrix_bytes(p, s_in, lay, 2)
                                           if lay is not None and lay["column_free"][1] else (s_in + 4) * p.nnz)
    vec_this = (4 + 12 * s_in) * n + (2 * s_in * m_eff * n + 2 * s_in * n if m_eff else 0)
    model_this = mat + vec_this
    model_f64 = 24 * p.nnz + 100 * n
    it_this = np.mean([c["this"]["iters"] + c["this"]["adjoint_iters"] for c in cmp_rows])
    it_f64 = np.mean([c["fp64_plain_forward"]["iters"] + c["fp64_plain_adjoint"]["iters"] for c in cmp_rows])
    # a paired iteration reads the matrix once for both systems
    np_this = np.mean([c["this"].get("paired", 0) for c in cmp_rows])
    bytes_this = np_this * (mat + 2 * vec_this) + (it_this - 2 * np_this) * model_this
    result["iteration_bandwidth"] = {
        "this": {"model_bytes_per_iter": model_this, "ms_per_iter": this_ms / it_this,
                 "paired_iters": float(np_this), "model_bytes": bytes_this,
                 "model_gbs": bytes_this / (this_ms / 1e3) / 1e9},
        "fp64_plain": {"model_bytes_per_iter": model_f64, "ms_per_iter": f64_ms / it_f64,
                       "model_gbs": model_f64 / (f64_ms / it_f64 / 1e3) / 1e9},
        "peak_gbs": peaks["hbm_gbs"], "peak_src": peaks["src"]}
    result["e2e"] = system_e2e(esd, p, args, torch, S, x, lam, src, neg2xt, Sa)
    return result, None


def system_e2e(esd, p, args, torch, S, x, lam, src, neg2xt, Sa=None):
    """The same step through the C ABI with host buffers: the right-hand sides and both
    solves (or the pair solve, with Sa) take pinned host arrays, so every system's inputs go
    in and its results come back inside the timed region (the library stages the copies)."""
    pin = lambda t: t.cpu().pin_memory()  # noqa: E731
    x_h, lam_h, src_h, n2_h = pin(x), pin(lam), pin(src), pin(neg2xt)
    b_h = torch.zeros(p.n, dtype=torch.float64).pin_memory()
    g_h = torch.zeros_like(b_h).pin_memory()
    inv_dt = 1.0 / p.dt

    def step():
        if Sa is not None:
            S.backward_euler_rhs(x_h, src_h, inv_dt, b_h)
            S.backward_euler_rhs(x_h, n2_h, 2.0, g_h)
            st, _, _, _ = S.solve_pair(Sa, b_h, x_h, g_h, lam_h, args.tol, 20000)
        else:
            S.backward_euler_rhs(x_h, src_h, inv_dt, b_h)
            st, _, _ = S.solve(b_h, x_h, args.tol, 20000, 0)
            if st == esd.OK:
                S.backward_euler_rhs(x_h, n2_h, 2.0, g_h)
                st, _, _ = S.solve(g_h, lam_h, args.tol, 20000, 0)
        if st != esd.OK:
            raise RuntimeError(f"end-to-end step returned {st}")

    step()
    torch.cuda.synchronize()
    k = 3
    t0 = time.perf_counter()
    for _ in range(k):
        step()
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    n = p.n
    # rhs: x_prev, s in, b out; solve: b, x in, x out; adjoint rhs: x, -2 x_t in, g out;
    # adjoint solve: g, lambda in, lambda out (paired: the same vectors)
    h2d = 8 * n * 8
    d2h = 8 * n * 4
    return {"value": 2 * k / sec, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": sec * 1e3 / k, "steps": k}


def c4_arm(args, esd, torch, dev, ws, rank):
    """One optimisation step of the differentiation form: theta moves, A(theta) is assembled
    on the device, refactored, AW/E refreshed for the kept W, then x = A^-1 b and the
    adjoint solve with the gradients through the autograd API."""
    from paper_2203_08498_gb300.adjoint import FVDiffusion, fv_solve
    p, theta, xt = workload(args)
    mode = {"plain": esd.PLAIN, "deflation": esd.DEFLATION, "sc": esd.SUBSPACE_CORRECTION}[args.mode]
    fp32 = args.precision == "fp32"
    model = FVDiffusion(p, mode=mode, precision=esd.FP32_REFINE if fp32 else esd.FP64, sample_cap=max(args.m, 2))
    th0 = torch.from_numpy(np.ascontiguousarray(theta.ravel(order="F"))).to(dev)
    b = torch.from_numpy(p.source).to(dev)
    xt_d = torch.from_numpy(xt).to(dev)
    kept = model.build_W(th0, b, m=args.m, tol=args.tol) if mode != esd.PLAIN else 0
    delta = torch.from_numpy(np.random.default_rng(20220316 + 8).standard_normal(p.n)).to(dev)
    counter = {"k": 0, "its": []}

    def step():
        counter["k"] += 1
        th = (th0 + 1e-4 * counter["k"] * delta).requires_grad_(True)
        x = fv_solve(th, b, model, tol=args.tol)
        fwd = model.solver.last_solve_info()["iters"]
        ((x - xt_d) ** 2).sum().backward()
        adj = model.solver.last_solve_info()["iters"]
        counter["its"].append((fwd, adj))
        return th.grad

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(torch.cuda.current_device())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    info = model.matrix.info()
    its = counter["its"][-args.steps:]
    flat = [k for pair in its for k in pair]
    launches = args.steps * (1 + info["fwd_levels"] + 1 + (9 + args.m if mode != esd.PLAIN else 0) + 1)
    launches += launch_count(info, args.mode, args.m, fp32, flat, [1] * len(flat))
    result = {
        "metric": METRIC, "value": 2 * args.steps * ws / (ms / 1e3), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if not fp32 else "f32 inner, f64 refinement",
        "data": "synthetic",
        "config": {"workload": workload_name(args, p), "config": "c4", "grid": args.grid, "n": p.n,
                   "nnz": p.nnz, "m": args.m, "m_kept": kept, "mode": args.mode, "tol": args.tol,
                   "precision": args.precision, "parallelism": "single GPU",
                   "l2": "inputs larger than L2"},
        "gpu_launches": launches, "clocks": clk,
        "iterations_forward_adjoint": its,
        "time_to_tol_ms_per_system": ms / args.steps / 2,
        "e2e": {"value": None, "unit": UNIT, "h2d_bytes_per_step": None, "d2h_bytes_per_step": None,
                "note": "end-to-end host-buffer timing is taken on the headline 128^3 sequence only"},
    }
    return result, None


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return {"hbm_gbs": d["hbm_gbs"], "src": "measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "src": "fallback"}


FP64_NOMINAL_TFLOPS = 1.25  # GB300 FP64 (CUDA cores and tensor), nominal


FP32_NOMINAL_TFLOPS = 80.5  # 152 SMs x 128 FP32 FMA/clk x 2 x 2.07 GHz


def matrix_bytes(p, s, layout, part):
    """Bytes of one pass over a matrix part (0: A, 1: L, 2: U; L + U together for one sweep
    pair) in the format the kernels of value size s read: (value, column) entries, s + 4
    bytes each; or, for the FP32 kernels of a part with the column-free copy, its 4-byte slot
    values and 32 bytes of slot bases per 32-row slice."""
    entries = p.nnz if part == 0 else (p.nnz - p.n) // 2
    if s == 4 and layout is not None and layout["column_free"][part]:
        return 4 * layout["slot_entries"][part] + 32 * layout["slices"]
    return (s + 4) * entries


def kernel_model(name, p, args, mode, esd, lv, layout=None, pair=False):
    """Algorithmic bytes and FMAs of one launch, each array element counted once; value
    size s = 8 (FP64) or 4 (FP32 inner kernels, whose SpMV also reads s = A 1). pair: the
    paired launch of two systems (plain FP32), which reads the matrix, s = A 1 and 1/l_ii
    once and every vector of each system."""
    if pair:
        one_b, one_f = kernel_model(name, p, args, mode, esd, lv, layout)
        if one_b is None:
            return None, None
        n = p.n
        shared = matrix_bytes(p, 4, layout, 0) + 4 * n if name == "spmv_pq" else 4 * int(lv[0][0])
        return 2 * one_b - shared, 2 * one_f
    n, nnz = p.n, p.nnz
    s = 4 if args.precision == "fp32" else 8
    m = args.m if mode != esd.PLAIN else 0
    rows, low, up = lv
    if name == "spmv_pq":
        mb = m if mode == esd.DEFLATION else 0
        extra = 4 * n if s == 4 else 0
        # FP64 deflation with up to 32 (padded) columns forms (AW)^T p in double-float on the
        # FP32 pipe: only the matrix product and (p, q) are FP64 FMAs
        df = s == 8 and 0 < mb and pad_m(mb) <= 32
        # the deflated FP32 product keeps the (value, column) pairs
        lay = layout if mb == 0 else None
        return (matrix_bytes(p, s, lay, 0) + (2 * s + 4) * n + extra + s * mb * n,
                nnz + n + (0 if df else mb * n))
    if name == "update":
        dm = m if mode == esd.DEFLATION else 0
        sm = m if mode == esd.SUBSPACE_CORRECTION else 0
        n0 = int(rows[0])  # forward level 0 (colour 0): y = r / l_ii
        # x read and written (FP64 in both forms: the refinement form keeps the iterate in
        # FP64), p and q read, r read and written
        base = 16 * n + 4 * s * n
        dm_fp64 = 0 if (s == 8 and 0 < dm and pad_m(dm) <= 32) else dm  # AW y in double-float
        return base + s * (dm + sm) * n + 2 * s * n0, 3 * n + (dm_fp64 + sm) * n + 2 * n0
    return None, None


def pad_m(m):
    """The column count the library compiles for m columns of W."""
    return 0 if m <= 0 else next(c for c in (8, 16, 24, 32, 64) if m <= c)


def roofline(prof, p, args, mode, esd, peaks, layout=None, pair=False):
    lv = level_stats(p)
    times = {nm: t for nm, t in prof}
    cand = [(t, nm) for nm, t in prof if nm in ("spmv_pq", "update")]
    t_ms, name = max(cand)
    by, fmas = kernel_model(name, p, args, mode, esd, lv, layout, pair)
    sec = t_ms / 1e3
    gbs = by / sec / 1e9
    tflops = 2 * fmas / sec / 1e12
    f_hbm = gbs / peaks["hbm_gbs"]
    alu_peak = FP32_NOMINAL_TFLOPS if args.precision == "fp32" else FP64_NOMINAL_TFLOPS
    f_alu = tflops / alu_peak
    full_size = args.grid == CONFIGS[args.config]["grid"]
    key = (args.config, args.precision, name + ("_pair" if pair else ""))
    traffic = read_traffic(TRAFFIC.get(key)) if full_size else None
    name = name + " (paired, two systems)" if pair else name
    if f_alu > f_hbm:
        roof = {"bound": "alu", "achieved": tflops, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": f_alu, "traffic": traffic, "kernel": name,
                "peak_src": "nominal FP64 (152 SMs x 2 FP64 FMA/clk x 2.07 GHz)",
                "hbm": {"achieved": gbs, "peak": peaks["hbm_gbs"], "frac": f_hbm, "peak_src": peaks["src"]}}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": f_hbm,
                "traffic": traffic, "kernel": name, "peak_src": peaks["src"],
                "alu": {"achieved": tflops, "peak": alu_peak, "frac": f_alu}}
    roof["bytes_per_launch"] = by
    roof["ms_per_launch"] = t_ms
    return roof, times


# ncu summaries that hold the DRAM traffic of a configuration's dominant kernel per launch at
# the configuration's full size: (config, precision, kernel) -> file under profiles/
TRAFFIC = {
    ("c2", "fp64", "spmv_pq"): "spmv_pq_fp64_plain_128cube_traffic.txt",
    ("c5", "fp32", "spmv_pq"): "spmv_pq_stream_colfree_fp32_256cube_traffic.txt",
    ("c5", "fp32", "spmv_pq_pair"): "spmv_pq_pair_colfree_fp32_256cube_traffic.txt",
}


def read_traffic(fname):
    """DRAM bytes per launch from the committed ncu summary of this kernel, if any."""
    if fname is None:
        return None
    path = os.path.join(ROOT, "profiles", fname)
    try:
        for ln in open(path):
            if ln.startswith("traffic_bytes_per_launch:"):
                return float(ln.split(":")[1])
    except OSError:
        pass
    return None


def power_method_report(esd, A, p, args, b, torch, peaks):
    """Algorithm PCG-con (Section 5.4) on one system of the sequence: ICCG with m sampled
    iterates and the power method multiplied in the same SpMV pass, then lambda_max, the
    smallest Ritz value of the sampled errors and kappa. Its cost: graph time per iteration
    of the same sampled solve with and without the power product, and the fused SpMV's live
    kernel time against its byte and FMA model (16 more bytes and nnz more FMAs per row)."""
    import workloads as wl
    S = esd.Solver(A, maxit_cap=20000, sample_cap=max(args.m, 2))
    v0 = torch.from_numpy(np.random.default_rng(wl.SEED_BASE + 7).standard_normal(p.n)).to(b.device)

    def timed_solve():
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, it, rr = S.solve(b, x, args.tol, 20000, args.m)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, it

    timed_solve()  # graph capture
    t_off, it_off = timed_solve()
    k_off = dict(S.profile_iterations(b, torch.zeros_like(b), reps=20))
    S.power_start(v0)
    timed_solve()  # graph capture with the power product
    S.power_start(v0)
    t_on, it_on = timed_solve()
    _, steps = S.power_estimate()
    S.sample_and_build_W()
    lmax, lmin, kappa = S.paper_cond_estimate()
    k_on = dict(S.profile_iterations(b, torch.zeros_like(b), reps=20))
    S.power_start(None)
    n, nnz = p.n, p.nnz
    t_k = k_on["spmv_pq"] / 1e3
    by = 12 * nnz + 20 * n + 16 * n
    fmas = 2 * nnz + 2 * n
    return {"lambda_max": lmax, "power_steps": steps, "ritz_min": lmin, "kappa": kappa,
            "iterations": it_on, "us_per_iteration_without": t_off / it_off * 1e6,
            "us_per_iteration_with": t_on / it_on * 1e6, "cost_frac": (t_on / it_on) / (t_off / it_off) - 1.0,
            "spmv_pq_us_without": k_off["spmv_pq"] * 1e3, "spmv_pq_us_with": k_on["spmv_pq"] * 1e3,
            "fused_spmv": {"model_bytes": by, "gbs": by / t_k / 1e9, "hbm_frac": by / t_k / 1e9 / peaks["hbm_gbs"],
                           "fp64_tflops": 2 * fmas / t_k / 1e12,
                           "fp64_frac": 2 * fmas / t_k / 1e12 / FP64_NOMINAL_TFLOPS}}


def sampling_comparison(esd, A, p, args, b, torch):
    """Sampling method A (Appendix A) against method B (Section 4.2) on the same first solve:
    m sampled iterates each, W = Q from their errors, then the deflated and the SC solve of
    another right-hand side (seeded uniform random, as the paper's later systems) from x = 0;
    the paper compares the two methods by such counts."""
    import workloads as wl
    b2 = torch.from_numpy(wl.random_rhs(p.n, wl.SEED_BASE + 8)).to(b.device)
    out = {}
    for name, method in (("A", esd.SAMPLING_A), ("B", esd.SAMPLING_B)):
        S = esd.Solver(A, maxit_cap=20000, sample_cap=max(args.m, 2), sampling=method)
        x = torch.zeros_like(b)
        st, it0, rr = S.solve(b, x, args.tol, 20000, args.m)
        kept = S.sample_and_build_W()
        row = {"first_solve_iterations": it0, "m_kept": kept, "ritz_min": float(S.ritz_values()[0])}
        for mname, md in (("plain", esd.PLAIN), ("deflation", esd.DEFLATION), ("sc", esd.SUBSPACE_CORRECTION)):
            S.set_mode(md)
            x = torch.zeros_like(b2)
            st, it, rr = S.solve(b2, x, args.tol, 20000, 0)
            row[mname + "_iterations"] = it
        out[name] = row
    return out


def ordering_comparison(esd, p, args, torch, device):
    """The first system of the sequence (b = s, x0 = 0, plain FP64 ICCG) with IC(0) in three
    orderings of the same operator: the configs' multicolour ordering; block-Jacobi IC with
    natural order inside 16^3 blocks (the paper's parallel solver, Section 5.3, with the
    blocks' wavefronts as launches); natural order (one launch per wavefront)."""
    import workloads as wl
    out = {}
    cases = (("multicolour", None, None), ("block_jacobi_16", wl.block_wavefront_colours(p.shape, 16), 16),
             ("natural", wl.wavefront_colours(p.shape), None))
    for name, colours, blk in cases:
        q = p if colours is None else wl.reorder(p, colours)
        A = esd.Matrix.from_problem(q)
        A.factor_ic0()
        S = esd.Solver(A, maxit_cap=20000, sample_cap=0)
        P = None
        if blk is not None:
            P = esd.Matrix.from_problem(wl.block_diagonal_part(q, wl.block_ids(p.shape, blk)))
            P.factor_ic0()
            S.set_precond_matrix(P)
        levels = (P or A).info()["fwd_levels"]
        bt = torch.from_numpy(q.source).to(device)
        x = torch.zeros_like(bt)
        S.solve(bt, x, args.tol, 20000, 0)  # graph capture
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, it, rr = S.solve(bt, x, args.tol, 20000, 0)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        out[name] = {"levels_per_sweep": levels, "iterations": it, "ms_per_solve": sec * 1e3,
                     "us_per_iteration": sec / max(it, 1) * 1e6}
    return out


def iteration_roofline(S, esd, p, args, x, b, src, peaks):
    """Time per iteration of each mode (graph launches of system 2) against the paper's
    per-iteration byte model (Eq. ticcg / tsciccg generalised to m columns)."""
    import torch
    out = {}
    n, nnz = p.n, p.nnz
    m = args.m
    for name, md in (("plain", esd.PLAIN), ("deflation", esd.DEFLATION), ("sc", esd.SUBSPACE_CORRECTION)):
        S.set_mode(md)
        x0 = torch.zeros_like(x)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, it, rr = S.solve(b, x0, args.tol, 20000, 0)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        model = 24 * nnz + 100 * n + (16 * m * n + 16 * n if md != esd.PLAIN else 0)
        tpi = sec / max(it, 1)
        out[name] = {"iters": it, "ms_per_iter": tpi * 1e3, "model_bytes_per_iter": model,
                     "model_gbs": model / tpi / 1e9, "frac_of_hbm_peak": model / tpi / 1e9 / peaks["hbm_gbs"]}
    return out


def e2e(esd, p, args, torch):
    """The same sequence through the C ABI with host buffers: CSR upload, factorisation and
    per system the right-hand side and the solve with host b and x (copies inside)."""
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
    rp, ci, va = pin(p.rowptr.astype(np.int32)), pin(p.colind.astype(np.int32)), pin(p.val)
    src_h = pin(p.source)
    x_h = torch.zeros(p.n, dtype=torch.float64).pin_memory()
    b_h = torch.zeros(p.n, dtype=torch.float64).pin_memory()
    mode = {"plain": esd.PLAIN, "deflation": esd.DEFLATION, "sc": esd.SUBSPACE_CORRECTION}[args.mode]

    def step():
        A = esd.Matrix(rp, ci, va, p.colour_ptr)
        A.factor_ic0()
        S = esd.Solver(A, maxit_cap=20000, sample_cap=max(args.m, 2))
        x_h.zero_()
        for t in range(args.systems):
            S.backward_euler_rhs(x_h, src_h, 1.0 / p.dt, b_h)
            if t == 0:
                S.solve(b_h, x_h, args.tol, 20000, args.m if mode != esd.PLAIN else 0)
                S.estimate_cond()
                if mode != esd.PLAIN:
                    S.sample_and_build_W()
                    S.set_mode(mode)
            else:
                S.solve(b_h, x_h, args.tol, 20000, 0)
        S.close()
        A.close()

    step()  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    k = max(1, args.steps)
    for _ in range(k):
        step()
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    n = p.n
    h2d = 4 * (n + 1) + 12 * p.nnz + args.systems * 32 * n
    d2h = args.systems * 16 * n
    return {"value": args.systems * k / sec, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": sec * 1e3 / k}


# ---------------------------------------------------------------- CPU oracle

def oracle_rates(p, args, iters_plain=20, iters_acc=20, m=None):
    """Seconds per oracle iteration (plain ICCG and the accelerated mode) with whichever
    oracle library is current (serial, or the OpenMP build under oracle.using)."""
    import oracle
    ic = oracle.IC0(p)
    rng = np.random.default_rng(0)
    out = {}
    t0 = time.perf_counter()
    oracle.System(p, ic).solve(p.source, tol=1e-300, maxit=iters_plain, history=False)
    out["plain"] = (time.perf_counter() - t0) / iters_plain
    m = m or args.m
    if args.mode != "plain" and m > 0:
        # any full-rank W costs the same per iteration: scaled Gaussian columns
        W = np.asfortranarray(rng.standard_normal((p.n, m)) / math.sqrt(p.n))
        aux = oracle.Aux.from_basis(p, W)
        md = oracle.DEFLATION if args.mode == "deflation" else oracle.SUBSPACE_CORRECTION
        t0 = time.perf_counter()
        oracle.System(p, ic, md, aux).solve(p.source, tol=1e-300, maxit=iters_acc, history=False)
        out["acc"] = (time.perf_counter() - t0) / iters_acc
    else:
        out["acc"] = out["plain"]
    return out


def extrapolate(rates, its, first_plain=True):
    """Solves per second of a run with these iteration counts per solve at these rates (the
    first solve plain when the sequence samples W in it)."""
    if first_plain:
        sec = rates["plain"] * its[0] + rates["acc"] * sum(its[1:])
    else:
        sec = rates["acc"] * sum(its)
    return len(its) / sec


def host_info():
    """Host cores and CPU model of the machine that timed the oracle."""
    import platform
    model = platform.processor() or platform.machine()
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model, "machine": platform.machine()}


def cpu_baseline(p, args, its, first_plain=True, m=None):
    """The oracle timed on the host: one thread, and the OpenMP build of the same source on
    every core (rows of a colour, SpMV rows and vector updates shared among threads; results
    bit-identical). A bounded sample of iterations, extrapolated to solves per second with
    this run's iteration counts."""
    import oracle
    k = 20 if p.nnz < 50_000_000 else 3  # keep the CPU sample to tens of seconds
    entries = []
    r1 = oracle_rates(p, args, iters_plain=k, iters_acc=k, m=m)
    entries.append({"cores": 1, "value": extrapolate(r1, its, first_plain), "s_per_iter": r1})
    try:
        omp = oracle.openmp_lib()
        with oracle.using(omp):
            rn = oracle_rates(p, args, iters_plain=k, iters_acc=k, m=m)
        entries.append({"cores": int(omp.orc_threads()), "value": extrapolate(rn, its, first_plain),
                        "s_per_iter": rn})
    except Exception as e:  # no OpenMP in this compiler: the single-thread timing stands alone
        entries.append({"cores": None, "value": None, "unavailable": f"OpenMP oracle: {e}"})
    best = max((e for e in entries if e.get("value")), key=lambda e: e["value"])
    return {"value": best["value"], "unit": UNIT, "cores": best["cores"], "kind": "oracle", "host": host_info(),
            "entries": entries,
            "sample": (f"{k} plain and {k} {args.mode} FP64 ICCG iterations of the {args.config} system "
                       f"(n={p.n}, m={m or args.m} columns of W) per timing, extrapolated with this run's "
                       f"iteration counts per solve; single thread and OpenMP on all host cores")}


def oracle_counts(args):
    """The oracle's iteration counts for this sequence (written by oracle/sequence_counts.py)."""
    path = os.path.join(ROOT, "oracle", "data", f"fv7_{args.grid}cube_{args.mode}_counts.json")
    try:
        its = json.load(open(path))["iterations"]
        return its[: args.systems]
    except (OSError, KeyError, ValueError):
        raise SystemExit(f"missing {path}: run python -m oracle.sequence_counts {args.mode}")


def c5_oracle_counts(args):
    """The oracle's own forward and adjoint iteration counts of the 256^3 sequence's systems
    in this mode (oracle/data, written by oracle/sequence_counts.py --c5 from the oracle
    alone); system 2 stands for every later system."""
    mode = "plain" if args.mode == "plain" else args.mode
    path = os.path.join(ROOT, "oracle", "data", f"fv7_256cube_{mode}_counts.json")
    try:
        d = json.load(open(path))
        k = 1 if len(d["iterations"]) > 1 else 0
        return d["iterations"][k], d["adjoint_iterations"][k], path
    except (OSError, KeyError, ValueError, IndexError):
        raise SystemExit(f"missing {path}: run python -m oracle.sequence_counts --c5 {mode}")


def reference_arm(args):
    """The CPU oracle on this arm's workload, metric and unit: per step a bounded sample of
    oracle iterations (plain and the configured mode), extrapolated to solves per second with
    the oracle's own iteration counts. C5 (one system = forward + adjoint solve) runs the
    OpenMP build of the oracle on every host core; C2 the single-threaded build."""
    import oracle
    ws, rank, local = dist_env()
    if rank != 0:
        return
    if args.config not in ("c2", "c5"):
        print(json.dumps({"impl": "reference", "unavailable": "the oracle arm is timed on the 128^3 and 256^3 "
                          "sequences (configs c2 and c5) only"}), flush=True)
        return
    p = workload(args)
    vals = []
    if args.config == "c5":
        fwd, adj, path = c5_oracle_counts(args)
        omp = oracle.openmp_lib()
        with oracle.using(omp):
            for s_ in range(args.warmup + args.steps):
                r = oracle_rates(p, args, iters_plain=4, iters_acc=4, m=args.m)
                sec = r["acc"] * (fwd + adj)
                if s_ >= args.warmup:
                    vals.append(2.0 / sec)
        cores = int(omp.orc_threads())
        sample = (f"4 plain and 4 {args.mode} FP64 oracle iterations per step (OpenMP, {cores} threads), "
                  f"extrapolated with the oracle's own forward + adjoint counts of system 2 ({fwd} + {adj}, "
                  f"{os.path.relpath(path, ROOT)}); the oracle has no FP32 form")
    else:
        its = oracle_counts(args)
        for s_ in range(args.warmup + args.steps):
            r = oracle_rates(p, args, iters_plain=5, iters_acc=5)
            if s_ >= args.warmup:
                vals.append(extrapolate(r, its))
        cores = 1
        sample = ("5 plain and 5 accelerated oracle iterations per step, extrapolated with the oracle's own "
                  "iteration counts of this sequence (oracle/data, written by oracle/sequence_counts.py)")
    v = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args, p), "config": args.config, "grid": args.grid, "n": p.n,
                       "nnz": p.nnz, "mode": args.mode},
            "cpu_baseline": {"value": v, "unit": UNIT, "kind": "oracle", "cores": cores, "host": host_info(),
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        reference_arm(args)
        return
    result, modes = gpu_arm(args)
    if rank == 0:
        if not args.no_extras and ws == 1:
            if args.config == "c4":
                p = workload(args)[0]
                its = [k for pair in result["iterations_forward_adjoint"] for k in pair]
            elif args.config == "c5":
                p = workload(args)
                its = list(result["iterations"]) + list(result["adjoint_iterations"])
                result["cpu_baseline"] = cpu_baseline(p, args, its, first_plain=False,
                                                      m=result["config"]["m_kept"])
            else:
                p = workload(args)
                its = list(result["iterations"])
                if args.adjoint:
                    its += list(result["adjoint_iterations"])
            if "cpu_baseline" not in result:
                result["cpu_baseline"] = cpu_baseline(p, args, its)
        print(json.dumps(result), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
