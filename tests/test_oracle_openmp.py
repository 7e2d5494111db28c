"""The OpenMP build of the oracle gives bit-identical results to the single-threaded build
(CPU only).

The all-core oracle timing shares the rows of one colour (substitutions), the rows of the
SpMV and the elements of the vector updates among threads; each of those results is
computed by one thread in the same order as in the serial build, and the dot products stay
serial pairwise sums. So the two builds must agree bit for bit, which this checks on the
IC(0) application and on plain, deflated and subspace-corrected solves.
"""
import subprocess

import numpy as np
import pytest

import oracle
import workloads as wl


def _omp_lib():
    try:
        return oracle.openmp_lib()
    except (subprocess.CalledProcessError, OSError) as e:  # a compiler without OpenMP
        pytest.skip(f"no OpenMP build: {e}")


def _run(p, aux, threads_lib=None):
    ctx = oracle.using(threads_lib) if threads_lib is not None else None
    if ctx:
        ctx.__enter__()
    try:
        ic = oracle.IC0(p)
        r = np.random.default_rng(3).standard_normal(p.n)
        out = [ic.apply(r), oracle.spmv(p, r)]
        for mode in (oracle.PLAIN, oracle.DEFLATION, oracle.SUBSPACE_CORRECTION):
            o = oracle.System(p, ic, mode, aux if mode != oracle.PLAIN else None).solve(p.source, tol=1e-10)
            out += [o["x"], o["alpha"], o["beta"], np.array([o["iters"]])]
        o = oracle.System(p, ic).solve(p.source, tol=1e-10, sample_m=8)
        out += [o["samples"], o["sample_iter"].astype(np.float64)]
        return out
    finally:
        if ctx:
            ctx.__exit__(None, None, None)


@pytest.mark.parametrize("name", ["c1", "fv7_12cube", "c3_16"])
def test_openmp_build_is_bit_identical(name, monkeypatch):
    monkeypatch.setenv("OMP_NUM_THREADS", "4")
    p = {"c1": wl.config_c1, "fv7_12cube": lambda: wl.small_3d(12, seed=5),
         "c3_16": lambda: wl.config_c3(N=16)}[name]()
    W, _ = np.linalg.qr(np.random.default_rng(9).standard_normal((p.n, 6)))
    aux = oracle.Aux.from_basis(p, W)
    serial = _run(p, aux)
    threaded = _run(p, aux, _omp_lib())
    for a, b in zip(serial, threaded):
        np.testing.assert_array_equal(a, b)
