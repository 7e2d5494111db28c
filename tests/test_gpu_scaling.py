"""Diagonal scaling at creation and switching precision on a live solver (GPU only).

  scaling     ESD_MATRIX_DIAG_SCALE holds D^-1/2 A D^-1/2: d equals the oracle's bit for bit
              (1/sqrt(a_ii), both IEEE-rounded), A^ v matches the oracle's scaled SpMV to
              1e-13, ICCG on A^ x^ = d b matches the oracle's (iterations +-1, x^ 1e-10), the
              theta filter on A^ keeps the oracle's columns; set_values rescales (4A scales to
              the same A^); bad diagonals and the unscaled-only entry points are refused;
  precision   a W built in FP64 and a switch to the refinement form give the same solve as a
              solver created in that form with the same W; switching back restores FP64.
"""
import copy

import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2203_08498_gb300 as esd  # noqa: E402

DEV = torch.device("cuda:0")

PROBLEMS = {
    "fv7_9cube_ragged": lambda: wl.small_3d(9, seed=11),
    "c1_64x64_redblack": lambda: wl.config_c1(),
    "lap1d_odd": lambda: wl.laplacian_1d(37),
}


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("name", sorted(PROBLEMS))
def test_scaled_matrix_matches_oracle(name):
    p = PROBLEMS[name]()
    ps, d_o = oracle.diag_scale(p)
    A = esd.Matrix.from_problem(p, diag_scale=True)
    assert np.array_equal(A.diag_scale(), d_o)
    v = np.random.default_rng(3).standard_normal(p.n)
    y = np.zeros(p.n)
    A.spmv(v, y)
    assert rel(y, oracle.spmv(ps, v)) <= 1e-13
    A.factor_ic0()
    S = esd.Solver(A, sample_cap=8)
    b = p.source if p.source is not None else wl.random_rhs(p.n, 5)
    x = np.zeros(p.n)
    st, it, rr = S.solve(d_o * b, x, tol=1e-8)
    out = oracle.System(ps, oracle.IC0(ps)).solve(d_o * b, tol=1e-8)
    assert st == esd.OK and abs(it - out["iters"]) <= 1
    assert rel(x, out["x"]) <= 1e-10


def test_theta_filter_on_scaled_matrix():
    """The paper's theta (1e-3 .. 1e-5) refers to the scaled matrix: the Ritz values of the
    sampled errors of A^ below theta select the same columns as the oracle's from the same
    samples."""
    p = wl.config_c1()
    ps, d = oracle.diag_scale(p)
    A = esd.Matrix.from_problem(p, diag_scale=True)
    A.factor_ic0()
    S = esd.Solver(A, sample_cap=8)
    x = np.zeros(p.n)
    S.solve(d * p.source, x, tol=1e-10, sample_m=8)
    samples, slot_iter = S.samples(8)
    S.sample_and_build_W()
    ritz = np.sort(S.ritz_values())
    theta = 0.5 * (ritz[2] + ritz[3])
    m = S.sample_and_build_W(theta)
    aux, info = oracle.build_w(ps, x, samples, slot_iter, theta=theta)
    assert m == aux.m == 3
    W, AW, E = S.get_W()
    np.testing.assert_allclose(np.diag(E), np.diag(aux.E), rtol=1e-10)
    assert ritz[-1] < 2.0  # the spectrum of a scaled M-matrix with unit diagonal lies in (0, 2)


def test_set_values_rescales():
    p = wl.small_3d(9, seed=11)
    A = esd.Matrix.from_problem(p, diag_scale=True)
    d0 = A.diag_scale()
    v = np.random.default_rng(4).standard_normal(p.n)
    y0, y1 = np.zeros(p.n), np.zeros(p.n)
    A.spmv(v, y0)
    A.set_values(4.0 * p.val)  # 4A scales to the same A^ with d / 2 (exact in binary)
    np.testing.assert_array_equal(A.diag_scale(), d0 / 2)
    A.spmv(v, y1)
    np.testing.assert_array_equal(y1, y0)
    bad = p.val.copy()
    rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    bad[np.flatnonzero(rows == p.colind)[5]] = 0.0
    with pytest.raises(esd.EsdError) as e:
        A.set_values(bad)
    assert e.value.code == esd.ERR_INVALID
    A.spmv(v, y1)  # unchanged by the refused update
    np.testing.assert_array_equal(y1, y0)


def test_scaling_refusals():
    p = wl.small_3d(5, seed=2)
    bad = p.val.copy()
    rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    bad[np.flatnonzero(rows == p.colind)[0]] = -1.0
    pb = copy.copy(p)
    pb.val = bad
    with pytest.raises(esd.EsdError) as e:
        esd.Matrix.from_problem(pb, diag_scale=True)
    assert e.value.code == esd.ERR_INVALID
    A = esd.Matrix.from_problem(p)
    with pytest.raises(esd.EsdError) as e:
        A.diag_scale()
    assert e.value.code == esd.ERR_STATE
    As = esd.Matrix.from_problem(p, diag_scale=True)
    g = esd.EsdFvGrid(3, 5, 5, 5, p.h, 1.0 / p.dt)
    theta = np.zeros(p.n)
    cell_row = np.empty(p.n, dtype=np.int32)
    cell_row[p.perm] = np.arange(p.n, dtype=np.int32)
    with pytest.raises(esd.EsdError) as e:
        esd.esd_fv_assemble(As.handle, g, theta, cell_row)
    assert e.value.code == esd.ERR_STATE


def test_set_precision_matches_created_form():
    p = wl.config_c1()
    A = esd.Matrix.from_problem(p)
    A.factor_ic0()
    S = esd.Solver(A, sample_cap=8)
    x = np.zeros(p.n)
    S.solve(p.source, x, tol=1e-8, sample_m=8)
    S.sample_and_build_W()
    W, _, _ = S.get_W()
    S.set_precision(esd.FP32_REFINE, inner_tol=0.1)
    S.set_mode(esd.DEFLATION)
    b = wl.random_rhs(p.n, 6)
    xa = np.zeros(p.n)
    st, ita, rra = S.solve(b, xa, tol=1e-8)
    assert st == esd.OK and S.last_solve_info()["outer_steps"] >= 1
    R = esd.Solver(A, sample_cap=8, precision=esd.FP32_REFINE, inner_tol=0.1)
    R.set_W(W)
    R.set_mode(esd.DEFLATION)
    xb = np.zeros(p.n)
    st, itb, rrb = R.solve(b, xb, tol=1e-8)
    assert ita == itb and rra == rrb
    np.testing.assert_array_equal(xa, xb)
    # back to FP64: the recursive residual is the FP64 one again
    S.set_precision(esd.FP64)
    xc = np.zeros(p.n)
    st, itc, rrc = S.solve(b, xc, tol=1e-8)
    assert st == esd.OK and S.last_solve_info()["outer_steps"] == 0
    assert np.linalg.norm(b - p.scipy() @ xc) <= 1.01e-8 * np.linalg.norm(b)


def test_set_precision_refusals():
    p = wl.config_c1()
    A = esd.Matrix.from_problem(p)
    A.factor_ic0()
    S = esd.Solver(A, sample_cap=8, sampling=esd.SAMPLING_B)
    with pytest.raises(esd.EsdError) as e:
        S.set_precision(esd.FP32_REFINE)
    assert e.value.code == esd.ERR_INVALID
    T = esd.Solver(A, sample_cap=8)
    T.power_start(np.ones(p.n))
    with pytest.raises(esd.EsdError) as e:
        T.set_precision(esd.FP32_REFINE)
    assert e.value.code == esd.ERR_STATE
    with pytest.raises(esd.EsdError) as e:
        T.set_precision(esd.FP32_REFINE, inner_tol=1.5)
    assert e.value.code == esd.ERR_INVALID
