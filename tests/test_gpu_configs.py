"""The configurations' own shapes against the oracle on the GPU, element by element.

What the smaller parity problems do not reach:
  27-point FE operator   C3's Q1 anisotropic log-normal matrix (27-wide rows, 8 colours over
                         a 27-point stencil, a matrix that is not an M-matrix): SpMV 1e-13,
                         IC(0) application 1e-12 and the FP64 ICCG solve (+-1 iteration,
                         solution 1e-10) at 24^3 and 40^3; SpMV and IC(0) on every row at
                         the full 192^3 size; the precision form with W sampled in it;
  FP32 W of 24 and 32    the slice-major FP32 copies of W and AW at C3's and C5's widths:
  columns                the first inner FP32 solve against the oracle's FP64 run with the
                         same W (coefficients 2e-4), and refined solves to 1e-10 / 1e-8
                         within kappa(A)(tol + 1e-12) of the oracle's tol-1e-12 solution;
  rank and failures      rank-deficient samples (SVQB, Eq. ekd: m-bar < m vectors), no sample
                         (ESD_ERR_RANK), NaN right-hand side and indefinite (p, Ap)
                         (ESD_ERR_BREAKDOWN), E = W^T A W not positive definite
                         (ESD_ERR_CHOL_E), an IC(0) that needs the diagonal shift;
  full-size solutions    the 128^3 system 2 in deflation and SC with the oracle's x_1 and W:
                         +-1 iteration, solution 1e-10.
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2203_08498_gb300 as esd  # noqa: E402

DEV = torch.device("cuda:0")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def rel(a, b):
    a = a.cpu().numpy() if hasattr(a, "cpu") else a
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def true_relres(p, x, b):
    x = x.cpu().numpy() if hasattr(x, "cpu") else x
    return np.linalg.norm(b - p.scipy() @ x) / np.linalg.norm(b)


def kappa(p):
    A = p.scipy().tocsc()
    lmax = spla.eigsh(A, k=1, which="LA", return_eigenvectors=False)[0]
    lmin = spla.eigsh(A, k=1, sigma=0.0, which="LM", return_eigenvectors=False)[0]
    return lmax / lmin


# ---------------------------------------------------------------- C3's 27-point operator

C3_SMALL = {}


def c3(N):
    if N not in C3_SMALL:
        C3_SMALL[N] = wl.config_c3(N=N)
    return C3_SMALL[N]


@pytest.mark.parametrize("N", [24, 40])
def test_c3_operator_kernels_and_iccg(N):
    p = c3(N)
    assert p.nnz == (3 * N - 2) ** 3 and p.ncolours == 8
    A = esd.Matrix.from_problem(p)
    v = np.random.default_rng(31).standard_normal(p.n)
    y = torch.empty(p.n, dtype=torch.float64, device=DEV)
    A.spmv(dev(v), y)
    assert rel(y, oracle.spmv(p, v)) <= 1e-13
    shift = A.factor_ic0()
    ic = oracle.IC0(p)
    assert shift == ic.shift
    A.apply_ic(dev(v), y)
    assert rel(y, ic.apply(v)) <= 1e-12
    S = esd.Solver(A, sample_cap=0)
    x = torch.zeros(p.n, dtype=torch.float64, device=DEV)
    st, it, rr = S.solve(dev(p.source), x, tol=1e-8)
    out = oracle.System(p, ic).solve(p.source, tol=1e-8)
    assert st == esd.OK and abs(it - out["iters"]) <= 1, (it, out["iters"])
    assert rel(x, out["x"]) <= 1e-10
    a, bb = S.history()
    k = min(it, out["iters"], 10)
    np.testing.assert_allclose(a[:k], out["alpha"][:k], rtol=1e-11)


@pytest.mark.parametrize("mode", [esd.DEFLATION, esd.SUBSPACE_CORRECTION])
def test_c3_operator_accelerated_with_oracle_w(mode):
    """System 2 of the 24^3 C3 sequence in FP64 with the oracle's W (m = 24 samples of
    system 1): iterations +-1, solution 1e-10."""
    p = c3(24)
    ic = oracle.IC0(p)
    o1 = oracle.System(p, ic).solve(p.source, tol=1e-10, sample_m=24)
    aux, info = oracle.build_w(p, o1["x"], o1["samples"], o1["sample_iter"])
    b2 = o1["x"] / p.dt + p.source
    A = esd.Matrix.from_problem(p)
    A.factor_ic0()
    S = esd.Solver(A, sample_cap=0)
    S.set_W(aux.W)
    S.set_mode(mode)
    x = dev(o1["x"].copy())
    st, it, rr = S.solve(dev(b2), x, tol=1e-10)
    out = oracle.System(p, ic, mode, aux).solve(b2, o1["x"], tol=1e-10)
    assert st == esd.OK and abs(it - out["iters"]) <= 1, (it, out["iters"])
    assert rel(x, out["x"]) <= 1e-10


def test_c3_precision_form_sampled_deflation():
    """C3's own path at 24^3: the refinement form samples m = 24 iterates of system 1, builds
    the FP32 W, and solves system 2 deflated to 1e-10 in truth, with fewer inner iterations
    than plain refinement, within kappa(A)(tol + 1e-12) of the oracle's tol-1e-12 solution."""
    p = c3(24)
    A = esd.Matrix.from_problem(p)
    A.factor_ic0()
    S = esd.Solver(A, sample_cap=24, precision=esd.FP32_REFINE)
    x = torch.zeros(p.n, dtype=torch.float64, device=DEV)
    st, it1, rr = S.solve(dev(p.source), x, tol=1e-10, sample_m=24)
    assert st == esd.OK and true_relres(p, x, p.source) <= 1.01e-10
    m = S.sample_and_build_W()
    assert 1 <= m <= 24
    x1 = x.cpu().numpy()
    b2 = x1 / p.dt + p.source
    S.set_mode(esd.PLAIN)
    xp = x1.copy()
    S.solve(b2, xp, tol=1e-10)
    it_plain = S.last_solve_info()["iters"]
    S.set_mode(esd.DEFLATION)
    xd = x1.copy()
    st, it, rr = S.solve(b2, xd, tol=1e-10)
    assert st == esd.OK and true_relres(p, xd, b2) <= 1.01e-10
    assert it < it_plain, (it, it_plain)
    ref = oracle.System(p, oracle.IC0(p)).solve(b2, x1, tol=1e-12)["x"]
    assert rel(xd, ref) <= kappa(p) * (1e-10 + 1e-12)


@pytest.mark.slow
def test_c3_full_size_kernels():
    """The 192^3 27-point operator (7.08M rows, 189M entries): SpMV and IC(0) application on
    every row against the oracle."""
    p = wl.config_c3()
    A = esd.Matrix.from_problem(p)
    v = np.random.default_rng(32).standard_normal(p.n)
    y = torch.empty(p.n, dtype=torch.float64, device=DEV)
    A.spmv(dev(v), y)
    assert rel(y, oracle.spmv(p, v)) <= 1e-13
    shift = A.factor_ic0()
    ic = oracle.IC0(p)
    assert shift == ic.shift
    A.apply_ic(dev(v), y)
    assert rel(y, ic.apply(v)) <= 1e-12


# ---------------------------------------------------------------- FP32 W at 24 and 32 columns

@pytest.fixture(scope="module", params=[24, 32])
def wide_w(request):
    """A 24^3 7-point problem with 1e5 inclusions (~50 ICCG iterations), the oracle's system 1
    with m = 24 or 32 samples, its W (all columns kept) and system 2."""
    m = request.param
    p = wl.small_3d(24, seed=13, count=4, rmin=2, rmax=4, value=1e5)
    ic = oracle.IC0(p)
    o1 = oracle.System(p, ic).solve(p.source, tol=1e-10, sample_m=m)
    aux, info = oracle.build_w(p, o1["x"], o1["samples"], o1["sample_iter"])
    assert aux.m == m
    b2 = o1["x"] / p.dt + p.source
    return m, p, ic, aux, o1["x"], b2


def refine_solver(p, **kw):
    A = esd.Matrix.from_problem(p)
    A.factor_ic0()
    return esd.Solver(A, precision=esd.FP32_REFINE, **kw)


@pytest.mark.parametrize("mode", [esd.DEFLATION, esd.SUBSPACE_CORRECTION])
def test_wide_fp32_w_first_inner_solve(wide_w, mode):
    """One FP32 inner solve of A d = b2 - A x1 with the oracle's W against the oracle's FP64
    run with the same W: coefficients to FP32 accuracy, count within max(2, 5 %)."""
    m, p, ic, aux, x1, b2 = wide_w
    S = refine_solver(p, sample_cap=0, max_outer=1, inner_tol=1e-4)
    S.set_W(aux.W)
    W, AW, E = S.get_W()
    assert W.shape[1] == m
    np.testing.assert_array_equal(W, W.astype(np.float32).astype(np.float64))
    assert np.abs(W - aux.W).max() <= 1e-6 * np.abs(aux.W).max()
    np.testing.assert_allclose(AW, p.scipy() @ W, rtol=1e-12, atol=1e-12 * np.abs(AW).max())
    S.set_mode(mode)
    r0 = b2 - p.scipy() @ x1
    d = torch.zeros(p.n, dtype=torch.float64, device=DEV)
    st, it, rr = S.solve(dev(r0), d, tol=1e-14)
    out = oracle.System(p, ic, mode, aux).solve(r0, np.zeros(p.n), tol=1e-4)
    assert st == esd.ERR_MAXIT and S.last_solve_info()["outer_steps"] == 1
    assert abs(it - out["iters"]) <= max(2, math.ceil(0.05 * out["iters"])), (it, out["iters"])
    # FP32 rounding of (p, q) - h^T E^-1 h drifts the coefficients apart exponentially on this
    # 1e5-contrast problem (1e-6 at the fifth, 1e-2 by the eighth): the first five are compared
    a, bb = S.history()
    k = min(it, out["iters"], 5)
    np.testing.assert_allclose(a[:k], out["alpha"][:k], rtol=2e-4)
    np.testing.assert_allclose(bb[:k - 1], out["beta"][:k - 1], rtol=2e-4)


@pytest.mark.parametrize("resume,inner_tol", [(1, 0.1), (0, 1e-4)])
@pytest.mark.parametrize("mode", [esd.DEFLATION, esd.SUBSPACE_CORRECTION])
def test_wide_fp32_w_refinement(wide_w, mode, resume, inner_tol):
    """System 2 refined to 1e-10 (m = 24, C3's tolerance) or 1e-8 (m = 32, C5's) with the
    oracle's W: the FP64 tolerance holds in truth, fewer inner iterations than plain
    refinement, and x within kappa(A)(tol + 1e-12) of the oracle's tol-1e-12 solution."""
    m, p, ic, aux, x1, b2 = wide_w
    tol = 1e-10 if m == 24 else 1e-8
    S = refine_solver(p, sample_cap=0, resume_direction=resume, inner_tol=inner_tol)
    xp = x1.copy()
    st0, it_plain, _ = S.solve(b2, xp, tol=tol)
    S.set_W(aux.W)
    S.set_mode(mode)
    x = x1.copy()
    st, it, rr = S.solve(b2, x, tol=tol)
    assert st0 == esd.OK and st == esd.OK
    assert true_relres(p, x, b2) <= 1.01 * tol
    assert it < it_plain, (it, it_plain)
    ref = oracle.System(p, ic, mode, aux).solve(b2, x1, tol=1e-12)["x"]
    assert rel(x, ref) <= kappa(p) * (tol + 1e-12)


# ---------------------------------------------------------------- rank and failure paths

def test_rank_deficient_samples_take_svqb():
    """A diagonal matrix and a right-hand side with 3 nonzero entries: every iterate lies in a
    3-dimensional space, but finite-precision CG takes 5 iterations and stores 4 samples.
    The rank rule keeps m-bar = 3 directions (Eq. ekd), built by SVQB plus one CholeskyQR
    pass; W spans the oracle's W from the same samples, and E matches."""
    n = 64
    d = np.linspace(1.0, 2.0, n)
    idx = [3, 17, 40]
    d[idx] = [1.0, 1e4, 1e8]
    p = wl.csr_of_dense(np.diag(d), ncolours=1)
    b = np.zeros(n)
    b[idx] = [1.0, 0.7, 0.3]
    A = esd.Matrix.from_problem(p)
    S = esd.Solver(A, precond=esd.PRECOND_NONE, maxit_cap=100, sample_cap=8)
    x = np.zeros(n)
    st, it, rr = S.solve(b, x, tol=1e-14, maxit=100, sample_m=8)
    samples, slot_iter = S.samples(8)
    filled = int((slot_iter > 0).sum())
    assert st == esd.OK and filled > 3, (it, slot_iter)
    m = S.sample_and_build_W()
    aux, info = oracle.build_w(p, x, samples, slot_iter)
    assert m == info["mbar"] == 3 < filled
    W, AW, E = S.get_W()
    np.testing.assert_allclose(W.T @ W, np.eye(3), atol=1e-12)
    assert np.linalg.norm(W @ (W.T @ aux.W) - aux.W) <= 1e-10 * np.linalg.norm(aux.W)
    assert np.abs(W[np.setdiff1d(np.arange(n), idx)]).max() == 0.0
    np.testing.assert_allclose(np.sort(S.ritz_values()), np.sort(aux.ritz), rtol=1e-10)


def test_no_sample_is_a_rank_error():
    """A solve that stops before its first sample (b = 0: no iteration) leaves nothing to
    build W from: ESD_ERR_RANK, and the solver keeps working."""
    p = wl.config_c1()
    A = esd.Matrix.from_problem(p)
    A.factor_ic0()
    S = esd.Solver(A, sample_cap=8)
    x = np.zeros(p.n)
    st, it, rr = S.solve(np.zeros(p.n), x, tol=1e-8, sample_m=8)
    assert st == esd.OK and it == 0
    with pytest.raises(esd.EsdError) as e:
        S.sample_and_build_W()
    assert e.value.code == esd.ERR_RANK
    st, it, rr = S.solve(p.source, x, tol=1e-8)
    assert st == esd.OK and rr <= 1e-8


def test_nan_rhs_is_a_breakdown():
    """NaN in b: the device loop stops at once with ESD_ERR_BREAKDOWN (the oracle, which has
    no such check, ends with a NaN residual and no iteration); the solver then solves the
    next system normally."""
    p = wl.small_3d(9, seed=11)
    A = esd.Matrix.from_problem(p)
    A.factor_ic0()
    S = esd.Solver(A, sample_cap=0)
    b = p.source.copy()
    b[5] = np.nan
    x = np.zeros(p.n)
    with pytest.raises(esd.EsdError) as e:
        S.solve(b, x, tol=1e-8)
    assert e.value.code == esd.ERR_BREAKDOWN
    out = oracle.System(p, oracle.IC0(p)).solve(b, tol=1e-8, history=False)
    assert out["iters"] == 0 and not np.isfinite(out["relres"])
    x = np.zeros(p.n)
    st, it, rr = S.solve(p.source, x, tol=1e-8)
    assert st == esd.OK and rr <= 1e-8


def test_indefinite_matrix_is_a_breakdown():
    """A symmetric indefinite matrix without a preconditioner: (p, Ap) < 0 in the first
    iteration, ESD_ERR_BREAKDOWN on both sides."""
    a = np.diag([1.0, -1.0, 2.0, 3.0])
    p = wl.csr_of_dense(a, ncolours=1)
    b = np.array([1.0, 2.0, 0.0, 0.0])
    A = esd.Matrix.from_problem(p)
    S = esd.Solver(A, precond=esd.PRECOND_NONE, maxit_cap=20, sample_cap=0)
    with pytest.raises(esd.EsdError) as e:
        S.solve(b, np.zeros(4), tol=1e-8, maxit=20)
    assert e.value.code == esd.ERR_BREAKDOWN
    assert oracle.System(p, None).solve(b, tol=1e-8, maxit=20, history=False)["status"] == oracle.ERR_BREAKDOWN


def test_singular_galerkin_matrix_is_refused():
    """A W with a zero column makes E = W^T A W singular: ESD_ERR_CHOL_E, no W is installed
    (deflation stays refused), and a proper W is accepted afterwards."""
    p = wl.config_c1()
    A = esd.Matrix.from_problem(p)
    A.factor_ic0()
    S = esd.Solver(A, sample_cap=0)
    W = np.asfortranarray(np.linalg.qr(np.random.default_rng(3).standard_normal((p.n, 4)))[0])
    Wz = W.copy(order="F")
    Wz[:, 2] = 0.0
    with pytest.raises(esd.EsdError) as e:
        S.set_W(Wz)
    assert e.value.code == esd.ERR_CHOL_E
    with pytest.raises(esd.EsdError) as e:
        S.set_mode(esd.DEFLATION)
    assert e.value.code == esd.ERR_STATE
    S.set_W(W)
    S.set_mode(esd.DEFLATION)
    x = np.zeros(p.n)
    st, it, rr = S.solve(p.source, x, tol=1e-8)
    assert st == esd.OK


def test_ic0_shift_matches_oracle():
    """An SPD matrix whose IC(0) meets a non-positive pivot: both sides retry with
    s = 1e-3, 2e-3, 4e-3 and succeed at s = 8e-3 on A + s diag(A); the shifted factor's
    application agrees to 1e-12, and ICCG with it to +-1 iteration and 1e-10."""
    p = wl.ic0_breakdown_spd()
    ic = oracle.IC0(p)
    assert ic.shift == pytest.approx(8e-3)
    A = esd.Matrix.from_problem(p)
    with pytest.raises(esd.EsdError) as e:
        A.factor_ic0(max_tries=4)
    assert e.value.code == esd.ERR_NOT_SPD
    shift = A.factor_ic0()
    assert shift == ic.shift
    r = np.random.default_rng(8).standard_normal(p.n)
    z = np.zeros(p.n)
    A.apply_ic(r, z)
    assert rel(z, ic.apply(r)) <= 1e-12
    S = esd.Solver(A, sample_cap=0)
    x = np.zeros(p.n)
    st, it, rr = S.solve(r, x, tol=1e-10)
    out = oracle.System(p, ic).solve(r, tol=1e-10)
    assert st == esd.OK and abs(it - out["iters"]) <= 1
    assert rel(x, out["x"]) <= 1e-10


# ---------------------------------------------------------------- full-size solutions

@pytest.fixture(scope="module")
def c2_oracle_w():
    """The oracle's system 1 of the 128^3 sequence with m = 16 samples, its W, and system 2."""
    p = wl.config_c2()
    ic = oracle.IC0(p)
    b1 = p.source  # x_0 = 0: b_1 = s
    o1 = oracle.System(p, ic).solve(b1, tol=1e-8, sample_m=16, history=False)
    aux, info = oracle.build_w(p, o1["x"], o1["samples"], o1["sample_iter"])
    b2 = o1["x"] / p.dt + p.source
    return p, ic, aux, o1["x"], b2


@pytest.mark.slow
@pytest.mark.parametrize("mode", [esd.DEFLATION, esd.SUBSPACE_CORRECTION])
def test_full_size_128cube_accelerated_solution(c2_oracle_w, mode):
    """System 2 of the 128^3 sequence (2.1M rows) in deflation and SC with the oracle's x_1
    and W, in the benchmark's launch configuration: iterations +-1, solution 1e-10."""
    p, ic, aux, x1, b2 = c2_oracle_w
    A = esd.Matrix.from_problem(p)
    A.factor_ic0()
    S = esd.Solver(A, sample_cap=0)
    S.set_W(aux.W)
    S.set_mode(mode)
    x = dev(x1.copy())
    st, it, rr = S.solve(dev(b2), x, tol=1e-8)
    out = oracle.System(p, ic, mode, aux).solve(b2, x1, tol=1e-8, history=False)
    assert st == esd.OK and abs(it - out["iters"]) <= 1, (it, out["iters"])
    assert rel(x, out["x"]) <= 1e-10
    assert S.true_relres() <= 1.05e-8
