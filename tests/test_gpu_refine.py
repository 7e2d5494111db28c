"""The FP32-inner / FP64-refinement form against the FP64 oracle (GPU only).

The refinement form solves A d = r in FP32 (matrix, IC(0) factor, W and AW in FP32; E^{-1}
in FP64) inside an FP64 loop x += d, r = b - A x, either restarting CG at every step or
resuming it (residual replacement). What can be compared, and how:
  first inner solve  the FP32 PCG / DPCG / SC-PCG run is the oracle's FP64 run of the same
                     system rounded to FP32: its CG coefficients agree to FP32 accuracy over
                     the first iterations and its iteration count to max(2, 5%);
  refined solution   the FP64 stopping test ||b - A x|| <= tol ||b|| holds when recomputed
                     here, and x differs from the oracle's tol-1e-12 solution by no more
                     than kappa(A) (tol + 1e-12), the bound the residual gives;
  resumed run        one CG run in FP32 arithmetic: FP32 rounding delays convergence (up to
                     ~50% more iterations on the 64 x 64 case), so its count is only bounded,
                     by twice the oracle's FP64 count plus 10, which a stalled run exceeds;
  sampling           the slots follow method A's schedule, bit-exact, for the length of the
                     sampled run (the first inner solve, or the whole resumed run); W built
                     from them is orthonormal and E = W^T A W.
"""
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
INNER_TOL = 1e-4

def dense_spd():
    """A general SPD matrix (no M-matrix structure, rows that do not sum to a small value):
    the difference-form FP32 product must still equal A v."""
    a = wl.random_spd_dense(np.geomspace(1.0, 1e3, 40), seed=21)
    p = wl.csr_of_dense(a, ncolours=40)  # dense: one row per colour, 40 colour levels
    p.source = np.random.default_rng(5).standard_normal(40)
    return p


PROBLEMS = {
    "c1_64x64_redblack": lambda: wl.config_c1(),
    "fv7_20cube": lambda: wl.small_3d(20, seed=12, count=3, rmin=2, rmax=3, value=1e4),
    "dense_spd_40": dense_spd,
}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def rel(a, b):
    a = a.cpu().numpy() if hasattr(a, "cpu") else a
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def kappa(p):
    """Spectral condition number of A (Lanczos for the largest, shift-invert for the smallest)."""
    A = p.scipy().tocsc()
    lmax = spla.eigsh(A, k=1, which="LA", return_eigenvectors=False)[0]
    lmin = spla.eigsh(A, k=1, sigma=0.0, which="LM", return_eigenvectors=False)[0]
    return lmax / lmin


def rhs_of(p):
    return p.source if p.source is not None else np.random.default_rng(4).uniform(size=p.n)


def true_relres(p, x, b):
    x = x.cpu().numpy() if hasattr(x, "cpu") else x
    return np.linalg.norm(b - p.scipy() @ x) / np.linalg.norm(b)


def residual_rounding_bound(p, x, b):
    """How far two FP64 evaluations of ||b - A x|| / ||b||, summed in different orders, may
    lie apart: component i of b - A x is a sum of k = (entries of row i) + 1 terms, so each
    evaluation carries at most gamma_k (|b| + |A||x|)_i of rounding error (Higham, Accuracy and
    Stability of Numerical Algorithms, 2nd ed., Sec. 3.5), and the two differ by at most twice
    that in norm."""
    x = x.cpu().numpy() if hasattr(x, "cpu") else x
    k = int(np.diff(p.rowptr).max()) + 1
    u = np.finfo(np.float64).eps / 2
    gamma = k * u / (1 - k * u)
    absA = abs(p.scipy())
    return 2 * gamma * np.linalg.norm(np.abs(b) + absA @ np.abs(x)) / np.linalg.norm(b)


@pytest.fixture(scope="module", params=sorted(PROBLEMS))
def problem(request):
    p = PROBLEMS[request.param]()
    return request.param, p, kappa(p)


def refine_solver(p, **kw):
    A = esd.Matrix.from_problem(p)
    A.factor_ic0()
    kw.setdefault("inner_tol", INNER_TOL)
    return esd.Solver(A, precision=esd.FP32_REFINE, **kw)


def count_slack(k):
    return max(2, int(np.ceil(0.05 * k)))


def test_first_inner_solve_is_the_fp64_krylov_run(problem):
    """One refinement step (max_outer = 1): the FP32 run against the oracle's FP64 ICCG at the
    inner tolerance, from x = 0."""
    name, p, _ = problem
    S = refine_solver(p, sample_cap=0, max_outer=1)
    b = rhs_of(p)
    x = torch.zeros(p.n, dtype=torch.float64, device=DEV)
    st, it, rr = S.solve(dev(b), x, tol=1e-12)
    info = S.last_solve_info()
    out = oracle.System(p, oracle.IC0(p)).solve(b, tol=INNER_TOL)
    assert st == esd.ERR_MAXIT and info["outer_steps"] == 1 and info["first_inner"] == it
    assert abs(it - out["iters"]) <= count_slack(out["iters"]), (it, out["iters"])
    a, bb = S.history()
    k = min(it, out["iters"], 10)
    np.testing.assert_allclose(a[:k], out["alpha"][:k], rtol=2e-4)
    np.testing.assert_allclose(bb[:k - 1], out["beta"][:k - 1], rtol=2e-4)
    # the step's FP64 x is the FP32 inner solution; its true residual is what FP32 allows
    assert rel(x, out["x"]) <= 1e-3
    assert true_relres(p, x, b) <= 1e-2


@pytest.mark.parametrize("resume,inner_tol", [(1, 0.3), (1, 1e-2), (0, 1e-4)])
@pytest.mark.parametrize("tol", [1e-8, 1e-10])
def test_refinement_reaches_fp64_tolerance(problem, tol, resume, inner_tol):
    name, p, kap = problem
    S = refine_solver(p, sample_cap=0, resume_direction=resume, inner_tol=inner_tol)
    b = rhs_of(p)
    x = np.zeros(p.n)
    st, it, rr = S.solve(b, x, tol=tol)
    info = S.last_solve_info()
    assert st == esd.OK and rr <= tol
    assert info["outer_steps"] >= 2 and info["iters"] == it
    if resume:
        k64 = oracle.System(p, oracle.IC0(p)).solve(b, tol=tol, history=False)["iters"]
        assert it <= 2 * k64 + 10, (it, k64)
    assert true_relres(p, x, b) <= 1.01 * tol + 1e-13
    assert abs(S.true_relres() - true_relres(p, x, b)) <= 1e-3 * tol + residual_rounding_bound(p, x, b)
    ref = oracle.System(p, oracle.IC0(p)).solve(b, tol=1e-12)["x"]
    assert rel(x, ref) <= kap * (tol + 1e-12)


@pytest.fixture(scope="module")
def c1_oracle_w():
    p = wl.config_c1()
    ic = oracle.IC0(p)
    o1 = oracle.System(p, ic).solve(p.source, tol=1e-8, sample_m=8)
    aux, info = oracle.build_w(p, o1["x"], o1["samples"], o1["sample_iter"])
    b2 = o1["x"] / p.dt + p.source
    return p, ic, aux, o1["x"], b2


@pytest.mark.parametrize("mode", [esd.DEFLATION, esd.SUBSPACE_CORRECTION])
def test_accelerated_first_inner_matches_oracle(c1_oracle_w, mode):
    """One step of deflated (SC) FP32 inner PCG with the oracle's W on system 2's residual
    equation A d = b2 - A x1, against the oracle's FP64 run of the same equation."""
    p, ic, aux, x1, b2 = c1_oracle_w
    S = refine_solver(p, sample_cap=0, max_outer=1)
    S.set_W(aux.W)
    S.set_mode(mode)
    r0 = b2 - p.scipy() @ x1
    d = torch.zeros(p.n, dtype=torch.float64, device=DEV)
    st, it, rr = S.solve(dev(r0), d, tol=1e-12)
    out = oracle.System(p, ic, mode, aux).solve(r0, np.zeros(p.n), tol=INNER_TOL)
    assert st == esd.ERR_MAXIT and S.last_solve_info()["outer_steps"] == 1
    assert abs(it - out["iters"]) <= count_slack(out["iters"]), (it, out["iters"])
    a, bb = S.history()
    k = min(it, out["iters"], 8)
    np.testing.assert_allclose(a[:k], out["alpha"][:k], rtol=2e-4)
    np.testing.assert_allclose(bb[:k - 1], out["beta"][:k - 1], rtol=2e-4)


@pytest.mark.parametrize("resume,inner_tol", [(1, 0.3), (0, 1e-4)])
@pytest.mark.parametrize("mode", [esd.DEFLATION, esd.SUBSPACE_CORRECTION])
def test_accelerated_refinement_converges(c1_oracle_w, mode, resume, inner_tol):
    """System 2 to 1e-8 in the refinement form with the oracle's W: FP64 tolerance met, the
    inner work below plain refinement's."""
    p, ic, aux, x1, b2 = c1_oracle_w
    kap = kappa(p)
    S = refine_solver(p, sample_cap=0, resume_direction=resume, inner_tol=inner_tol)
    x = x1.copy()
    st0, it_plain, _ = S.solve(b2, x, tol=1e-8)
    S.set_W(aux.W)
    S.set_mode(mode)
    x = x1.copy()
    st, it, rr = S.solve(b2, x, tol=1e-8)
    assert st0 == esd.OK and st == esd.OK
    assert true_relres(p, x, b2) <= 1.01e-8
    assert it < it_plain, (it, it_plain)
    ref = oracle.System(p, ic, mode, aux).solve(b2, x1, tol=1e-12)["x"]
    assert rel(x, ref) <= kap * (1e-8 + 1e-12)


@pytest.mark.parametrize("resume,inner_tol", [(1, 0.3), (0, 1e-4)])
def test_sampling_in_refinement(resume, inner_tol):
    """Method A samples the first inner solve (restart) or the whole run (resume): the slot
    schedule is the one the oracle gives for that length; W from the samples is orthonormal,
    AW = A W, E = W^T A W, and it deflates system 2 (fewer inner iterations than plain)."""
    p = wl.config_c1()
    S = refine_solver(p, sample_cap=8, resume_direction=resume, inner_tol=inner_tol)
    x = torch.zeros(p.n, dtype=torch.float64, device=DEV)
    st, it, rr = S.solve(dev(p.source), x, tol=1e-8, sample_m=8)
    info = S.last_solve_info()
    assert st == esd.OK and info["outer_steps"] >= 2
    samples, slot_iter = S.samples(8)
    k1 = it if resume else info["first_inner"]
    lmax = oracle.default_lmax(8, S.maxit_cap)
    assert slot_iter.tolist() == oracle.sampling_a_schedule(8, k1, lmax).tolist()
    assert np.all(np.isfinite(samples))
    m = S.sample_and_build_W()
    assert 1 <= m <= 8
    W, AW, E = S.get_W()
    # the refinement form keeps W rounded to FP32 (and AW, E of exactly that W)
    np.testing.assert_array_equal(W, W.astype(np.float32).astype(np.float64))
    np.testing.assert_allclose(W.T @ W, np.eye(m), atol=1e-6)
    np.testing.assert_allclose(AW, p.scipy() @ W, rtol=1e-12, atol=1e-12 * np.abs(AW).max())
    np.testing.assert_allclose(E, W.T @ AW, rtol=1e-10, atol=1e-12 * np.abs(E).max())
    b2 = x.cpu().numpy() / p.dt + p.source
    x1 = x.cpu().numpy()
    S.set_mode(esd.PLAIN)
    xp = x1.copy()
    S.solve(b2, xp, tol=1e-8)
    it_plain = S.last_solve_info()["iters"]
    S.set_mode(esd.DEFLATION)
    xd = x1.copy()
    st, it_defl, _ = S.solve(b2, xd, tol=1e-8)
    assert st == esd.OK and true_relres(p, xd, b2) <= 1.01e-8
    assert it_defl < it_plain, (it_defl, it_plain)


def test_refinement_zero_rhs_and_step_limit():
    p = wl.config_c1()
    S = refine_solver(p, sample_cap=0, max_outer=1)
    x = np.ones(p.n)
    st, it, rr = S.solve(np.zeros(p.n), x, tol=1e-8)
    assert st == esd.OK and it == 0 and np.all(x == 0.0)
    assert S.last_solve_info()["outer_steps"] == 0
    x = np.zeros(p.n)
    st, it, rr = S.solve(p.source, x, tol=1e-10)
    assert st == esd.ERR_MAXIT and rr > 1e-10
    assert S.last_solve_info()["outer_steps"] == 1


def test_refinement_parameters_checked():
    p = wl.config_c1()
    A = esd.Matrix.from_problem(p)
    A.factor_ic0()
    for kw in ({"inner_tol": 0.0}, {"inner_tol": 1.5}, {"max_outer": 0}):
        with pytest.raises(esd.EsdError):
            esd.Solver(A, precision=esd.FP32_REFINE, **kw)
