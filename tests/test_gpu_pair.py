"""esd_solve_pair: two systems with one matrix solved together (GPU only).

The paired kernels stream each matrix part once for both systems and keep every system's
CG recurrence, scalars and vectors apart; each row's products are taken in the order of
the single kernels, only the dot products' partial sums cover other rows. So each system of
a pair must end as it ends alone:
  stopping test   ||b - A x|| <= tol ||b||, recomputed here in FP64 from the returned x;
  coefficients    the first CG coefficients (alpha, beta) of each system equal esd_solve's
                  to 1e-3: the runs differ only in the rounding of the FP32 sums, which a
                  row left out of a product or a dot product would exceed;
  iterations      the pair's inner total of each system within max(3, 5%) of esd_solve's
                  (25% at a contrast of 1e6, where the FP32 trajectory, its refinement
                  restarts and so its count depend on that rounding);
  solution        within kappa-free reach of the single run: both meet the same residual
                  bound, so ||A (x_pair - x_single)|| <= 2 tol ||b||;
  independence    a system that is solved already (or has b = 0) costs nothing: the other
                  runs alone, the same bits with either;
  determinism     the same pair twice (and with the solvers swapped) gives the same bits.
Layouts: the column-free FP32 copy (natural order inside the colours), the (value, column)
pairs (rows of each colour shuffled), and a ragged grid (odd N: colours and slices ragged).
"""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2203_08498_gb300 as esd  # noqa: E402

TOL = 1e-8


def _problem(which):
    if which == "natural":
        return wl.small_3d(24, seed=12, count=3, rmin=2, rmax=3, value=1e4)
    if which == "shuffled":
        return wl.shuffle_within_colours(wl.small_3d(24, seed=12, count=3, rmin=2, rmax=3, value=1e4), 7)
    return wl.small_3d(23, seed=13, count=3, rmin=2, rmax=3, value=1e6)  # ragged


SLACK = {"natural": 0.05, "shuffled": 0.05, "ragged": 0.25}  # iteration counts (see above)


@pytest.fixture(scope="module", params=["natural", "shuffled", "ragged"])
def case(request):
    p = _problem(request.param)
    A = esd.Matrix.from_problem(p)
    A.factor_ic0()
    mk = lambda: esd.Solver(A, precision=esd.FP32_REFINE, sample_cap=0, inner_tol=0.1)  # noqa: E731
    S1, S2, S3 = mk(), mk(), mk()
    rng = np.random.default_rng(3)
    b1 = p.source.copy()
    b2 = rng.uniform(-1.0, 1.0, p.n) * float(np.abs(p.source).max())
    x2 = rng.standard_normal(p.n) * 1e-3  # a warm start for the second system
    return dict(p=p, A=A, S=(S1, S2, S3), b1=b1, b2=b2, x2=x2, csr=p.scipy(), slack=SLACK[request.param])


def relres(csr, b, x):
    return np.linalg.norm(b - csr @ x) / np.linalg.norm(b)


def single(S, b, x0):
    x = x0.copy()
    st, it, rr = S.solve(b, x, TOL)
    assert st == esd.OK
    return x, it


def test_pair_meets_the_stopping_test_and_follows_the_single_runs(case):
    S1, S2, _ = case["S"]
    csr = case["csr"]
    xs1, it_s1 = single(S1, case["b1"], np.zeros(case["p"].n))
    h_s1 = S1.history()
    xs2, it_s2 = single(S2, case["b2"], case["x2"])
    h_s2 = S2.history()
    x1, x2 = np.zeros(case["p"].n), case["x2"].copy()
    st, (it1, rr1), (it2, rr2), paired = S1.solve_pair(S2, case["b1"], x1, case["b2"], x2, TOL)
    assert st == esd.OK
    for S, (a_s, b_s) in ((S1, h_s1), (S2, h_s2)):
        a, b = S.history()
        k = min(len(a), len(a_s), 8)
        np.testing.assert_allclose(a[:k], a_s[:k], rtol=1e-3)
        np.testing.assert_allclose(b[:k - 1], b_s[:k - 1], rtol=1e-3)
    # the paired loop runs while both inner runs go on: at least the shorter first inner run
    assert 0 < paired <= min(it1, it2)
    for x, b, rr in ((x1, case["b1"], rr1), (x2, case["b2"], rr2)):
        assert rr <= TOL
        assert relres(csr, b, x) <= 1.01 * TOL
    for it, it_s in ((it1, it_s1), (it2, it_s2)):
        assert abs(it - it_s) <= max(3, int(np.ceil(case["slack"] * it_s))), (it, it_s)
    for x, xs, b in ((x1, xs1, case["b1"]), (x2, xs2, case["b2"])):
        assert np.linalg.norm(csr @ (x - xs)) <= 2.02 * TOL * np.linalg.norm(b)


def test_pair_is_deterministic_and_symmetric(case):
    S1, S2, _ = case["S"]
    n = case["p"].n
    runs = []
    for swap in (False, False, True):
        x1, x2 = np.zeros(n), case["x2"].copy()
        if swap:
            st, r2, r1, pr = S2.solve_pair(S1, case["b2"], x2, case["b1"], x1, TOL)
        else:
            st, r1, r2, pr = S1.solve_pair(S2, case["b1"], x1, case["b2"], x2, TOL)
        assert st == esd.OK
        runs.append((x1, x2, r1, r2, pr))
    for x1, x2, r1, r2, pr in runs[1:]:
        assert np.array_equal(x1, runs[0][0]) and np.array_equal(x2, runs[0][1])
        assert (r1, r2, pr) == runs[0][2:]


def test_a_solved_system_leaves_the_other_unchanged(case):
    """System 2 starts at its solution (its first FP64 residual meets tol) or has b = 0:
    it takes no iteration, the paired kernels never run, and x2 comes back as it went in (0
    for b = 0); system 1 runs the same iterations, bit for bit, in both pairs."""
    S1, S2, S3 = case["S"]
    n = case["p"].n
    xs2, _ = single(S3, case["b2"], case["x2"])
    outs = []
    for b2, x2in in ((case["b2"], xs2), (np.zeros(n), case["x2"])):
        x1, x2 = np.zeros(n), x2in.copy()
        st, (it1, rr1), (it2, rr2), paired = S1.solve_pair(S2, case["b1"], x1, b2, x2, TOL)
        assert st == esd.OK and it2 == 0 and paired == 0
        if b2.any():
            assert np.array_equal(x2, x2in)
        else:
            assert not x2.any() and rr2 == 0.0
        assert relres(case["csr"], case["b1"], x1) <= 1.01 * TOL
        outs.append((x1, it1, rr1))
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1:] == outs[1][1:]


def test_pair_maxit(case):
    S1, S2, _ = case["S"]
    n = case["p"].n
    x1, x2 = np.zeros(n), case["x2"].copy()
    st, (it1, _), (it2, _), _ = S1.solve_pair(S2, case["b1"], x1, case["b2"], x2, TOL, maxit=5)
    assert st == esd.ERR_MAXIT
    assert 0 < it1 <= 5 and 0 < it2 <= 5


def test_pair_device_tensors(case):
    """Device tensors in and out (the call the time-stepping loop makes)."""
    S1, S2, _ = case["S"]
    n = case["p"].n
    b1, b2 = torch.from_numpy(case["b1"]).cuda(), torch.from_numpy(case["b2"]).cuda()
    x1, x2 = torch.zeros(n, dtype=torch.float64, device="cuda"), torch.from_numpy(case["x2"]).cuda()
    st, (it1, _), (it2, _), _ = S1.solve_pair(S2, b1, x1, b2, x2, TOL)
    assert st == esd.OK and it1 > 0 and it2 > 0
    assert relres(case["csr"], case["b1"], x1.cpu().numpy()) <= 1.01 * TOL
    assert relres(case["csr"], case["b2"], x2.cpu().numpy()) <= 1.01 * TOL


def test_pair_refusals():
    p = wl.small_3d(12, seed=12, count=1, rmin=2, rmax=3, value=1e3)
    A, B = esd.Matrix.from_problem(p), esd.Matrix.from_problem(p)
    A.factor_ic0()
    B.factor_ic0()
    mk = lambda M, **kw: esd.Solver(M, sample_cap=0, **{"precision": esd.FP32_REFINE, **kw})  # noqa: E731
    S1, S2 = mk(A), mk(A)
    b, x1, x2 = p.source, np.zeros(p.n), np.zeros(p.n)
    cases = [
        (S1, S1, esd.ERR_INVALID),  # one solver twice
        (S1, mk(B), esd.ERR_INVALID),  # another matrix
        (S1, mk(A, precision=esd.FP64), esd.ERR_STATE),  # not the refinement form
        (S1, mk(A, precond=esd.PRECOND_NONE), esd.ERR_STATE),  # not IC(0)
    ]
    for a, c, code in cases:
        with pytest.raises(esd.EsdError) as e:
            a.solve_pair(c, b, x1, b, x2, TOL)
        assert e.value.code == code, str(e.value)
    with pytest.raises(esd.EsdError) as e:
        S1.solve_pair(S2, b, x1, b, x2, -1.0)
    assert e.value.code == esd.ERR_INVALID
    st, _, _, _ = S1.solve_pair(S2, b, x1, b, x2, TOL)  # the refusals left the solvers usable
    assert st == esd.OK
