"""The power method of the condition estimate (Algorithm PCG-con, Section 5.4) on the GPU
against the oracle, through the C ABI (GPU only).

  vector         after k CG iterations the power vector is the oracle's v_k (k steps of
                 v <- A v / ||A v|| from the same seeded start) to 1e-10, and
                 lambda_max = (v_k, A v_k) agrees to 1e-12 (summation order only);
  fused product  running the power method changes nothing in the solve: iterations,
                 alpha history and x are bit-identical with and without it;
  kappa          the paper's kappa = lambda_max / (smallest Ritz value of the sampled
                 errors) equals the oracle's from the same samples to 1e-10, and the
                 oracle's own run of Algorithm PCG-con to 1e-6;
  state          the vector carries over across solves (plain and SC), deflation and the
                 FP32 refinement form are refused, a zero start vector is rejected.
"""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def start_vector(n, seed):
    """The paper's unit random start vector, drawn by the shared seeded generator."""
    return np.random.default_rng(seed).standard_normal(n)


PROBLEMS = {
    "fv7_9cube_ragged": lambda: wl.small_3d(9, seed=11, dt=np.inf),
    "c1_64x64_redblack": lambda: wl.config_c1(),
    "lap2d_12": lambda: wl.laplacian_2d(12),
}


@pytest.mark.parametrize("name", sorted(PROBLEMS))
@pytest.mark.parametrize("precond", [esd.PRECOND_IC0, esd.PRECOND_NONE])
def test_power_vector_matches_oracle(name, precond):
    p = PROBLEMS[name]()
    A = esd.Matrix.from_problem(p)
    if precond == esd.PRECOND_IC0:
        A.factor_ic0()
    S = esd.Solver(A, precond=precond, sample_cap=8)
    v0 = start_vector(p.n, 21)
    S.power_start(dev(v0))
    b = p.source if p.source is not None else wl.random_rhs(p.n, 27)
    x = torch.zeros(p.n, dtype=torch.float64, device=DEV)
    st, it, _ = S.solve(dev(b), x, tol=1e-10, maxit=3000)
    assert st == esd.OK
    lam, k, v = S.power_estimate(vector=True)
    assert k == it
    lam_o, v_o = oracle.power_method(p, v0, k)
    assert abs(lam - lam_o) <= 1e-12 * abs(lam_o)
    assert np.abs(v - v_o).max() <= 1e-10
    assert abs(np.linalg.norm(v) - 1.0) <= 1e-14


def test_power_method_leaves_the_solve_unchanged():
    p = wl.small_3d(9, seed=11)
    A = esd.Matrix.from_problem(p)
    A.factor_ic0()
    S = esd.Solver(A, sample_cap=8)
    b = dev(p.source)
    runs = []
    for on in (False, True):
        S.power_start(dev(start_vector(p.n, 22)) if on else None)
        x = torch.zeros(p.n, dtype=torch.float64, device=DEV)
        st, it, rr = S.solve(b, x, tol=1e-10, sample_m=8)
        a, bh = S.history()
        runs.append((it, rr, x.cpu().numpy(), a, bh, S.samples(8)[1]))
    (i0, r0, x0, a0, b0, s0), (i1, r1, x1, a1, b1, s1) = runs
    assert i0 == i1 and r0 == r1
    assert np.array_equal(x0, x1) and np.array_equal(a0, a1) and np.array_equal(b0, b1)
    assert np.array_equal(s0, s1)


@pytest.mark.parametrize("precond", [esd.PRECOND_NONE, esd.PRECOND_IC0])
def test_paper_kappa_matches_oracle(precond):
    """Algorithm PCG-con end to end: PCG with m = 12 samples and the power method, then the
    smallest Ritz value of the sampled errors; kappa = lambda_max / lambda_min."""
    p = wl.small_3d(6, seed=4, dt=np.inf)
    A = esd.Matrix.from_problem(p)
    if precond == esd.PRECOND_IC0:
        A.factor_ic0()
    S = esd.Solver(A, precond=precond, sample_cap=12)
    v0 = start_vector(p.n, 13)
    S.power_start(v0)
    x = np.zeros(p.n)
    st, it, _ = S.solve(p.source, x, tol=1e-10, maxit=2000, sample_m=12)
    assert st == esd.OK
    samples, slot_iter = S.samples(12)
    S.sample_and_build_W()
    lmax, lmin, kappa = S.paper_cond_estimate()
    # the same samples through the oracle's W construction; the oracle's power method
    aux, info = oracle.build_w(p, x, samples, slot_iter)
    lam_o, _ = oracle.power_method(p, v0, it)
    assert abs(lmax - lam_o) <= 1e-12 * lam_o
    assert abs(lmin - info["ritz"][0]) <= 1e-10 * info["ritz"][0]
    assert abs(kappa - lam_o / info["ritz"][0]) <= 1e-10 * kappa
    # the oracle's own run of the algorithm (its own trajectory)
    est = oracle.pcg_cond_estimate(p, p.source, v0, m=12, tol=1e-10, maxit=2000,
                                   precond=precond == esd.PRECOND_IC0)
    if est["iters"] == it:
        assert abs(kappa - est["kappa"]) <= 1e-6 * est["kappa"]
    ev = np.linalg.eigvalsh(p.scipy().toarray())
    assert kappa <= ev[-1] / ev[0] * (1 + 1e-10)


def test_power_vector_carries_over_solves_and_sc_mode():
    p = wl.config_c1()
    A = esd.Matrix.from_problem(p)
    A.factor_ic0()
    S = esd.Solver(A, sample_cap=8)
    v0 = start_vector(p.n, 23)
    S.power_start(v0)
    x = np.zeros(p.n)
    st, it1, _ = S.solve(p.source, x, tol=1e-8, sample_m=8)
    S.sample_and_build_W()
    S.set_mode(esd.SUBSPACE_CORRECTION)
    x2 = np.zeros(p.n)
    st, it2, _ = S.solve(p.source, x2, tol=1e-8)
    assert st == esd.OK
    lam, k = S.power_estimate()
    assert k == it1 + it2
    lam_o, _ = oracle.power_method(p, v0, k)
    assert abs(lam - lam_o) <= 1e-12 * lam_o
    # a new start resets the count
    S.power_start(v0)
    assert S.power_estimate()[1] == 0
    lam0, _ = oracle.power_method(p, v0, 0)
    assert abs(S.power_estimate()[0] - lam0) <= 1e-12 * lam0


def test_power_method_state_errors():
    p = wl.config_c1()
    A = esd.Matrix.from_problem(p)
    A.factor_ic0()
    S = esd.Solver(A, sample_cap=8)
    with pytest.raises(esd.EsdError) as e:
        S.power_estimate()
    assert e.value.code == esd.ERR_STATE
    with pytest.raises(esd.EsdError) as e:
        S.power_start(np.zeros(p.n))
    assert e.value.code == esd.ERR_INVALID
    S.power_start(start_vector(p.n, 24))
    x = np.zeros(p.n)
    S.solve(p.source, x, tol=1e-8, sample_m=8)
    S.sample_and_build_W()
    S.set_mode(esd.DEFLATION)
    with pytest.raises(esd.EsdError) as e:
        S.solve(p.source, np.zeros(p.n), tol=1e-8)
    assert e.value.code == esd.ERR_STATE
    S.power_start(None)  # stopped: deflation runs again
    st, it, _ = S.solve(p.source, np.zeros(p.n), tol=1e-8)
    assert st == esd.OK
    S32 = esd.Solver(A, precision=esd.FP32_REFINE, sample_cap=8)
    with pytest.raises(esd.EsdError) as e:
        S32.power_start(start_vector(p.n, 25))
    assert e.value.code == esd.ERR_STATE


def test_full_size_128cube_power_method():
    """The 128^3 7-point workload in the benchmark's launch configuration: the first ICCG
    solve with the power method fused into its SpMV, against the oracle's power method for
    the same number of steps."""
    p = wl.config_c2()
    A = esd.Matrix.from_problem(p)
    A.factor_ic0()
    S = esd.Solver(A, sample_cap=16)
    v0 = start_vector(p.n, 26)
    S.power_start(dev(v0))
    x = torch.zeros(p.n, dtype=torch.float64, device=DEV)
    st, it, _ = S.solve(dev(p.source), x, tol=1e-8, sample_m=16)
    assert st == esd.OK
    lam, k, v = S.power_estimate(vector=True)
    assert k == it
    lam_o, v_o = oracle.power_method(p, v0, k)
    assert abs(lam - lam_o) <= 1e-12 * lam_o
    assert np.abs(v - v_o).max() <= 1e-10
