"""The allocation-free condition estimate against esd_estimate_cond (GPU only).

esd_lanczos_extremes_noalloc serves callers that cannot call cudaMalloc: it takes the CG
coefficients from caller-owned device arrays and keeps its scratch in a static device
array. Two calls in a row must each reproduce what esd_estimate_cond returns for the same
solve, within the tolerance the other GPU tests use for such values (1e-12 relative).
This file is collected last on purpose and also passes when run alone.
"""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2203_08498_gb300 as esd  # noqa: E402


def test_noalloc_estimate_matches_existing_entry_point():
    dev = torch.device("cuda:0")
    out = torch.full((3,), float("nan"), dtype=torch.float64, device=dev)
    for prob, precond in ((wl.config_c1(), esd.PRECOND_IC0), (wl.laplacian_1d(50), esd.PRECOND_NONE)):
        A = esd.Matrix.from_problem(prob)
        if precond == esd.PRECOND_IC0:
            A.factor_ic0()
        S = esd.Solver(A, precond=precond, maxit_cap=2000, sample_cap=0)
        b = prob.source if prob.source is not None else np.random.default_rng(0).standard_normal(prob.n)
        S.solve(b, np.zeros(prob.n), tol=1e-10, maxit=2000)
        lmin, lmax, kappa, _ = S.estimate_cond()
        alpha, beta = S.history()
        k = len(alpha)
        a_d = torch.from_numpy(alpha.copy()).to(dev)
        b_d = torch.from_numpy(beta.copy() if k > 1 else np.zeros(1)).to(dev)
        for call in range(2):
            out.fill_(float("nan"))
            esd.esd_lanczos_extremes_noalloc(a_d, b_d, k, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            np.testing.assert_allclose(got, [lmin, lmax, kappa], rtol=1e-12)


def test_noalloc_rejects_sizes_beyond_the_scratch():
    dev = torch.device("cuda:0")
    out = torch.zeros(3, dtype=torch.float64, device=dev)
    a = torch.ones(4, dtype=torch.float64, device=dev)
    with pytest.raises(esd.EsdError) as e:
        esd.esd_lanczos_extremes_noalloc(a, a, esd.NOALLOC_MAX_K + 1, out)
    assert e.value.code == esd.ERR_INVALID and "scratch" in str(e.value)
