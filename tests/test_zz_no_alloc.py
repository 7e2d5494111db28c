"""The allocation-free condition estimate, called through the C ABI (GPU only).

``esd_lanczos_extremes_noalloc`` is for callers that cannot call cudaMalloc: code that has
handed all of the device's memory to another allocator (a framework's caching pool), or a
time-stepping loop that must not stall on the device-wide synchronisation an allocation
may bring. It reads CG coefficients from the caller's device arrays and keeps its scratch
in one static device array, so nothing is allocated on any call.

Checks, each on two calls in a row (the array keeps the previous call's contents):

- it returns what ``esd_estimate_cond`` returns for the same solve (1e-12 relative);
- on plain CG of the 1D Laplacian tridiag(-1, 2, -1) it meets the closed-form extremes
  2 - 2cos(pi/(n+1)) and 2 - 2cos(n pi/(n+1)), and it matches the oracle's estimate from the
  oracle's own CG run;
- at the largest size it accepts, coefficients whose Lanczos matrix is exactly the k x k
  1D Laplacian give that matrix's closed-form extremes;
- sizes beyond the static array and arguments that are not device memory are refused
  before any launch.

This file is collected last on purpose and also passes when run alone.
"""
import ctypes as C
import math

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


def _noalloc_twice(alpha, beta):
    """Two calls in a row on the same device arrays; returns both results."""
    k = len(alpha)
    a_d = torch.from_numpy(np.ascontiguousarray(alpha, dtype=np.float64)).to(DEV)
    b_d = torch.from_numpy(np.ascontiguousarray(beta[: k - 1] if k > 1 else np.zeros(1), dtype=np.float64)).to(DEV)
    out = torch.empty(3, dtype=torch.float64, device=DEV)
    got = []
    for _ in range(2):
        out.fill_(float("nan"))
        esd.esd_lanczos_extremes_noalloc(a_d, b_d, k, out)
        torch.cuda.synchronize()
        got.append(out.cpu().numpy().copy())
    return got


def test_noalloc_estimate_matches_existing_entry_point():
    for prob, precond in ((wl.config_c1(), esd.PRECOND_IC0), (wl.laplacian_1d(50), esd.PRECOND_NONE)):
        A = esd.Matrix.from_problem(prob)
        if precond == esd.PRECOND_IC0:
            A.factor_ic0()
        S = esd.Solver(A, precond=precond, maxit_cap=2000, sample_cap=0)
        b = prob.source if prob.source is not None else np.random.default_rng(0).standard_normal(prob.n)
        S.solve(b, np.zeros(prob.n), tol=1e-10, maxit=2000)
        lmin, lmax, kappa, _ = S.estimate_cond()
        alpha, beta = S.history()
        for got in _noalloc_twice(alpha, beta):
            np.testing.assert_allclose(got, [lmin, lmax, kappa], rtol=1e-12)


def test_noalloc_laplacian_closed_form_and_oracle():
    """Plain CG on tridiag(-1, 2, -1), n = 50, random b, tol 1e-14: the Lanczos extremes are
    the matrix's own, 2 - 2cos(pi/51) and 2 - 2cos(50 pi/51). The oracle's CG run of the same
    system gives its own coefficients; both estimates must agree with the closed form and
    with each other."""
    n = 50
    prob = wl.laplacian_1d(n)
    b = np.random.default_rng(7).standard_normal(n)
    exact = (2 - 2 * math.cos(math.pi / (n + 1)), 2 - 2 * math.cos(n * math.pi / (n + 1)))
    exact = np.array([exact[0], exact[1], exact[1] / exact[0]])

    A = esd.Matrix.from_problem(prob)
    S = esd.Solver(A, precond=esd.PRECOND_NONE, maxit_cap=200, sample_cap=0)
    S.solve(b, np.zeros(n), tol=1e-14, maxit=200)
    alpha, beta = S.history()
    for got in _noalloc_twice(alpha, beta):
        np.testing.assert_allclose(got, exact, rtol=1e-8)

    ref = oracle.System(prob, None).solve(b, tol=1e-14, maxit=200)
    orc = np.array(oracle.estimate_cond(ref["alpha"], ref["beta"]))
    np.testing.assert_allclose(orc, exact, rtol=1e-8)
    for got in _noalloc_twice(ref["alpha"], ref["beta"]):
        np.testing.assert_allclose(got, orc, rtol=1e-10)


def test_noalloc_largest_size_closed_form():
    """alpha_j = (j+1)/(j+2), beta_j = alpha_j^2 make T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1}
    = 2 and T_{j,j+1} = sqrt(beta_j)/alpha_j = 1: T is the k x k 1D Laplacian, whose extremes
    are 2 - 2cos(pi/(k+1)) and 2 - 2cos(k pi/(k+1)). Run at k = ESD_NOALLOC_MAX_K, the whole
    scratch array, after a small call that leaves other values in it."""
    for k in (7, esd.NOALLOC_MAX_K):
        j = np.arange(k, dtype=np.float64)
        alpha = (j + 1) / (j + 2)
        beta = alpha[:-1] ** 2
        lo = 2 - 2 * math.cos(math.pi / (k + 1))
        hi = 2 - 2 * math.cos(k * math.pi / (k + 1))
        for got in _noalloc_twice(alpha, beta):
            # lambda_min ~ 9e-9 at the largest k: the Sturm counts resolve it to about
            # 1e-15 absolute (rounding of the diagonal 2), hence the relative 1e-6.
            np.testing.assert_allclose(got[0], lo, rtol=1e-6 if k > 1000 else 1e-10)
            np.testing.assert_allclose(got[1], hi, rtol=1e-12)
            np.testing.assert_allclose(got[2], got[1] / got[0], rtol=1e-14)


def test_noalloc_rejects_sizes_beyond_the_scratch():
    out = torch.zeros(3, dtype=torch.float64, device=DEV)
    a = torch.ones(esd.NOALLOC_MAX_K + 1, dtype=torch.float64, device=DEV)
    with pytest.raises(esd.EsdError) as e:
        esd.esd_lanczos_extremes_noalloc(a, a, esd.NOALLOC_MAX_K + 1, out)
    assert e.value.code == esd.ERR_INVALID and "scratch" in str(e.value)


def test_noalloc_rejects_memory_that_is_not_on_the_device():
    """Host arrays handed straight to the C entry point are refused with ESD_ERR_INVALID
    (no kernel is launched); the binding refuses wrong types and short tensors itself."""
    lib = esd.lib()
    host = np.ones(4)
    host_out = np.zeros(3)
    dev_a = torch.ones(4, dtype=torch.float64, device=DEV)
    dev_out = torch.zeros(3, dtype=torch.float64, device=DEV)
    hp = C.c_void_p(host.ctypes.data)
    dp, op = C.c_void_p(dev_a.data_ptr()), C.c_void_p(dev_out.data_ptr())
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for args, what in (((hp, dp, 4, op), "alpha"), ((dp, hp, 4, op), "beta"),
                       ((dp, dp, 4, C.c_void_p(host_out.ctypes.data)), "out")):
        assert lib.esd_lanczos_extremes_noalloc(*args, st) == esd.ERR_INVALID
        assert what in esd.esd_last_error()
    torch.cuda.synchronize()
    assert torch.all(dev_out == 0)

    with pytest.raises(TypeError):
        esd.esd_lanczos_extremes_noalloc(host, dev_a, 4, dev_out)
    with pytest.raises(TypeError):
        esd.esd_lanczos_extremes_noalloc(dev_a.float(), dev_a, 4, dev_out)
    with pytest.raises(ValueError):
        esd.esd_lanczos_extremes_noalloc(dev_a, dev_a, 5, dev_out)
    with pytest.raises(ValueError):
        esd.esd_lanczos_extremes_noalloc(dev_a, dev_a[:2], 4, dev_out)
    with pytest.raises(ValueError):
        esd.esd_lanczos_extremes_noalloc(dev_a, dev_a, 4, dev_out[:2])
