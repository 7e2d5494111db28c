"""The FP32 storage of the refinement form's staged kernels (GPU only): the column-free copy
(slot bases + 4-byte values) where a matrix's slices admit one, the (value, column) pairs
where they do not, and the oracle's FP64 Krylov run through either.

A multicolour 7-point ordering with rows in natural order inside each colour gives every
32-row slice at most 7 distinct (column - lane) values, so A, L and U get the copy. The same
operator with the rows of each colour shuffled (still a valid colouring: rows of one colour
are uncoupled, so IC(0) is the same factor, permuted) scatters the neighbours of a slice and
keeps the pairs. Both must run the oracle's iteration: the FP32 CG coefficients of the first
inner solve agree with the oracle's FP64 run to FP32 accuracy, the count within max(2, 5%),
and the refined solution meets its tolerance.
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


@pytest.fixture(scope="module")
def problems():
    p = wl.small_3d(24, seed=12, count=3, rmin=2, rmax=3, value=1e4)
    return {"natural": (p, True), "shuffled": (wl.shuffle_within_colours(p, 7), False)}


@pytest.mark.parametrize("which", ["natural", "shuffled"])
def test_layout_flags(problems, which):
    p, column_free = problems[which]
    A = esd.Matrix.from_problem(p)
    lay = A.layout()
    assert lay["column_free"] == [column_free] * 3
    assert lay["slices"] == sum((int(p.colour_ptr[c + 1] - p.colour_ptr[c]) + 31) // 32
                                for c in range(p.ncolours))
    if column_free:
        # every entry has a slot (absent neighbours hold zeros), at most 8 slots per slice; A's
        # copy has none for the diagonal (the difference-form product multiplies it by 0)
        nnz_lower = (p.nnz - p.n) // 2
        assert p.nnz - p.n <= lay["slot_entries"][0] <= 8 * 32 * lay["slices"]
        for part in (1, 2):
            assert nnz_lower <= lay["slot_entries"][part] <= 8 * 32 * lay["slices"]
    else:
        assert lay["slot_entries"] == [0, 0, 0]


@pytest.mark.parametrize("which", ["natural", "shuffled"])
def test_fp32_run_matches_the_oracle_in_either_layout(problems, which):
    p, _ = problems[which]
    b = p.source
    A = esd.Matrix.from_problem(p)
    A.factor_ic0()
    # one refinement step: the FP32 inner run from x = 0 to 1e-4
    S = esd.Solver(A, precision=esd.FP32_REFINE, sample_cap=0, max_outer=1, inner_tol=1e-4)
    x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    st, it, _ = S.solve(torch.from_numpy(b).cuda(), x, tol=1e-12)
    out = oracle.System(p, oracle.IC0(p)).solve(b, tol=1e-4)
    assert st == esd.ERR_MAXIT
    assert abs(it - out["iters"]) <= max(2, int(np.ceil(0.05 * out["iters"]))), (it, out["iters"])
    a, bb = S.history()
    k = min(it, out["iters"], 10)
    np.testing.assert_allclose(a[:k], out["alpha"][:k], rtol=2e-4)
    np.testing.assert_allclose(bb[:k - 1], out["beta"][:k - 1], rtol=2e-4)
    # refined to 1e-10 in FP64
    S2 = esd.Solver(A, precision=esd.FP32_REFINE, sample_cap=0, inner_tol=0.1)
    x2 = np.zeros(p.n)
    st, it, rr = S2.solve(b, x2, tol=1e-10)
    assert st == esd.OK and rr <= 1e-10
    assert np.linalg.norm(b - p.scipy() @ x2) / np.linalg.norm(b) <= 1.01e-10
