"""Other IC orderings on the GPU against the oracle (GPU only).

  natural order   IC(0) in wavefront order (x + y + z; the same preconditioner as natural
                  order, one launch per wavefront and sweep) against the oracle on the same
                  problem: iterations +-1, solution 1e-10, also with subspace correction;
  block-Jacobi    A in block-wavefront order preconditioned by IC(0) of its block-diagonal
                  part (esd_solver_set_precond_matrix): iterations +-1, solution 1e-10; the
                  levels come from the blocks (3b - 2 per sweep);
  refinement      the FP32 inner solves use the preconditioning matrix's FP32 factor;
  full size       natural-order ICCG on the 128^3 workload (381 wavefront launches per sweep)
                  against the oracle's count.
"""
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


def rel(a, b):
    a = a.cpu().numpy() if hasattr(a, "cpu") else a
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("N", [9, 16, 24])  # 25, 46 and 70 wavefronts (above 64: the wide adjacency)
def test_wavefront_ic0_matches_oracle(N):
    p = wl.reorder(wl.small_3d(N, seed=11), wl.wavefront_colours((N, N, N)))
    A = esd.Matrix.from_problem(p)
    info = A.info()
    assert info["ncolours"] == 3 * N - 2
    assert info["fwd_levels"] == info["bwd_levels"] == 3 * N - 2
    A.factor_ic0()
    S = esd.Solver(A, sample_cap=8)
    x = np.zeros(p.n)
    st, it, rr = S.solve(p.source, x, tol=1e-10, sample_m=8)
    ic = oracle.IC0(p)
    out = oracle.System(p, ic).solve(p.source, tol=1e-10, sample_m=8)
    assert st == esd.OK and abs(it - out["iters"]) <= 1, (it, out["iters"])
    assert rel(x, out["x"]) <= 1e-10
    # subspace correction with W from the same samples
    samples, slot_iter = S.samples(8)
    S.sample_and_build_W()
    aux, _ = oracle.build_w(p, x, samples, slot_iter)
    S.set_mode(esd.SUBSPACE_CORRECTION)
    b2 = wl.random_rhs(p.n, 3)
    x2 = np.zeros(p.n)
    st, it2, _ = S.solve(b2, x2, tol=1e-10)
    out2 = oracle.System(p, ic, oracle.SUBSPACE_CORRECTION, aux).solve(b2, tol=1e-10)
    assert st == esd.OK and abs(it2 - out2["iters"]) <= 1
    assert rel(x2, out2["x"]) <= 1e-9


@pytest.mark.parametrize("N,b", [(12, 4), (16, 8), (13, 5)])
def test_block_jacobi_ic_matches_oracle(N, b):
    shape = (N, N, N)
    p = wl.reorder(wl.small_3d(N, seed=12), wl.block_wavefront_colours(shape, b))
    Pp = wl.block_diagonal_part(p, wl.block_ids(shape, b))
    A = esd.Matrix.from_problem(p)
    A.factor_ic0()
    P = esd.Matrix.from_problem(Pp)
    assert P.info()["fwd_levels"] == 3 * b - 2  # the wavefronts of one block
    P.factor_ic0()
    S = esd.Solver(A)
    S.set_precond_matrix(P)
    x = np.zeros(p.n)
    st, it, rr = S.solve(p.source, x, tol=1e-10)
    out = oracle.System(p, oracle.IC0(Pp)).solve(p.source, tol=1e-10)
    assert st == esd.OK and abs(it - out["iters"]) <= 1, (it, out["iters"])
    assert rel(x, out["x"]) <= 1e-10
    assert np.linalg.norm(p.source - p.scipy() @ x) <= 1.01e-10 * np.linalg.norm(p.source)
    # back to A's own IC(0): the oracle's plain ICCG in the same ordering
    S.set_precond_matrix(None)
    x = np.zeros(p.n)
    st, it_a, _ = S.solve(p.source, x, tol=1e-10)
    out_a = oracle.System(p, oracle.IC0(p)).solve(p.source, tol=1e-10)
    assert abs(it_a - out_a["iters"]) <= 1


def test_refinement_with_block_jacobi():
    N, b = 16, 8
    shape = (N, N, N)
    p = wl.reorder(wl.small_3d(N, seed=13, value=1e4), wl.block_wavefront_colours(shape, b))
    Pp = wl.block_diagonal_part(p, wl.block_ids(shape, b))
    A = esd.Matrix.from_problem(p)
    A.factor_ic0()
    P = esd.Matrix.from_problem(Pp)
    P.factor_ic0()
    S = esd.Solver(A, precision=esd.FP32_REFINE)
    S.set_precond_matrix(P)
    x = np.zeros(p.n)
    st, it, rr = S.solve(p.source, x, tol=1e-10)
    assert st == esd.OK
    assert np.linalg.norm(p.source - p.scipy() @ x) <= 1.01e-10 * np.linalg.norm(p.source)
    plain = oracle.System(p, oracle.IC0(Pp)).solve(p.source, tol=1e-10, history=False)["iters"]
    assert it <= 2 * plain + 10


def test_precond_matrix_refusals():
    N = 8
    p = wl.reorder(wl.small_3d(N, seed=14), wl.wavefront_colours((N, N, N)))
    A = esd.Matrix.from_problem(p)
    A.factor_ic0()
    S = esd.Solver(A)
    other = esd.Matrix.from_problem(wl.small_3d(N, seed=14))  # multicolour: other colour_ptr
    other.factor_ic0()
    with pytest.raises(esd.EsdError) as e:
        S.set_precond_matrix(other)
    assert e.value.code == esd.ERR_INVALID
    unfactored = esd.Matrix.from_problem(p)
    with pytest.raises(esd.EsdError) as e:
        S.set_precond_matrix(unfactored)
    assert e.value.code == esd.ERR_STATE


def test_full_size_128cube_natural_order():
    """The 128^3 workload's first system with natural-order IC(0): 381 forward and 381 backward
    wavefront launches per iteration inside the solve graph, against the oracle's count."""
    base = wl.config_c2()
    p = wl.reorder(base, wl.wavefront_colours(base.shape))
    A = esd.Matrix.from_problem(p)
    assert A.info()["ncolours"] == 382
    A.factor_ic0()
    S = esd.Solver(A, sample_cap=0)
    x = torch.zeros(p.n, dtype=torch.float64, device=DEV)
    st, it, rr = S.solve(torch.from_numpy(p.source).to(DEV), x, tol=1e-8)
    out = oracle.System(p, oracle.IC0(p)).solve(p.source, tol=1e-8, history=False)
    assert st == esd.OK and abs(it - out["iters"]) <= max(1, math.ceil(0.02 * out["iters"]))
    assert rel(x, out["x"]) <= 1e-8
