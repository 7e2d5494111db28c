"""The differentiation form on the GPU against the oracle (GPU only).

  assembly       esd_fv_assemble(theta) reproduces the generator's matrix: A v agrees to
                 1e-14 (exp and the face formula may round differently by an ulp);
  chain rule     esd_fv_grad_theta equals the oracle's fv_theta_gradient on the same
                 lambda and x to 1e-12;
  autograd       dL/dtheta and dL/db of L = ||x - x_target||^2 through AdjointSolve match
                 the oracle's ICCG adjoint gradient to 1e-8 (both solves at tol 1e-13) and
                 central finite differences on 32 seeded cells in theta (step 1e-6) and 8 in
                 b, to 1e-5, with the forward and the adjoint solve deflated by the same W;
  state          solves refuse a stale factor or a W formed for other matrix values.
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
from paper_2203_08498_gb300.adjoint import FVDiffusion, fv_solve  # noqa: E402

DEV = torch.device("cuda:0")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def nat(theta_grid):
    return np.ascontiguousarray(np.asarray(theta_grid).ravel(order="F"))


def cell_row(p):
    inv = np.empty(p.n, dtype=np.int32)
    inv[p.perm] = np.arange(p.n, dtype=np.int32)
    return inv


def grid_of(p):
    d = len(p.shape)
    inv_dt = 0.0 if not np.isfinite(p.dt) else 1.0 / p.dt
    return esd.EsdFvGrid(d, p.shape[0], p.shape[1], p.shape[2] if d == 3 else 1, p.h, inv_dt)


def case(name):
    rng = np.random.default_rng({"2d": 1, "3d_dt": 2, "3d_steady": 3}[name])
    if name == "2d":
        shape, dt = (13, 9), 0.05
    elif name == "3d_dt":
        shape, dt = (7, 6, 5), 1e-3
    else:
        shape, dt = (8, 8, 8), np.inf
    theta = rng.standard_normal(shape)
    p = wl.fv_diffusion(np.exp(theta), 1.0 / shape[0], dt)
    return p, theta


@pytest.mark.parametrize("name", ["2d", "3d_dt", "3d_steady"])
def test_fv_assemble_matches_generator(name):
    p, theta = case(name)
    p_other = wl.fv_diffusion(np.ones(theta.shape), p.h, p.dt)  # same pattern, other values
    A_ref = esd.Matrix.from_problem(p)
    A = esd.Matrix.from_problem(p_other)
    esd.esd_fv_assemble(A.handle, grid_of(p), dev(nat(theta)), dev(cell_row(p)))
    v = np.random.default_rng(0).standard_normal(p.n)
    y_ref, y = np.zeros(p.n), np.zeros(p.n)
    A_ref.spmv(v, y_ref)
    A.spmv(v, y)
    assert np.linalg.norm(y - y_ref) <= 1e-14 * np.linalg.norm(y_ref)
    # host inputs take the same path
    A2 = esd.Matrix.from_problem(p_other)
    esd.esd_fv_assemble(A2.handle, grid_of(p), nat(theta), cell_row(p))
    A2.spmv(v, y)
    assert np.linalg.norm(y - y_ref) <= 1e-14 * np.linalg.norm(y_ref)


def test_fv_assemble_rejects_bad_input_and_keeps_A():
    p, theta = case("3d_dt")
    A = esd.Matrix.from_problem(p)
    v = np.random.default_rng(1).standard_normal(p.n)
    y0, y = np.zeros(p.n), np.zeros(p.n)
    A.spmv(v, y0)
    bad = cell_row(p)
    bad[5] = p.n + 3  # outside 0..n-1: the kernel checks before it reads
    with pytest.raises(esd.EsdError) as e:
        esd.esd_fv_assemble(A.handle, grid_of(p), nat(theta + 1.0), bad)
    assert e.value.code == esd.ERR_INVALID
    A.spmv(v, y)
    assert np.array_equal(y, y0)
    g = grid_of(p)
    g.nx += 1  # grid does not match n
    with pytest.raises(esd.EsdError):
        esd.esd_fv_assemble(A.handle, g, nat(theta), cell_row(p))


@pytest.mark.parametrize("name", ["2d", "3d_dt", "3d_steady"])
def test_fv_grad_theta_matches_oracle(name):
    p, theta = case(name)
    A = esd.Matrix.from_problem(p)
    rng = np.random.default_rng(4)
    lam, x = rng.standard_normal(p.n), rng.standard_normal(p.n)
    g = torch.empty(p.n, dtype=torch.float64, device=DEV)
    esd.esd_fv_grad_theta(A.handle, grid_of(p), dev(nat(theta)), dev(cell_row(p)), dev(lam), dev(x), g)
    ref = nat(oracle.fv_theta_gradient(theta, p.h, oracle.to_grid(p, lam), oracle.to_grid(p, x)))
    assert np.abs(g.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()


def test_set_values_and_stale_state():
    p, theta = case("3d_dt")
    A = esd.Matrix.from_problem(p)
    A.factor_ic0()
    S = esd.Solver(A, sample_cap=8)
    b = np.random.default_rng(2).uniform(size=p.n)
    x = np.zeros(p.n)
    S.solve(b, x, tol=1e-8, sample_m=8)
    S.sample_and_build_W()
    S.set_mode(esd.DEFLATION)
    A.set_values(2.0 * p.val)
    v = np.random.default_rng(3).standard_normal(p.n)
    y = np.zeros(p.n)
    A.spmv(v, y)
    assert np.linalg.norm(y - 2.0 * (p.scipy() @ v)) <= 1e-14 * np.linalg.norm(y)
    with pytest.raises(esd.EsdError) as e:  # factor dropped
        S.solve(b, np.zeros(p.n), tol=1e-8)
    assert e.value.code == esd.ERR_STATE
    A.factor_ic0()
    with pytest.raises(esd.EsdError) as e:  # W formed for the old values
        S.solve(b, np.zeros(p.n), tol=1e-8)
    assert e.value.code == esd.ERR_STATE
    S.refresh_W()
    W, AW, E = S.get_W()
    np.testing.assert_allclose(AW, 2.0 * (p.scipy() @ W), rtol=1e-12, atol=1e-12 * np.abs(AW).max())
    x = np.zeros(p.n)
    st, it, rr = S.solve(b, x, tol=1e-8)
    assert st == esd.OK
    assert np.linalg.norm(b - 2.0 * (p.scipy() @ x)) <= 1.01e-8 * np.linalg.norm(b)


@pytest.fixture(scope="module")
def c4_small():
    p, theta, xt = wl.config_c4(N=16)
    return p, theta, xt


@pytest.mark.parametrize("precision", [esd.FP64, esd.FP32_REFINE])
def test_autograd_matches_oracle_adjoint(c4_small, precision):
    p, theta, xt = c4_small
    model = FVDiffusion(p, mode=esd.DEFLATION, precision=precision, sample_cap=16)
    th = dev(nat(theta)).requires_grad_(True)
    b = dev(p.source).requires_grad_(True)
    kept = model.build_W(th, b.detach(), m=16, tol=1e-10)
    assert kept >= 4
    x = fv_solve(th, b, model, tol=1e-13)
    loss = ((x - dev(xt)) ** 2).sum()
    loss.backward()
    adj_iters = model.solver.last_solve_info()["iters"]
    ref = oracle.adjoint_gradient(p, theta, p.source, xt, tol=1e-13)
    assert abs(loss.item() - ref["loss"]) <= 1e-9 * ref["loss"]
    gb = b.grad.cpu().numpy()
    gt = th.grad.cpu().numpy()
    assert np.linalg.norm(gb - ref["grad_b"]) <= 1e-8 * np.linalg.norm(ref["grad_b"])
    rt = nat(ref["grad_theta"])
    assert np.abs(gt - rt).max() <= 1e-8 * np.abs(rt).max()
    # the adjoint ran deflated with the forward's W: fewer iterations than plain ICCG
    plain = oracle.System(p, oracle.IC0(p)).solve(2.0 * (ref["x"] - xt), tol=1e-13, history=False)["iters"]
    assert adj_iters < plain, (adj_iters, plain)


def test_autograd_matches_finite_differences(c4_small):
    p, theta, xt = c4_small
    model = FVDiffusion(p, mode=esd.DEFLATION, sample_cap=16)
    th0 = dev(nat(theta))
    b = dev(p.source)
    model.build_W(th0, b, m=16, tol=1e-10)
    th = th0.clone().requires_grad_(True)
    x = fv_solve(th, b, model, tol=1e-13)
    ((x - dev(xt)) ** 2).sum().backward()
    g = th.grad.cpu().numpy()

    def loss(t):
        with torch.no_grad():
            xx = fv_solve(t, b, model, tol=1e-13)
            return float(((xx - dev(xt)) ** 2).sum())

    cells = np.random.default_rng(7).choice(p.n, size=32, replace=False)
    step = 1e-6
    for c in cells:
        tp, tm = th0.clone(), th0.clone()
        tp[c] += step
        tm[c] -= step
        fd = (loss(tp) - loss(tm)) / (2 * step)
        assert abs(fd - g[c]) <= 1e-5 * np.abs(g).max(), (c, fd, g[c])
    # dL/db against central differences in b on 8 cells
    bb = b.clone().requires_grad_(True)
    x = fv_solve(th0, bb, model, tol=1e-13)
    ((x - dev(xt)) ** 2).sum().backward()
    gb = bb.grad.cpu().numpy()

    def loss_b(bv):
        with torch.no_grad():
            xx = fv_solve(th0, bv, model, tol=1e-13)
            return float(((xx - dev(xt)) ** 2).sum())

    hb = 1e-6 * float(b.abs().max())
    for c in np.random.default_rng(8).choice(p.n, size=8, replace=False):
        bp, bm = b.clone(), b.clone()
        bp[c] += hb
        bm[c] -= hb
        fd = (loss_b(bp) - loss_b(bm)) / (2 * hb)
        assert abs(fd - gb[c]) <= 1e-5 * np.abs(gb).max(), (c, fd, gb[c])


@pytest.mark.slow
def test_full_size_gradient_matches_oracle():
    """The 128^3 log-normal workload at full size: the adjoint gradients through the autograd
    API (deflation, m = 16, both solves at tol 1e-12) against the oracle's ICCG adjoint
    gradient at tol 1e-12 (1e-7: the two FP64 runs each stop at 1e-12), and central finite
    differences (step 1e-5) on 4 seeded cells to 1e-4."""
    p, theta, xt = wl.config_c4(N=128)
    model = FVDiffusion(p, mode=esd.DEFLATION, sample_cap=16)
    th0 = dev(nat(theta))
    b = dev(p.source)
    model.build_W(th0, b, m=16, tol=1e-10)
    th = th0.clone().requires_grad_(True)
    x = fv_solve(th, b, model, tol=1e-12)
    ((x - dev(xt)) ** 2).sum().backward()
    g = th.grad.cpu().numpy()
    ref = oracle.adjoint_gradient(p, theta, p.source, xt, tol=1e-12)
    rt = nat(ref["grad_theta"])
    assert np.abs(g - rt).max() <= 1e-7 * np.abs(rt).max()

    def loss(t):
        with torch.no_grad():
            xx = fv_solve(t, b, model, tol=1e-12)
            return float(((xx - dev(xt)) ** 2).sum())

    step = 1e-5
    for c in np.random.default_rng(9).choice(p.n, size=4, replace=False):
        tp, tm = th0.clone(), th0.clone()
        tp[c] += step
        tm[c] -= step
        fd = (loss(tp) - loss(tm)) / (2 * step)
        assert abs(fd - g[c]) <= 1e-4 * np.abs(g).max(), (c, fd, g[c])
