"""Pins of the oracle's adjoint gradient (CPU only).

The oracle's dL/dtheta and dL/db for L = ||x - x_target||^2, A(theta) x = b, are checked
against central finite differences of the exact loss, computed with dense solves of the
assembled matrix, on small 2D and 3D grids; and the ICCG-based adjoint against the same
gradient from dense solves. Nothing here reuses the oracle's chain rule.
"""
import numpy as np
import pytest

import oracle
import workloads as wl

GRIDS = {
    "3d_3x4x2_steady": ((3, 4, 2), np.inf),
    "2d_5x4_dt": ((5, 4), 0.05),
    "3d_2x2x2_dt": ((2, 2, 2), 0.5),
}
H = 0.25
FD_STEP = 1e-5


def _setup(name, seed=0):
    shape, dt = GRIDS[name]
    rng = np.random.default_rng(seed)
    theta = rng.standard_normal(shape)
    p = wl.fv_diffusion(np.exp(theta), H, dt)
    b = rng.standard_normal(p.n)
    xt = rng.standard_normal(p.n)
    return shape, dt, theta, p, b, xt


def _loss(theta, dt, b, xt):
    A = wl.fv_diffusion(np.exp(theta), H, dt).scipy().toarray()
    x = np.linalg.solve(A, b)
    return float(np.dot(x - xt, x - xt))


def _dense_grad(p, theta, b, xt):
    A = p.scipy().toarray()
    x = np.linalg.solve(A, b)
    lam = np.linalg.solve(A, 2.0 * (x - xt))
    return lam, oracle.fv_theta_gradient(theta, H, oracle.to_grid(p, lam), oracle.to_grid(p, x))


@pytest.mark.parametrize("name", sorted(GRIDS))
def test_theta_gradient_matches_finite_differences(name):
    shape, dt, theta, p, b, xt = _setup(name)
    _, g = _dense_grad(p, theta, b, xt)
    fd = np.zeros(shape)
    for idx in np.ndindex(shape):
        tp, tm = theta.copy(), theta.copy()
        tp[idx] += FD_STEP
        tm[idx] -= FD_STEP
        fd[idx] = (_loss(tp, dt, b, xt) - _loss(tm, dt, b, xt)) / (2 * FD_STEP)
    assert np.abs(g - fd).max() <= 1e-5 * np.abs(fd).max()


@pytest.mark.parametrize("name", sorted(GRIDS))
def test_b_gradient_is_lambda(name):
    shape, dt, theta, p, b, xt = _setup(name, seed=1)
    lam, _ = _dense_grad(p, theta, b, xt)
    A = p.scipy().toarray()
    fd = np.zeros(p.n)
    for i in range(p.n):
        e = np.zeros(p.n)
        e[i] = FD_STEP
        xp, xm = np.linalg.solve(A, b + e), np.linalg.solve(A, b - e)
        fd[i] = (np.dot(xp - xt, xp - xt) - np.dot(xm - xt, xm - xt)) / (2 * FD_STEP)
    assert np.abs(lam - fd).max() <= 1e-6 * np.abs(fd).max()


def test_adjoint_identity():
    """lambda^T b = x^T (dL/dx) for the linear map b -> x (A symmetric)."""
    shape, dt, theta, p, b, xt = _setup("3d_3x4x2_steady", seed=2)
    A = p.scipy().toarray()
    x = np.linalg.solve(A, b)
    g = 2.0 * (x - xt)
    lam = np.linalg.solve(A, g)
    assert abs(lam @ b - x @ g) <= 1e-12 * abs(x @ g)


def test_iccg_adjoint_gradient_equals_dense():
    """The ICCG forward + adjoint (tol 1e-13) reproduce the dense-solve gradient."""
    rng = np.random.default_rng(3)
    theta = rng.standard_normal((6, 5, 4))
    p = wl.fv_diffusion(np.exp(theta), 1.0 / 6, np.inf)
    b = rng.standard_normal(p.n)
    xt = rng.standard_normal(p.n)
    out = oracle.adjoint_gradient(p, theta, b, xt, tol=1e-13)
    A = p.scipy().toarray()
    x = np.linalg.solve(A, b)
    lam = np.linalg.solve(A, 2.0 * (x - xt))
    g = oracle.fv_theta_gradient(theta, p.h, oracle.to_grid(p, lam), oracle.to_grid(p, x))
    assert np.linalg.norm(out["grad_b"] - lam) <= 1e-9 * np.linalg.norm(lam)
    assert np.abs(out["grad_theta"] - g).max() <= 1e-9 * np.abs(g).max()


def test_grid_order_round_trip():
    p = wl.small_3d(5, seed=1)
    v = np.arange(p.n, dtype=np.float64)
    assert np.array_equal(oracle.from_grid(p, oracle.to_grid(p, v)), v)
    # natural order: x fastest
    nat = oracle.to_grid(p, v).ravel(order="F")
    assert np.array_equal(nat[p.perm], v)
