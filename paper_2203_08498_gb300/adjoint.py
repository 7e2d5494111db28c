"""Differentiable solves: ``x = A(theta)^-1 b`` as a ``torch.autograd.Function``.

The backward pass is the adjoint solve ``A lambda = dL/dx``. A is symmetric, so the adjoint
is one more system with the same matrix: it runs with the same mode (plain, deflation or
subspace correction) and the same W and E as the forward solve. Then ``dL/db = lambda``
and ``dL/dtheta`` comes from ``esd_fv_grad_theta`` (the chain rule through the harmonic-mean
faces and k = exp(theta), on the device). The operator is the cell-centred finite-volume
diffusion ``A = I/dt + K(exp(theta))`` of ``esd_fv_assemble``, assembled on the device
whenever theta changes, then refactored (IC(0)) with AW, E formed again for the kept W.

Argument marshalling only, like the rest of the binding: every numerical step runs in the
library's kernels.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import (DEFLATION, FP64, OK, PLAIN, EsdError, EsdFvGrid, Matrix, Solver, esd_fv_assemble,
               esd_fv_grad_theta)

__all__ = ["FVDiffusion", "AdjointSolve", "fv_solve", "natural_order"]


def natural_order(theta_grid: torch.Tensor) -> torch.Tensor:
    """Grid-shaped tensor (axis 0 = x) -> 1-D natural order (x fastest)."""
    return theta_grid.permute(*reversed(range(theta_grid.dim()))).reshape(-1).contiguous()


class FVDiffusion:
    """Matrix, IC(0) factor, solver and W of ``A(theta)`` on one structured grid.

    ``prob`` supplies the pattern and its colour-major ordering (rowptr, colind, val,
    colour_ptr, perm with perm[row] = natural cell, shape, h, dt); its values are replaced
    by the device assembly at the first ``set_theta``.
    """

    def __init__(self, prob, mode=DEFLATION, precision=FP64, maxit=20000, sample_cap=32, device=None):
        self.device = torch.device(device or "cuda")
        self.shape = tuple(prob.shape)
        self.n = prob.n
        dt = prob.dt
        self.grid = EsdFvGrid(len(self.shape), self.shape[0], self.shape[1],
                              self.shape[2] if len(self.shape) == 3 else 1, prob.h,
                              0.0 if (dt is None or not math.isfinite(dt) or dt == 0.0) else 1.0 / dt)
        inv = np.empty(self.n, dtype=np.int32)
        inv[np.asarray(prob.perm)] = np.arange(self.n, dtype=np.int32)
        self.cell_row = torch.from_numpy(inv).to(self.device)
        self.matrix = Matrix.from_problem(prob)
        self.matrix.factor_ic0()  # a solver is created on a factored matrix
        self.solver = Solver(self.matrix, maxit_cap=maxit, sample_cap=sample_cap, precision=precision)
        self.mode = mode
        self.maxit = maxit
        self.has_W = False
        self._theta = None

    def set_theta(self, theta: torch.Tensor):
        """Assemble A(theta) on the device when theta differs from the current one."""
        theta = theta.detach().to(self.device, torch.float64).contiguous()
        if self._theta is not None and torch.equal(theta, self._theta):
            return
        esd_fv_assemble(self.matrix.handle, self.grid, theta, self.cell_row)
        self.matrix.factor_ic0()
        if self.has_W:
            self.solver.refresh_W()
        self._theta = theta.clone()

    def build_W(self, theta, b, m=16, tol=1e-8):
        """Solve A(theta) x = b in plain mode while sampling m iterates (method A), build W
        from their errors and switch to ``mode``. Returns the number of columns kept."""
        self.set_theta(theta)
        x = torch.zeros(self.n, dtype=torch.float64, device=self.device)
        self.solver.set_mode(PLAIN)
        st, it, rr = self.solver.solve(b, x, tol=tol, maxit=self.maxit, sample_m=m)
        if st != OK:
            raise EsdError(st, "sampled solve did not converge")
        kept = self.solver.sample_and_build_W()
        self.has_W = True
        self.solver.set_mode(self.mode)
        return kept

    def solve(self, b, x, tol):
        self.solver.set_mode(self.mode if self.has_W else PLAIN)
        st, it, rr = self.solver.solve(b, x, tol=tol, maxit=self.maxit)
        if st != OK:
            raise EsdError(st, f"solve stopped at relative residual {rr:.3e} after {it} iterations")
        return it

    def grad_theta(self, theta, lam, x, out):
        esd_fv_grad_theta(self.matrix.handle, self.grid, theta, self.cell_row, lam, x, out)


class AdjointSolve(torch.autograd.Function):
    """x = A(theta)^-1 b; backward: A lambda = dL/dx with the same mode, W and E."""

    @staticmethod
    def forward(ctx, theta, b, model: FVDiffusion, tol: float):
        model.set_theta(theta)
        b = b.detach().contiguous()
        x = torch.zeros_like(b)
        ctx.forward_iters = model.solve(b, x, tol)
        ctx.save_for_backward(theta, x)
        ctx.model, ctx.tol = model, tol
        return x

    @staticmethod
    def backward(ctx, gx):
        theta, x = ctx.saved_tensors
        model = ctx.model
        model.set_theta(theta)
        gx = gx.detach().contiguous()
        lam = torch.zeros_like(gx)
        model.solve(gx, lam, ctx.tol)
        g_theta = None
        if ctx.needs_input_grad[0]:
            g_theta = torch.empty_like(theta, dtype=torch.float64).contiguous()
            model.grad_theta(theta.detach().contiguous(), lam, x, g_theta)
        g_b = lam if ctx.needs_input_grad[1] else None
        return g_theta, g_b, None, None


def fv_solve(theta: torch.Tensor, b: torch.Tensor, model: FVDiffusion, tol: float = 1e-10) -> torch.Tensor:
    """Differentiable ``A(theta)^-1 b`` (theta in natural cell order, b in matrix order)."""
    return AdjointSolve.apply(theta, b, model, tol)
