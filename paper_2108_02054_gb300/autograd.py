"""Differentiable pressure solve u(theta, f) = A(exp(theta))^-1 f.

forward:  assemble A from the per-cell log-density theta on the device, refresh
          the hierarchy (full setup the first time, partial rebuild -- Alg. 4 --
          afterwards), solve with V-cycle-preconditioned CG.  Only u is kept
          for the backward pass (no Krylov iterates).
backward: A is symmetric, so the adjoint system A lam = dL/du is solved with
          the same, already refreshed hierarchy; one kernel then forms dL/dA on
          A's pattern (-lam_i u_j) chained through the harmonic-mean face
          coefficients to dL/dtheta per cell; dL/df = lam.

All numerical work runs in libamgpr.so; PyTorch only holds the tensors.
"""
from __future__ import annotations

import torch

from . import amg as B


class PoissonSolver:
    """Owns the pattern and one AMG context for a fixed N^dim grid."""

    def __init__(self, dim: int, N: int, tol: float = 1e-10, dirichlet_top: bool = True, **params):
        self.dim, self.N, self.tol, self.top = dim, N, tol, dirichlet_top
        self.ptr, self.col = B.poisson_pattern(dim, N)
        self.amg = B.AMG(**params)
        self.ready = False
        self.last_info = None
        self.adjoint_info = None

    def assemble(self, theta: torch.Tensor):
        rho = torch.exp(theta.detach().to(torch.float64)).contiguous()
        return rho, B.poisson_values(self.dim, self.N, rho, self.ptr, self.top)

    def refresh(self, val):
        if not self.ready:
            self.amg.full_setup(self.ptr, self.col, val)
            self.ready = True
        else:
            self.amg.partial_rebuild(val)

    def solve(self, f: torch.Tensor):
        u, info = self.amg.solve(f.detach().to(torch.float64).contiguous(), self.tol, allow_not_converged=False)
        return u, info


class AMGSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, f, solver: PoissonSolver):
        rho, val = solver.assemble(theta)
        solver.refresh(val)
        u, info = solver.solve(f)
        solver.last_info = info
        ctx.solver = solver
        ctx.save_for_backward(rho, u)
        return u

    @staticmethod
    def backward(ctx, g):
        solver = ctx.solver
        rho, u = ctx.saved_tensors
        lam, info = solver.solve(g.contiguous())
        solver.adjoint_info = info
        grad_theta = B.poisson_grad_theta(solver.dim, solver.N, rho, u, lam, solver.top)
        return grad_theta, lam, None


def solve(theta: torch.Tensor, f: torch.Tensor, solver: PoissonSolver) -> torch.Tensor:
    return AMGSolve.apply(theta, f, solver)
