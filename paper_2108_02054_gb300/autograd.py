"""Differentiable pressure solve u(theta, f) = A(exp(theta))^-1 f.

forward:  assemble A from the per-cell log-density theta on the device (the
          kernel forms rho = exp(theta)), refresh the hierarchy (full setup
          the first time, partial rebuild -- Alg. 4 -- afterwards), solve with
          V-cycle-preconditioned CG.  Only theta and u are kept for the
          backward pass (no Krylov iterates).
backward: A is symmetric, so the adjoint system A lam = dL/du is solved with
          the same, already refreshed hierarchy; one kernel then forms dL/dA on
          A's pattern (-lam_i u_j) chained through the harmonic-mean face
          coefficients to dL/dtheta per cell; dL/df = lam.  If another forward
          refreshed the shared hierarchy in between (a second loss, a
          finite-difference probe), the hierarchy is first rebuilt from the
          saved theta, so the adjoint always solves with A(theta) of its own
          forward.

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
        self.generation = 0     # bumped by every refresh: which theta the hierarchy holds
        self.last_info = None
        self.adjoint_info = None

    def assemble(self, theta: torch.Tensor):
        th = theta.detach().to(torch.float64).contiguous()
        return th, B.poisson_values_log(self.dim, self.N, th, self.ptr, self.top)

    def refresh(self, val):
        if not self.ready:
            self.amg.full_setup(self.ptr, self.col, val)
            self.ready = True
        else:
            self.amg.partial_rebuild(val)
        self.generation += 1
        return self.generation

    def solve(self, f: torch.Tensor):
        u, info = self.amg.solve(f.detach().to(torch.float64).contiguous(), self.tol, allow_not_converged=False)
        return u, info


class AMGSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, f, solver: PoissonSolver):
        th, val = solver.assemble(theta)
        ctx.generation = solver.refresh(val)
        u, info = solver.solve(f)
        solver.last_info = info
        ctx.solver = solver
        ctx.save_for_backward(th, u)
        return u

    @staticmethod
    def backward(ctx, g):
        solver = ctx.solver
        th, u = ctx.saved_tensors
        if solver.generation != ctx.generation:
            # the hierarchy now holds another forward's A: rebuild it for this theta
            solver.refresh(solver.assemble(th)[1])
        lam, info = solver.solve(g.contiguous())
        solver.adjoint_info = info
        grad_theta = B.poisson_grad_log(solver.dim, solver.N, th, u, lam, solver.top)
        return grad_theta, lam, None


def solve(theta: torch.Tensor, f: torch.Tensor, solver: PoissonSolver) -> torch.Tensor:
    return AMGSolve.apply(theta, f, solver)
