"""Differentiable sparse least squares on top of the spaQR factorization.

x(vals, b) = argmin ||A x - b||_2 = (A^T A)^{-1} A^T b, where A has the fixed
sparsity pattern of a factorization and the nonzero values ``vals``.  The
backward pass is the adjoint of the normal equations: with g = dL/dx,
lambda = (A^T A)^{-1} g (CG preconditioned by the stored factor W, a W^{-T}
then a W^{-1} sweep per iteration) and r = b - A x,

    dL/db = A lambda,      dL/dA_ij = r_i lambda_j - (A lambda)_i x_j,

the latter on the nonzeros of A, computed by one fused CUDA kernel.
"""
from __future__ import annotations

import torch

from . import solve_batch, solve_normal_batch

__all__ = ["SpaqrLstsq", "SpaqrLstsqBatch", "lstsq", "lstsq_batch"]


class SpaqrLstsq(torch.autograd.Function):
    """x = argmin ||A(vals) x - b|| through one factorization ``solver`` (a SpaQR).

    forward loads ``vals`` into the solver (keeping its factor as the
    preconditioner unless ``refactor``); backward uses the values of the last
    forward call of that solver."""

    @staticmethod
    def forward(ctx, vals, b, solver, tol_adjoint=1e-12, refactor=False):
        solver.update_values(vals.detach().to(torch.float64).contiguous(), refactor=refactor)
        x = solver.solve(b.detach().to(torch.float64).contiguous())
        ctx.solver = solver
        ctx.tol = tol_adjoint
        ctx.save_for_backward(b.detach(), x)
        return x

    @staticmethod
    def backward(ctx, gx):
        b, x = ctx.saved_tensors
        lam = ctx.solver.solve_normal(gx.detach().to(torch.float64).contiguous(), tol=ctx.tol)
        gb, gv = ctx.solver.lstsq_grad(b.to(torch.float64).contiguous(), x, lam)
        return gv, gb, None, None, None


class SpaqrLstsqBatch(torch.autograd.Function):
    """Row i of X = argmin ||A_i(vals[i]) x - b[i]|| for a list of factorizations
    (one pattern); the solves and the adjoint solves of all problems iterate
    side by side."""

    @staticmethod
    def forward(ctx, vals, bs, solvers, tol_adjoint=1e-12, refactor=False):
        for s, v in zip(solvers, vals):
            s.update_values(v.detach().to(torch.float64).contiguous(), refactor=refactor)
        xs, _ = solve_batch(solvers, [b.detach().to(torch.float64).contiguous() for b in bs])
        X = torch.stack(xs)
        ctx.solvers = solvers
        ctx.tol = tol_adjoint
        ctx.save_for_backward(bs.detach(), X)
        return X

    @staticmethod
    def backward(ctx, gX):
        bs, X = ctx.saved_tensors
        lams, _ = solve_normal_batch(ctx.solvers, [g.to(torch.float64).contiguous() for g in gX], tol=ctx.tol)
        gbs, gvs = [], []
        for s, b, x, lam in zip(ctx.solvers, bs, X, lams):
            gb, gv = s.lstsq_grad(b.to(torch.float64).contiguous(), x.contiguous(), lam)
            gbs.append(gb)
            gvs.append(gv)
        return torch.stack(gvs), torch.stack(gbs), None, None, None


def lstsq(vals, b, solver, tol_adjoint: float = 1e-12, refactor: bool = False):
    return SpaqrLstsq.apply(vals, b, solver, tol_adjoint, refactor)


def lstsq_batch(vals, bs, solvers, tol_adjoint: float = 1e-12, refactor: bool = False):
    return SpaqrLstsqBatch.apply(vals, bs, solvers, tol_adjoint, refactor)
