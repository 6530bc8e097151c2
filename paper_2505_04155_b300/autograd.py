"""torch.autograd integration: the backward of a solve is the adjoint solve.

For x = A^-1 b with A symmetric, a loss L(x) has dL/db = lambda with
A lambda = dL/dx (solved with the same mixed-precision PCG and policy as the
forward solve) and dL/dA = -lambda x^T on the sparsity pattern (ampcg_adjoint).
Two parameterisations are provided:
  - ValuesSolve: the FP64 CSR values themselves are the leaf;
  - LogCoeffSolve: a node log-coefficient field theta with
    a_ij = -exp((theta_i + theta_j)/2), a_ii = sum_j exp(...) + nb_i exp(theta_i);
    the library assembles A(theta) and chains dL/dA to dL/dtheta on the GPU
    (ampcg_assemble_log_coeff, ampcg_grad_log_coeff).
Tensors are CUDA FP64; every arithmetic step runs in the library's kernels.
"""
from __future__ import annotations

import torch

from . import Policy, Solver


class ValuesSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vals, b, solver: Solver, tol: float, maxit: int, policy: Policy | None):
        vals = vals.detach().contiguous()
        solver.update_values(vals)
        x, info = solver.solve(b.detach().contiguous(), tol=tol, maxit=maxit, policy=policy,
                               history=False)
        ctx.save_for_backward(vals, x)
        ctx.args = (solver, tol, maxit, policy)
        return x

    @staticmethod
    def backward(ctx, gx):
        vals, x = ctx.saved_tensors
        solver, tol, maxit, policy = ctx.args
        solver.update_values(vals)          # the values this x was computed with
        lam, dA, _ = solver.adjoint(x, gx.contiguous(), tol=tol, maxit=maxit, policy=policy,
                                    want_dA=ctx.needs_input_grad[0])
        return dA, lam, None, None, None, None


class LogCoeffSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, b, solver: Solver, nbound, tol: float, maxit: int,
                policy: Policy | None):
        theta = theta.detach().contiguous()
        solver.assemble_log_coeff(theta, nbound)
        x, _ = solver.solve(b.detach().contiguous(), tol=tol, maxit=maxit, policy=policy,
                            history=False)
        ctx.save_for_backward(theta, x)
        ctx.args = (solver, nbound, tol, maxit, policy)
        return x

    @staticmethod
    def backward(ctx, gx):
        theta, x = ctx.saved_tensors
        solver, nbound, tol, maxit, policy = ctx.args
        solver.assemble_log_coeff(theta, nbound)
        lam, _, _ = solver.adjoint(x, gx.contiguous(), tol=tol, maxit=maxit, policy=policy,
                                   want_dA=False)
        dtheta = solver.grad_log_coeff(x, lam) if ctx.needs_input_grad[0] else None
        return dtheta, lam, None, None, None, None, None


def solve_values(vals, b, solver: Solver, tol: float = 1e-10, maxit: int = 5000,
                 policy: Policy | None = None):
    """x = A(vals)^-1 b, differentiable in vals and b."""
    return ValuesSolve.apply(vals, b, solver, tol, maxit, policy)


def solve_log_coeff(theta, b, solver: Solver, nbound, tol: float = 1e-10, maxit: int = 5000,
                    policy: Policy | None = None):
    """x = A(theta)^-1 b, differentiable in theta and b."""
    return LogCoeffSolve.apply(theta, b, solver, nbound, tol, maxit, policy)
