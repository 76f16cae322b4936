"""torch.autograd wrappers over the C ABI (differentiation of far-field
objectives with respect to excitation coefficients).

Every forward and backward step runs in libpie:
  Apply     y = Z x          backward: Z^H g           (pie_apply / pie_apply_t)
  Solve     x = Z^-1 b       backward: Z^-H g = conj(Z^-1 conj g)  (pie_solve / pie_solve_nested)
  FarField  E = F x          backward: F^H g           (pie_farfield / pie_farfield_adjoint)
For complex tensors torch passes the conjugate-Wirtinger gradient, so the
backward of a complex-linear map A is A^H applied to the incoming gradient.
"""
import torch


class Apply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, problem):
        ctx.problem = problem
        return problem.apply(x.contiguous())

    @staticmethod
    def backward(ctx, g):
        return ctx.problem.apply_t(g.contiguous(), conj=True), None


def _solve(problem, inner, b, tol, maxit, restart):
    """pie_solve, or pie_solve_nested with the complex-float operator inner."""
    if inner is None:
        return problem.solve(b, tol=tol, maxit=maxit, restart=restart)
    return problem.solve_nested(b, inner, tol=tol)


class Solve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, b, problem, tol, maxit, restart, adj_tol, inner):
        ctx.problem, ctx.inner, ctx.args = problem, inner, (adj_tol, maxit, restart)
        x, st = _solve(problem, inner, b.contiguous(), tol, maxit, restart)
        if not st["converged"]:
            raise RuntimeError(f"GMRES did not converge: {st}")
        return x

    @staticmethod
    def backward(ctx, g):
        tol, maxit, restart = ctx.args
        lam, st = _solve(ctx.problem, ctx.inner, g.conj().contiguous(), tol, maxit, restart)
        if not st["converged"]:
            raise RuntimeError(f"adjoint GMRES did not converge: {st}")
        return lam.conj(), None, None, None, None, None, None


class FarField(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, problem, rhat):
        ctx.problem, ctx.rhat = problem, rhat
        return problem.farfield(x.contiguous(), rhat)

    @staticmethod
    def backward(ctx, g):
        return ctx.problem.farfield_adjoint(g.contiguous(), ctx.rhat), None, None


def apply(problem, x):
    return Apply.apply(x, problem)


def solve(problem, b, tol=1e-6, maxit=3000, restart=100, adj_tol=1e-4, inner=None):
    """x = Z^-1 b; the backward pass solves Z^H lam = g to adj_tol (Z^H =
    conj Z conj, Z being complex symmetric).  With inner (a complex-float
    Problem on the same mesh) both solves are nested ones (pie_solve_nested).
    With plain GMRES on a PIE_FP64 problem (1280-triangle sphere, kR = 0.01)
    the adjoint right-hand side F^H E was measured to stall near 5e-5; the
    default adj_tol of 1e-4 is ample for gradients."""
    return Solve.apply(b, problem, tol, maxit, restart, adj_tol, inner)


def farfield(problem, x, rhat):
    return FarField.apply(x, problem, rhat)
