"""torch.autograd wrappers over the C ABI (differentiation of far-field
objectives with respect to excitation coefficients).

Every forward and backward step runs in libpie:
  Apply     y = Z x          backward: Z^H g           (pie_apply / pie_apply_t)
  Solve     x = Z^-1 b       backward: Z^-H g = conj(Z^-1 conj g)  (pie_solve)
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


class Solve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, b, problem, tol, maxit, restart, adj_tol):
        ctx.problem, ctx.args = problem, (adj_tol, maxit, restart)
        x, st = problem.solve(b.contiguous(), tol=tol, maxit=maxit, restart=restart)
        if not st["converged"]:
            raise RuntimeError(f"GMRES did not converge: {st}")
        return x

    @staticmethod
    def backward(ctx, g):
        tol, maxit, restart = ctx.args
        lam, st = ctx.problem.solve(g.conj().contiguous(), tol=tol, maxit=maxit, restart=restart)
        if not st["converged"]:
            raise RuntimeError(f"adjoint GMRES did not converge: {st}")
        return lam.conj(), None, None, None, None, None


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


def solve(problem, b, tol=1e-6, maxit=3000, restart=100, adj_tol=1e-4):
    """x = Z^-1 b; the backward pass solves Z^H lam = g to adj_tol.  The
    far part's FP64 rounding gives the operator a small nonlinearity, so
    right-hand sides such as F^H E (receiving-type) stall near 5e-5; 1e-4 is
    ample for gradients."""
    return Solve.apply(b, problem, tol, maxit, restart, adj_tol)


def farfield(problem, x, rhat):
    return FarField.apply(x, problem, rhat)
