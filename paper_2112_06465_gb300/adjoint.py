"""Differentiable Helmholtz solves: torch.autograd.Function wrappers whose
backward pass is a hand-written adjoint BiCGStab plus a sparse outer product.

For x = A^{-1} b and the conjugate-Wirtinger gradient g = dL/dx that PyTorch
hands to backward (for a real loss L), the adjoint system is A^H lambda = g.
Writing mu = conj(lambda) turns it into A^T mu = conj(g); A is complex
symmetric, so this is a second solve with the SAME operator (and the same
captured solver graph).  Then
    dL/db        = conj(mu)
    dL/dA_ij     = -conj(mu_i x_j)          (stored entries only)
    dL/dtheta_i  = conj(c) * dL/dA_ii       for A_ii = base_i + c * theta_i.
All three are formed by library kernels (hz_zconj, hz_outer_on_pattern,
hz_diag_grad).  The forward and the adjoint solve use the same Krylov method
(``method``, ``ell`` and ``precond`` as in ``hz.zsolve``): on operators where
BiCGStab stagnates, TFQMR or BiCGStab(l) may still reach the tolerance.
"""

import torch

from . import hz


class DiagParamSolve(torch.autograd.Function):
    """x = A(theta)^{-1} b with A(theta)_ii = base_i + scale * theta_i.

    The off-diagonal entries of ``A`` are fixed; its diagonal is rewritten
    from theta on every forward (and again before the adjoint solve, so a
    later forward with other parameters does not corrupt this backward).
    """

    @staticmethod
    def forward(ctx, theta, b, A, base, scale, tol, maxit, opts):
        theta = theta.contiguous()
        b = b.contiguous()
        hz.mat_set_diag(A, base, scale, theta)
        x, info = hz.zsolve(A, b, tol=tol, maxit=maxit, **opts)
        if not info.converged:
            raise RuntimeError(f"forward solve did not converge: {info}")
        ctx.A, ctx.base, ctx.scale, ctx.tol, ctx.maxit, ctx.opts = A, base, scale, tol, maxit, opts
        ctx.fwd_info = info
        ctx.save_for_backward(theta, x)
        return x

    @staticmethod
    def backward(ctx, g):
        theta, x = ctx.saved_tensors
        A = ctx.A
        hz.mat_set_diag(A, ctx.base, ctx.scale, theta)
        rhs = hz.zconj(g.contiguous())
        mu, info = hz.zsolve(A, rhs, tol=ctx.tol, maxit=ctx.maxit, **ctx.opts)
        if not info.converged:
            raise RuntimeError(f"adjoint solve did not converge: {info}")
        ctx.adj_info = info
        grad_theta = hz.diag_grad(A, mu, x, ctx.scale) if ctx.needs_input_grad[0] else None
        grad_b = hz.zconj(mu) if ctx.needs_input_grad[1] else None
        return grad_theta, grad_b, None, None, None, None, None, None


def _opts(method, ell, precond):
    return {"method": method, "ell": ell, "precond": precond}


def solve_diag_param(theta, b, A, base, scale, tol=1e-12, maxit=5000, method="bicgstab", ell=4, precond="none"):
    """Differentiable x = A(theta)^{-1} b (see DiagParamSolve); method, ell and
    precond select the Krylov solver of both the forward and the adjoint solve."""
    return DiagParamSolve.apply(theta, b, A, base, scale, tol, maxit, _opts(method, ell, precond))


class ValuesSolve(torch.autograd.Function):
    """x = A(val)^{-1} b where val are the stored entries of A's pattern."""

    @staticmethod
    def forward(ctx, val, b, A, tol, maxit, opts):
        hz.zcopy(val.contiguous(), A.val)
        A.refresh_values()
        x, info = hz.zsolve(A, b.contiguous(), tol=tol, maxit=maxit, **opts)
        if not info.converged:
            raise RuntimeError(f"forward solve did not converge: {info}")
        ctx.A, ctx.tol, ctx.maxit, ctx.opts = A, tol, maxit, opts
        ctx.save_for_backward(val, x)
        return x

    @staticmethod
    def backward(ctx, g):
        val, x = ctx.saved_tensors
        A = ctx.A
        hz.zcopy(val.contiguous(), A.val)
        A.refresh_values()
        mu, info = hz.zsolve(A, hz.zconj(g.contiguous()), tol=ctx.tol, maxit=ctx.maxit, **ctx.opts)
        if not info.converged:
            raise RuntimeError(f"adjoint solve did not converge: {info}")
        grad_val = hz.outer_on_pattern(A, mu, x) if ctx.needs_input_grad[0] else None
        grad_b = hz.zconj(mu) if ctx.needs_input_grad[1] else None
        return grad_val, grad_b, None, None, None, None


def solve_values(val, b, A, tol=1e-12, maxit=5000, method="bicgstab", ell=4, precond="none"):
    """Differentiable x = A(val)^{-1} b with gradients for the stored values;
    method, ell and precond select the Krylov solver of both solves."""
    return ValuesSolve.apply(val, b, A, tol, maxit, _opts(method, ell, precond))
