"""Differentiable absorber solve over the C-ABI (argument marshalling only).

absorber_solve(coef, ...) returns x = A(sigma)^-1 b(sigma) for a conductivity
sigma given as a cubic B-spline with coefficients coef [S] (Eq. 23 in a
smooth basis).  Its backward pass solves the adjoint system A^T lam =
conj(dJ/dx) with the transposed operator (GMRES, scabem_solve with
transpose = 1) and turns lam and x into dJ/dcoef = -Re(g) with g from
scabem_sigma_gradient (both A and b are affine in sigma).
"""

from __future__ import annotations

import torch

from . import (SCABEM_C128, make_source, scabem_rhs, scabem_set_sigma, scabem_sigma_gradient,  # noqa: F401
               scabem_solve)


class _BSplineAbsorberSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coef, op, n_unknowns, spline, sources, solve_kw):
        x0, L, axis = spline
        c = coef.detach().to("cpu", torch.float64).numpy()
        scabem_set_sigma(op, bspline=(x0, L, axis, c))
        b = torch.zeros(n_unknowns, dtype=torch.complex128, device="cuda")
        scabem_rhs(op, list(sources), b, prec=SCABEM_C128)
        x = torch.zeros_like(b)
        scabem_solve(op, b, x, **solve_kw)
        ctx.op, ctx.spline, ctx.sources, ctx.solve_kw = op, spline, list(sources), dict(solve_kw)
        ctx.save_for_backward(coef, x)
        return x

    @staticmethod
    def backward(ctx, gx):
        coef, x = ctx.saved_tensors
        x0, L, axis = ctx.spline
        c = coef.detach().to("cpu", torch.float64).numpy()
        scabem_set_sigma(ctx.op, bspline=(x0, L, axis, c))  # the operator may have changed since forward
        rhs = torch.conj(gx).resolve_conj().to(torch.complex128).contiguous()
        lam = torch.zeros_like(rhs)
        scabem_solve(ctx.op, rhs, lam, transpose=True, **ctx.solve_kw)
        g = scabem_sigma_gradient(ctx.op, x.contiguous(), lam, ctx.sources, bspline=(x0, L, axis, len(c)))
        grad = torch.as_tensor(-g.real, dtype=coef.dtype, device=coef.device)
        return grad, None, None, None, None, None


def absorber_solve(coef, op, n_unknowns, spline, sources, **solve_kw):
    """x(coef) for sigma = cubic B-spline(coef) on spline = (x0, L, axis) and the
    excitation `sources` (make_source list); solve_kw goes to scabem_solve."""
    return _BSplineAbsorberSolve.apply(coef, op, n_unknowns, spline, tuple(sources), solve_kw)
