"""Differentiable sparse solve x = A^{-1} b through the AMG-preconditioned FCG.

forward:  builds the hierarchy of A (amg_setup) and solves A x = b (amg_pcg_solve).
backward: for an incoming dL/dx, solves the adjoint system A lambda = dL/dx with the SAME
          hierarchy (A is symmetric, so the preconditioner applies unchanged), then
          dL/db = lambda and dL/dA_ij = -lambda_i x_j on the stored pattern of A
          (cwm_pattern_outer).  Tie a_ij to a_ji, or to physical coefficients, by
          differentiating the assembly of `val` (see problems.diffusion_fv_torch).

All computation runs in the CUDA library through the binding; tensors are float64 CUDA.
"""
from __future__ import annotations

import torch

from . import binding as B


class AmgSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, val, b, row_ptr, col, v, params, rtol, itmax):
        h = B.amg_setup(row_ptr, col, val.detach().contiguous(), v, params)
        x = torch.zeros_like(b)
        st, info = B.amg_pcg_solve(h, b.detach().contiguous(), x, rtol=rtol, itmax=itmax)
        if st != B.AMG_OK:
            h.free()
            raise B.AmgError(st, "AmgSolve.forward", "FCG did not reach the tolerance")
        ctx.h = h
        ctx.rtol, ctx.itmax = rtol, itmax
        ctx.info = info
        ctx.save_for_backward(x, row_ptr, col)
        return x

    @staticmethod
    def backward(ctx, gx):
        x, row_ptr, col = ctx.saved_tensors
        lam = torch.zeros_like(x)
        st, info = B.amg_pcg_solve(ctx.h, gx.contiguous(), lam, rtol=ctx.rtol, itmax=ctx.itmax)
        ctx.adjoint_info = info
        ctx.h.free()
        if st != B.AMG_OK:
            raise B.AmgError(st, "AmgSolve.backward", "adjoint FCG did not reach the tolerance")
        dval = B.cwm_pattern_outer(row_ptr, col, lam, x, alpha=-1.0) if ctx.needs_input_grad[0] else None
        db = lam if ctx.needs_input_grad[1] else None
        return dval, db, None, None, None, None, None, None


def amg_solve(row_ptr, col, val, b, v=None, params=None, rtol: float = 1e-10, itmax: int = 5000):
    """x = A^{-1} b with A given by (row_ptr, col, val); differentiable in val and b."""
    if v is None:
        v = torch.ones_like(b)
    return AmgSolve.apply(val, b, row_ptr, col, v, params, rtol, itmax)
