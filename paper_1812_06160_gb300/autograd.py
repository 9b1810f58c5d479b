"""Differentiable preconditioner apply z = U^-1 L^-1 r.

Forward: one forward and one backward substitution (Sec. VI, stri) with the
ILU(0) factor.  Backward, for an upstream gradient gz (all through the
library's kernels):

    gy = U^-T gz                 (forward solve over the columns of U)
    gr = L^-T gy                 (backward solve over the columns of L)
    y  = L^-1 r                  (recomputed, not stored)
    g_lu[p] = -sum_c gr[i,c] y[j,c]   for p = (i, j), j < i   (gradient of L)
    g_lu[p] = -sum_c gy[i,c] z[j,c]   for p = (i, j), j >= i  (gradient of U)

i.e. the gradient with respect to the stored factor values, restricted to
the pattern.  The paper has no adjoint; this is the extension's definition.
"""
from __future__ import annotations

import torch

from . import _jv


class IluApply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, r, lu, handle):
        y = _jv.jv_lsolve(handle, lu, r, x_dtype=lu.dtype)
        z = _jv.jv_usolve(handle, lu, y, x_dtype=r.dtype)
        ctx.handle = handle
        ctx.save_for_backward(r, lu, z)
        return z

    @staticmethod
    def backward(ctx, gz):
        r, lu, z = ctx.saved_tensors
        h = ctx.handle
        gz = gz.contiguous().to(lu.dtype)
        gy = _jv.jv_usolve_t(h, lu, gz)
        gr = _jv.jv_lsolve_t(h, lu, gy)
        glu = None
        if ctx.needs_input_grad[1]:
            y = _jv.jv_lsolve(h, lu, r.to(lu.dtype))
            zc = z.to(lu.dtype)
            glu = _jv.jv_masked_outer(h, 0, gr, y, alpha=-1.0)
            _jv.jv_masked_outer(h, 1, gy, zc, alpha=-1.0, g=glu)
        return gr.to(r.dtype), glu, None


def ilu_apply(r, lu, handle):
    """z = U^-1 L^-1 r, differentiable in r and in the factor values lu."""
    return IluApply.apply(r, lu, handle)
