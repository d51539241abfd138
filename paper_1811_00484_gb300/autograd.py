"""Differentiable solve: E(chi) = e_inc + G w with A(chi) w = chi e_inc.

Backward (adjoint method): for an upstream gradient gE of a real loss,
dL = Re <gE, dE>, dE = G dw and A dw = dchi * E, so
    A^H mu = G^H gE,   grad_chi = sum_b sum_a mu conj(E),
i.e. one adjoint matvec, one adjoint GMRES solve and one reduction, all in
libvie (vie_matvec_adjoint, vie_solve with VIE_SOLVE_ADJOINT,
vie_contrast_gradient with scale 1).
"""
from __future__ import annotations

import torch


class SolveFields(torch.autograd.Function):
    @staticmethod
    def forward(ctx, chi, einc, op, opts):
        w, info = op.solve(chi, einc, incident=True, **opts)
        E = op.total_field(einc, w, path=opts.get("path", "tucker"))
        ctx.op = op
        ctx.opts = opts
        ctx.info = info
        ctx.save_for_backward(chi, E)
        return E

    @staticmethod
    def backward(ctx, gE):
        chi, E = ctx.saved_tensors
        op, opts = ctx.op, ctx.opts
        rhs = op.matvec_adjoint(gE.contiguous(), path=opts.get("path", "tucker"))
        mu, _ = op.solve(chi, rhs, incident=False, adjoint=True, **opts)
        gchi = op.contrast_gradient(mu, E, scale=1.0)
        return gchi, None, None, None


def solve_fields(op, chi, einc, **opts):
    """Total field E for contrast ``chi`` and incident field ``einc`` (differentiable in chi)."""
    return SolveFields.apply(chi, einc, op, opts)
