"""The corrected layer potential as a differentiable PyTorch operation (an extension: the
paper has no gradients).

    u = corrected_potential(ctx, deg, node_off, xyz, sigma, tgt_xyz, tgt_node, kernel, k, prm)

runs build_near_lists, gen_corrections and apply_corrected_* in the library; backward
calls lcq_apply_adjoint for the density gradient (A^H g) and lcq_shape_gradient for the
node-coordinate gradient (discrete choices frozen, refinement trees recomputed).  Both
gradients are the library's kernels; this module only passes tensors.
"""
from __future__ import annotations

import torch

from . import lcq

_APPLY = {"S": lcq.apply_corrected_S, "D": lcq.apply_corrected_D, "CFIE": lcq.apply_corrected_CFIE}


class CorrectedPotential(torch.autograd.Function):
    @staticmethod
    def forward(fctx, sigma, xyz, ctx, deg, node_off, tgt_xyz, tgt_node, kernel, k, prm, alpha,
                beta, precision):
        ds = lcq.DeviceSurface(deg, node_off, xyz.detach().contiguous())
        near = lcq.build_near_lists(ctx, ds, tgt_xyz, tgt_node, prm)
        corr = lcq.gen_corrections(ctx, ds, near, kernel, k, prm, alpha, beta, precision)
        sig = sigma.detach().contiguous()
        u = _APPLY[kernel](ctx, ds, near, corr, sig, int(tgt_node.shape[0]))
        fctx.lcq = (ctx, ds, near, corr, sig)
        return u

    @staticmethod
    def backward(fctx, gu):
        ctx, ds, near, corr, sig = fctx.lcq
        g = gu.contiguous()
        gs = gy = None
        if fctx.needs_input_grad[0]:
            gs = lcq.apply_adjoint(ctx, ds, near, corr, g)
        if fctx.needs_input_grad[1]:
            gy = lcq.shape_gradient(ctx, ds, near, corr, sig, g)
        return (gs, gy) + (None,) * 11


def corrected_potential(ctx, deg, node_off, xyz, sigma, tgt_xyz, tgt_node, kernel, k, prm,
                        alpha=1.0, beta=0.0, precision="fp64"):
    """u at the targets (complex128 [NT]); differentiable in sigma (complex128 [N]) and in
    the node coordinates xyz (float64 [3][N]; off-surface targets only)."""
    return CorrectedPotential.apply(sigma, xyz, ctx, deg, node_off, tgt_xyz, tgt_node, kernel, k,
                                    prm, alpha, beta, precision)
