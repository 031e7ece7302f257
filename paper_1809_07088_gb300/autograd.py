"""torch.autograd.Function over the library's forward (ds_request_intensity) and adjoint
(ds_backward): I(u) for displacements or I(M) for moments, TOTAL mode, so that a refinement
loop can optimise a model against a target volume with torch optimisers.

The forward uploads the tensor into the model (device to device), computes the volume on the
tensor's stream and saves nothing but the grid and options; the backward recomputes the forward
inside ds_backward and returns dL/du (or dL/dM) in the upload layout.
"""
from __future__ import annotations

import torch

from . import DS_DISP, DS_FP32, DS_SPIN, DS_TOTAL


class _DiffuseIntensity(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, model, qgrid, opts):
        xc = x.detach().contiguous()
        if opts["disorder"] == DS_DISP:
            model.upload_displacements(xc)
        else:
            model.upload_spins(xc)
        dt = torch.float64 if opts["precision"] == 0 else torch.float32
        out = torch.empty(tuple(int(c) for c in qgrid[2]), dtype=dt, device=x.device)
        model.intensity(qgrid, out=out, **opts)
        ctx.model, ctx.qgrid, ctx.opts, ctx.dtype = model, qgrid, opts, x.dtype
        return out

    @staticmethod
    def backward(ctx, grad_out):
        g = grad_out.contiguous()
        grad = torch.empty(ctx.model._shape(3), dtype=g.dtype, device=g.device)
        ctx.model.backward(ctx.qgrid, g, grad=grad, **ctx.opts)
        return grad.to(ctx.dtype), None, None, None


def diffuse_intensity(model, x, qgrid, disorder=DS_DISP, precision=DS_FP32, taylor_order=-1, taylor_eps=1e-8):
    """I(G) of `model` with displacements (disorder=DS_DISP) or moments (DS_SPIN) `x`, a CUDA
    float32 tensor [model][site][n1][n2][n3][3]; differentiable with respect to x."""
    if disorder not in (DS_DISP, DS_SPIN):
        raise ValueError("differentiable for displacements or moments only")
    opts = dict(disorder=disorder, mode=DS_TOTAL, precision=precision, taylor_order=taylor_order,
                taylor_eps=taylor_eps)
    return _DiffuseIntensity.apply(x, model, qgrid, opts)
