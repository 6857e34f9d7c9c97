"""torch.autograd.Function front of the render-and-compare step.

`latents(ctx, job)` returns leaf tensors (requires_grad) that alias the job's
library-owned latents: positions (base positions of a tessellated job), the
level 0 of every optimized texture, and the displacement map. Calling
`render_loss(...)` runs adms_forward_loss; its backward runs the hand-written
backward kernels (AA, shading, texel and vertex scatter, tangent frame,
tessellation adjoints) in recompute mode, so nothing the forward rasterized
is read back: keys, pre-AA colours and loss gradients are rebuilt from the
latents and the reference images. `laplacian(...)` wraps Eq. 4's L_delta and
its hand-written gradient. All arithmetic runs in libadms.so.

A job holds one forward's state at a time: call backward before the next
forward of the same job. After changing latents in place (e.g. a torch
optimizer step), call `invalidate(ctx, job)` so mip chains and the vertex
frame are rebuilt.
"""

from __future__ import annotations

import torch

from . import binding as B

TEXTURES = ("kd", "orm", "nrm")


def latents(ctx, job, names=None):
    """{name: leaf tensor aliasing the job's latent, requires_grad=True} for the optimized latents."""
    p = ctx.params(job)
    out = {}
    for name in names or ("pos", "kd", "orm", "nrm", "disp"):
        if name not in p or p[name] is None:
            continue
        if name in TEXTURES and p["g_" + name] is None:
            continue
        if name == "disp" and p.get("g_disp") is None:
            continue
        out[name] = p[name].requires_grad_(True)
    return out


def invalidate(ctx, job):
    B.adms_job_invalidate(ctx.ctx, job)


class _RenderLoss(torch.autograd.Function):
    @staticmethod
    def forward(fctx, ctx, job, views, refs, names, *tensors):
        loss = ctx.forward_loss([job], [views], [refs])
        fctx.ctx, fctx.job, fctx.names = ctx, job, names
        fctx.shapes = [t.shape for t in tensors]
        return loss[0].clone()

    @staticmethod
    def backward(fctx, g):
        ctx, job = fctx.ctx, fctx.job
        B.adms_job_zero_gradients(ctx.ctx, job)
        ctx.backward([job], recompute_raster=True)
        p = ctx.params(job)
        grads = []
        for name, shape in zip(fctx.names, fctx.shapes):
            if name in TEXTURES:
                buf = torch.empty(shape, dtype=torch.float32, device=g.device)
                B.adms_job_fold_gradients(ctx.ctx, job, **{"g_" + name: buf})
            else:
                buf = p["g_" + name].clone()
            grads.append(buf * g)
        B.adms_job_zero_gradients(ctx.ctx, job)
        return (None, None, None, None, None, *grads)


def render_loss(ctx, job, views, refs, lat):
    """L_image of one job on one batch of views (Sec. 5.3), differentiable in `lat`."""
    names = tuple(lat.keys())
    return _RenderLoss.apply(ctx, job, views, refs, names, *[lat[n] for n in names])


class _Laplacian(torch.autograd.Function):
    @staticmethod
    def forward(fctx, ctx, job, pos):
        out = torch.zeros(1, dtype=torch.float32, device=pos.device)
        grad = torch.empty_like(pos)
        B.adms_laplacian(ctx.ctx, job, out, grad)
        fctx.save_for_backward(grad)
        return out[0].clone()

    @staticmethod
    def backward(fctx, g):
        (grad,) = fctx.saved_tensors
        return None, None, grad * g


def laplacian(ctx, job, pos):
    """L_delta of Eq. 4 for the job's positions (pos must alias them)."""
    return _Laplacian.apply(ctx, job, pos)
