"""The object-aware rasterizer as a differentiable PyTorch function.

`render(scorer, cams, i, means, log_scales, quats, opacity, sh, obj_logits)`
returns (rgb [H,W,3], depth [H,W], alpha [H,W], obj [H,W,K+1]) of camera i;
its backward is the library's hand-written backward pass (nbv_render_backward:
per-tile recomputation of the forward pass, back-to-front adjoints, the chain
rule through the projection). Forward and backward both run in the library's
kernels; this module only passes tensors.
"""
from __future__ import annotations

import torch


class _Render(torch.autograd.Function):
    @staticmethod
    def forward(ctx, scorer, cams, i, means, log_scales, quats, opacity, sh, obj_logits):
        params = (means, log_scales, quats, opacity, sh, obj_logits)
        scorer.load_gaussians(*[p.detach() for p in params])
        out = scorer.render_camera(cams, i)
        ctx.scorer, ctx.cams, ctx.i = scorer, cams, i
        ctx.save_for_backward(*params)
        return out["rgb"], out["depth"], out["alpha"], out["obj"]

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_alpha, g_obj):
        params = ctx.saved_tensors
        sc = ctx.scorer
        sc.load_gaussians(*[p.detach() for p in params])      # the Gaussians this output came from
        g = sc.render_backward(ctx.cams, ctx.i, g_rgb, g_depth, g_alpha, g_obj)
        out = [g["means"], g["log_scales"], g["quats"], g["opacity"], g["sh"], g["obj_logits"]]
        out = [o.reshape(p.shape) if ctx.needs_input_grad[3 + k] else None for k, (o, p) in enumerate(zip(out, params))]
        return (None, None, None, *out)


def render(scorer, cams, i, means, log_scales, quats, opacity, sh, obj_logits):
    return _Render.apply(scorer, cams, i, means, log_scales, quats, opacity, sh, obj_logits)
