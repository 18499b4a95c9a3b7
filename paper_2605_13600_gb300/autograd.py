"""torch.autograd.Function around scoup_render / scoup_render_backward.

``SparseRender.apply(opacity, topk_val, renderer, view)`` renders one view of
``renderer`` (a ``Render``) with the given opacities and Top-K values and
returns the dense code map [H, W, C]; its backward returns the gradients
with respect to both (Top-K indices and compositing decisions held fixed).
Both directions run in libscoup.so.
"""
from __future__ import annotations

import torch

from .scoup import Render, scene_struct, scoup_render, scoup_render_backward


class SparseRender(torch.autograd.Function):
    @staticmethod
    def forward(ctx, opacity: torch.Tensor, topk_val: torch.Tensor, renderer: Render, view: int):
        r = renderer
        op = opacity.detach().contiguous()
        val = topk_val.detach().contiguous()
        sc = scene_struct(r.means, r.scales, r.quats, op)
        cam = r.cams[view]
        out = r.outputs(cam)
        scoup_render(sc, r.topk_idx, val, r.K, r.C, cam, out[0], out[1], out[2], r.workspace, stats=False)
        ctx.save_for_backward(op, val)
        ctx.renderer = r
        ctx.view = view
        return out[0]

    @staticmethod
    def backward(ctx, grad_codes: torch.Tensor):
        op, val = ctx.saved_tensors
        r = ctx.renderer
        sc = scene_struct(r.means, r.scales, r.quats, op)
        d_val = torch.zeros_like(val)
        d_op = torch.zeros_like(op)
        scoup_render_backward(sc, r.topk_idx, val, r.K, r.C, r.cams[ctx.view],
                              grad_codes.contiguous().float(), d_val, d_op, r.workspace)
        return d_op, d_val, None, None
