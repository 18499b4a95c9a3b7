"""torch.autograd.Functions around the differentiable sparse render.

``SparseRender.apply(opacity, topk_val, renderer, view)`` renders one view of
``renderer`` (a ``Render``) with the given opacities and Top-K values and
returns the dense code map [H, W, C]; its backward returns the gradients
with respect to both (Top-K indices and compositing decisions held fixed).
``SparseDecode.apply(codes, codebook)`` decodes code rows [P, C] to features
[P, D] (Eq. 8, bf16 tensor cores, FP32 output); its backward returns
dL/dcodes = dL/dF codebook^T (the codebook is held fixed).  All directions
run in libscoup.so.
"""
from __future__ import annotations

import torch

from .scoup import (Render, scene_struct, scoup_decode, scoup_decode_backward, scoup_render,
                    scoup_render_backward)


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


class SparseDecode(torch.autograd.Function):
    @staticmethod
    def forward(ctx, codes: torch.Tensor, codebook: torch.Tensor):
        c = codes.detach().contiguous()
        cb = codebook.detach().contiguous()
        feats = torch.empty((c.shape[0], cb.shape[1]), dtype=torch.float32, device=c.device)
        scoup_decode(c, cb, feats)
        ctx.save_for_backward(cb)
        return feats

    @staticmethod
    def backward(ctx, grad_feats: torch.Tensor):
        (cb,) = ctx.saved_tensors
        g = grad_feats.contiguous().float()
        d_codes = torch.empty((g.shape[0], cb.shape[0]), dtype=torch.float32, device=g.device)
        scoup_decode_backward(g, cb, d_codes)
        return d_codes, None
