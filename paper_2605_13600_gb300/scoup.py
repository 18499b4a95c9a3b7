"""Python binding of the C ABI: argument marshalling only.

Functions carry the C names (``scoup_uplift`` ...) and take torch tensors
already on the GPU; every step of the computation runs in libscoup.so.
``Uplift`` is a convenience wrapper that sizes and allocates the workspace
and outputs with torch and then calls the same entry points.
"""
from __future__ import annotations

import ctypes as ct
from typing import Optional, Sequence

import numpy as np

from . import _lib
from ._lib import (SCOUP_ACCUM_COMPENSATED, SCOUP_ACCUM_CONTINUE, SCOUP_BATCH_EAGER, SCOUP_UPLIFT_CHUNKED, BatchItem,
                   Camera, Level, PlanInfo, Scene, ScoupError, Stats, check, load)


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _need(t, dtype, name):
    import torch
    if t is None:
        return
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() and not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")


def scene_struct(means, scales, quats, opacity) -> Scene:
    import torch
    for t, nm in ((means, "means"), (scales, "scales"), (quats, "quats"), (opacity, "opacity")):
        _need(t, torch.float32, nm)
    sc = Scene()
    sc.n = int(means.shape[0])
    sc.means, sc.scales, sc.quats, sc.opacity = _ptr(means), _ptr(scales), _ptr(quats), _ptr(opacity)
    sc._keep = (means, scales, quats, opacity)
    return sc


def camera_array(cams: Sequence) -> ct.Array:
    arr = (Camera * max(1, len(cams)))()
    for k, c in enumerate(cams):
        vm = np.asarray(c.viewmat, np.float32).reshape(12)
        for i in range(12):
            arr[k].viewmat[i] = float(vm[i])
        arr[k].fx, arr[k].fy, arr[k].cx, arr[k].cy = float(c.fx), float(c.fy), float(c.cx), float(c.cy)
        arr[k].width, arr[k].height = int(c.width), int(c.height)
    return arr


def scoup_version() -> str:
    return load().scoup_version().decode()


def scoup_uplift_workspace_size(n: int, max_width: int, max_height: int, dup_capacity: int) -> int:
    return int(load().scoup_uplift_workspace_size(n, max_width, max_height, dup_capacity))


def scoup_uplift_chunked_workspace_size(n: int, max_width: int, max_height: int, dup_capacity: int) -> int:
    """Workspace bytes of scoup_uplift with SCOUP_UPLIFT_CHUNKED."""
    return int(load().scoup_uplift_chunked_workspace_size(n, max_width, max_height, dup_capacity))


def scoup_uplift_plan(scene: Scene, cams: Sequence, workspace, stream=None) -> int:
    import torch
    _need(workspace, torch.uint8, "workspace")
    out = ct.c_int64(0)
    ca = camera_array(cams)
    check(load().scoup_uplift_plan(ct.byref(scene), ct.cast(ca, ct.c_void_p), len(cams),
                                   _ptr(workspace), workspace.numel(), ct.byref(out), _stream(stream)))
    return int(out.value)


def scoup_uplift(scene: Scene, cams: Sequence, region_maps, map_offsets, R_total: int, code_idx,
                 code_val, s: int, C: int, K: int, accum, accum_mode: int, topk_idx, topk_val,
                 workspace, stats: bool = True, stream=None):
    """Returns the stats dict (synchronising) when stats=True, else None.

    With SCOUP_ACCUM_COMPENSATED in accum_mode, accum holds 2 * n * C floats
    (the sums, then their compensation terms)."""
    import torch
    if accum is not None and accum.numel() < scene.n * C * (2 if accum_mode & SCOUP_ACCUM_COMPENSATED else 1):
        raise ValueError("accum is too small for n x C (x 2 when compensated)")
    _need(region_maps, torch.int32, "region_maps")
    _need(code_idx, torch.int32, "code_idx")
    _need(code_val, torch.float32, "code_val")
    _need(accum, torch.float32, "accum")
    _need(topk_idx, torch.int32, "topk_idx")
    _need(topk_val, torch.float32, "topk_val")
    _need(workspace, torch.uint8, "workspace")
    offs = np.ascontiguousarray(np.asarray(map_offsets, np.int64)[:max(1, len(cams))])
    ca = camera_array(cams)
    st = Stats()
    rc = load().scoup_uplift(ct.byref(scene), ct.cast(ca, ct.c_void_p), len(cams), _ptr(region_maps),
                             offs.ctypes.data_as(ct.c_void_p), int(R_total), _ptr(code_idx),
                             _ptr(code_val), int(s), int(C), int(K), _ptr(accum), int(accum_mode),
                             _ptr(topk_idx), _ptr(topk_val), _ptr(workspace),
                             0 if workspace is None else workspace.numel(),
                             ct.byref(st) if stats else None, _stream(stream))
    check(rc)
    return st.as_dict() if stats else None


def scoup_uplift_host_maps_workspace_size(n: int, max_width: int, max_height: int, dup_capacity: int) -> int:
    return int(load().scoup_uplift_host_maps_workspace_size(n, max_width, max_height, dup_capacity))


def scoup_uplift_host_maps_chunked_workspace_size(n: int, max_width: int, max_height: int, dup_capacity: int) -> int:
    """Workspace bytes of scoup_uplift_host_maps with SCOUP_UPLIFT_CHUNKED."""
    return int(load().scoup_uplift_host_maps_chunked_workspace_size(n, max_width, max_height, dup_capacity))


def scoup_uplift_host_maps(scene: Scene, cams: Sequence, host_region_maps, map_offsets, R_total: int, code_idx,
                           code_val, s: int, C: int, K: int, accum, accum_mode: int, topk_idx, topk_val,
                           workspace, stats: bool = True, stream=None):
    """scoup_uplift with the region maps in host memory (a CPU tensor, pinned
    for asynchronous copies): each view's map is staged into the workspace
    while earlier views compute."""
    import torch
    if not isinstance(host_region_maps, torch.Tensor) or host_region_maps.device.type != "cpu":
        raise TypeError("host_region_maps must be a CPU tensor (pinned for asynchronous copies)")
    if accum is not None and accum.numel() < scene.n * C * (2 if accum_mode & SCOUP_ACCUM_COMPENSATED else 1):
        raise ValueError("accum is too small for n x C (x 2 when compensated)")
    if host_region_maps.dtype != torch.int32 or not host_region_maps.is_contiguous():
        raise TypeError("host_region_maps must be a contiguous int32 tensor")
    _need(code_idx, torch.int32, "code_idx")
    _need(code_val, torch.float32, "code_val")
    _need(accum, torch.float32, "accum")
    _need(topk_idx, torch.int32, "topk_idx")
    _need(topk_val, torch.float32, "topk_val")
    _need(workspace, torch.uint8, "workspace")
    offs = np.ascontiguousarray(np.asarray(map_offsets, np.int64)[:max(1, len(cams))])
    ca = camera_array(cams)
    st = Stats()
    rc = load().scoup_uplift_host_maps(ct.byref(scene), ct.cast(ca, ct.c_void_p), len(cams), _ptr(host_region_maps),
                                       offs.ctypes.data_as(ct.c_void_p), int(R_total), _ptr(code_idx),
                                       _ptr(code_val), int(s), int(C), int(K), _ptr(accum), int(accum_mode),
                                       _ptr(topk_idx), _ptr(topk_val), _ptr(workspace),
                                       0 if workspace is None else workspace.numel(),
                                       ct.byref(st) if stats else None, _stream(stream))
    check(rc)
    return st.as_dict() if stats else None


def scoup_uplift_noalloc(scene: Scene, cams: Sequence, region_maps, map_offsets, R_total: int,
                         code_idx, code_val, s: int, C: int, K: int, accum, accum_mode: int,
                         topk_idx, topk_val, stream=None) -> dict:
    """scoup_uplift with the library's fixed scratch array (no workspace
    argument, nothing allocated); synchronises and returns the stats dict."""
    import torch
    if accum is not None and accum.numel() < scene.n * C * (2 if accum_mode & SCOUP_ACCUM_COMPENSATED else 1):
        raise ValueError("accum is too small for n x C (x 2 when compensated)")
    _need(region_maps, torch.int32, "region_maps")
    _need(code_idx, torch.int32, "code_idx")
    _need(code_val, torch.float32, "code_val")
    _need(accum, torch.float32, "accum")
    _need(topk_idx, torch.int32, "topk_idx")
    _need(topk_val, torch.float32, "topk_val")
    offs = np.ascontiguousarray(np.asarray(map_offsets, np.int64)[:max(1, len(cams))])
    ca = camera_array(cams)
    st = Stats()
    check(load().scoup_uplift_noalloc(ct.byref(scene), ct.cast(ca, ct.c_void_p), len(cams),
                                      _ptr(region_maps), offs.ctypes.data_as(ct.c_void_p), int(R_total),
                                      _ptr(code_idx), _ptr(code_val), int(s), int(C), int(K), _ptr(accum),
                                      int(accum_mode), _ptr(topk_idx), _ptr(topk_val), ct.byref(st),
                                      _stream(stream)))
    return st.as_dict()


def scoup_uplift_noalloc_max_bytes() -> int:
    return int(load().scoup_uplift_noalloc_max_bytes())


def scoup_topk(accum, K: int, topk_idx, topk_val, stream=None) -> None:
    import torch
    _need(accum, torch.float32, "accum")
    _need(topk_idx, torch.int32, "topk_idx")
    _need(topk_val, torch.float32, "topk_val")
    n, C = accum.shape
    check(load().scoup_topk(_ptr(accum), n, C, K, _ptr(topk_idx), _ptr(topk_val), _stream(stream)))


def scoup_render(scene: Scene, topk_idx, topk_val, K: int, C: int, cam, out_codes, out_T, out_last,
                 workspace, stats: bool = True, stream=None):
    """Eq. 7 for one view into out_codes [H, W, C] (float32 or bfloat16); returns stats when stats=True."""
    import torch
    _need(topk_idx, torch.int32, "topk_idx")
    _need(topk_val, torch.float32, "topk_val")
    if out_codes.dtype not in (torch.float32, torch.bfloat16):
        raise TypeError("out_codes must be float32 or bfloat16")
    _need(out_codes, out_codes.dtype, "out_codes")
    _need(out_T, torch.float32, "out_T")
    _need(out_last, torch.int32, "out_last")
    _need(workspace, torch.uint8, "workspace")
    ca = camera_array([cam])
    st = Stats()
    check(load().scoup_render(ct.byref(scene), _ptr(topk_idx), _ptr(topk_val), int(K), int(C),
                              ct.cast(ca, ct.POINTER(Camera)), _ptr(out_codes),
                              1 if out_codes.dtype == torch.bfloat16 else 0, _ptr(out_T), _ptr(out_last),
                              _ptr(workspace), workspace.numel(), ct.byref(st) if stats else None,
                              _stream(stream)))
    return st.as_dict() if stats else None


def scoup_render_backward(scene: Scene, topk_idx, topk_val, K: int, C: int, cam, dL_dcodes, d_topk_val,
                          d_opacity, workspace, stats: bool = False, stream=None):
    """Adds dL/dval and dL/dopacity of one view into d_topk_val [n, K], d_opacity [n]."""
    import torch
    for t, nm in ((topk_val, "topk_val"), (dL_dcodes, "dL_dcodes"), (d_topk_val, "d_topk_val"),
                  (d_opacity, "d_opacity")):
        _need(t, torch.float32, nm)
    _need(topk_idx, torch.int32, "topk_idx")
    _need(workspace, torch.uint8, "workspace")
    ca = camera_array([cam])
    st = Stats()
    check(load().scoup_render_backward(ct.byref(scene), _ptr(topk_idx), _ptr(topk_val), int(K), int(C),
                                       ct.cast(ca, ct.POINTER(Camera)), _ptr(dL_dcodes), _ptr(d_topk_val),
                                       _ptr(d_opacity), _ptr(workspace), workspace.numel(),
                                       ct.byref(st) if stats else None, _stream(stream)))
    return st.as_dict() if stats else None


class Render:
    """Device copies of a scene and its K-sparse codes plus a planned workspace
    for rendering views of up to max_width x max_height."""

    def __init__(self, scene, topk_idx, topk_val, C: int, cams, device: str = "cuda",
                 dup_capacity: Optional[int] = None):
        import torch
        dev = torch.device(device)
        self.means = torch.as_tensor(scene.means, device=dev).contiguous()
        self.scales = torch.as_tensor(scene.scales, device=dev).contiguous()
        self.quats = torch.as_tensor(scene.quats, device=dev).contiguous()
        self.opacity = torch.as_tensor(scene.opacity, device=dev).contiguous()
        self.scene = scene_struct(self.means, self.scales, self.quats, self.opacity)
        self.topk_idx = torch.as_tensor(np.asarray(topk_idx, np.int32), device=dev).contiguous()
        self.topk_val = torch.as_tensor(np.asarray(topk_val, np.float32), device=dev).contiguous()
        self.K = int(self.topk_idx.shape[1]) if self.topk_idx.ndim == 2 else 1
        self.C = int(C)
        self.cams = list(cams)
        n = int(scene.means.shape[0])
        maxw = max([c.width for c in self.cams] + [1])
        maxh = max([c.height for c in self.cams] + [1])
        if dup_capacity is None:
            probe = torch.empty(scoup_uplift_workspace_size(n, maxw, maxh, 0), dtype=torch.uint8, device=dev)
            dup_capacity = scoup_uplift_plan(self.scene, self.cams, probe) + 1
            del probe
        self.workspace = torch.empty(scoup_uplift_workspace_size(n, maxw, maxh, dup_capacity),
                                     dtype=torch.uint8, device=dev)
        self.device = dev
        self.n, self.maxw, self.maxh, self.dup_capacity = n, maxw, maxh, dup_capacity
        self._fused_ws = None

    def outputs(self, cam, dtype=None):
        import torch
        H, W = cam.height, cam.width
        return (torch.empty((H, W, self.C), dtype=dtype or torch.float32, device=self.device),
                torch.empty((H, W), dtype=torch.float32, device=self.device),
                torch.empty((H, W), dtype=torch.int32, device=self.device))

    def run(self, v: int, out=None, stats: bool = True, stream=None):
        cam = self.cams[v]
        out = self.outputs(cam) if out is None else out
        st = scoup_render(self.scene, self.topk_idx, self.topk_val, self.K, self.C, cam, out[0], out[1],
                          out[2], self.workspace, stats=stats, stream=stream)
        return out, st

    def run_decode(self, v: int, codebook, features, feat_norm2=None, out_T=None, out_last=None,
                   stats: bool = True, stream=None):
        """View v rendered and decoded in one call (scoup_render_decode_fused):
        features [H * W, D] (float32 or bfloat16) = bf16(What) @ codebook."""
        import torch
        D = int(codebook.shape[1])
        need = scoup_render_decode_workspace_size(self.n, self.maxw, self.maxh, self.C, D, self.dup_capacity)
        if self._fused_ws is None or self._fused_ws.numel() < need:
            self._fused_ws = torch.empty(need, dtype=torch.uint8, device=self.device)
        return scoup_render_decode_fused(self.scene, self.topk_idx, self.topk_val, self.K, self.C, self.cams[v],
                                         codebook, features, feat_norm2, out_T, out_last, self._fused_ws,
                                         stats=stats, stream=stream)


def scoup_decode_workspace_size(P: int, C: int, D: int) -> int:
    return int(load().scoup_decode_workspace_size(P, C, D))


def scoup_decode(codes, codebook, features, feat_norm2=None, workspace=None, stream=None):
    """Eq. 8: features = codes @ codebook on the tensor cores (bf16 operands, f32 accumulate).

    codes [P, C] float32 or bfloat16; codebook [C, D] float32; features [P, D]
    float32 or bfloat16 (the output type); feat_norm2 [P] float32 (bf16 output
    only) receives the squared norms of the stored rows.  Returns the workspace.
    """
    import torch
    if codes.dtype not in (torch.float32, torch.bfloat16):
        raise TypeError("codes must be float32 or bfloat16")
    if features.dtype not in (torch.float32, torch.bfloat16):
        raise TypeError("features must be float32 or bfloat16")
    _need(codes, codes.dtype, "codes")
    _need(codebook, torch.float32, "codebook")
    _need(features, features.dtype, "features")
    _need(feat_norm2, torch.float32, "feat_norm2")
    P, C = codes.shape
    D = codebook.shape[1]
    if codebook.shape[0] != C or tuple(features.shape) != (P, D):
        raise ValueError("shape mismatch")
    if workspace is None:
        workspace = torch.empty(scoup_decode_workspace_size(P, C, D), dtype=torch.uint8, device=codes.device)
    _need(workspace, torch.uint8, "workspace")
    check(load().scoup_decode(_ptr(codes), 1 if codes.dtype == torch.bfloat16 else 0, P, C, _ptr(codebook), D,
                              _ptr(features), 1 if features.dtype == torch.bfloat16 else 0, _ptr(feat_norm2),
                              _ptr(workspace), workspace.numel(), _stream(stream)))
    return workspace


def scoup_render_decode_workspace_size(n: int, width: int, height: int, C: int, D: int, dup_capacity: int) -> int:
    return int(load().scoup_render_decode_workspace_size(n, width, height, C, D, dup_capacity))


def scoup_render_decode_fused(scene: Scene, topk_idx, topk_val, K: int, C: int, cam, codebook, features,
                              feat_norm2, out_T, out_last, workspace, stats: bool = True, stream=None):
    """Eq. 7 then Eq. 8 for one view in one call: features [H * W, D] = bf16(What) @ codebook.
    out_T / out_last / feat_norm2 may be None.  Returns stats when stats=True."""
    import torch
    _need(topk_idx, torch.int32, "topk_idx")
    _need(topk_val, torch.float32, "topk_val")
    _need(codebook, torch.float32, "codebook")
    if features.dtype not in (torch.float32, torch.bfloat16):
        raise TypeError("features must be float32 or bfloat16")
    _need(features, features.dtype, "features")
    _need(feat_norm2, torch.float32, "feat_norm2")
    _need(out_T, torch.float32, "out_T")
    _need(out_last, torch.int32, "out_last")
    _need(workspace, torch.uint8, "workspace")
    D = int(codebook.shape[1])
    if int(codebook.shape[0]) != int(C) or tuple(features.shape) != (cam.width * cam.height, D):
        raise ValueError("shape mismatch")
    ca = camera_array([cam])
    st = Stats()
    check(load().scoup_render_decode_fused(ct.byref(scene), _ptr(topk_idx), _ptr(topk_val), int(K), int(C),
                                           ct.cast(ca, ct.POINTER(Camera)), _ptr(codebook), D, _ptr(features),
                                           1 if features.dtype == torch.bfloat16 else 0, _ptr(feat_norm2),
                                           _ptr(out_T), _ptr(out_last), _ptr(workspace), workspace.numel(),
                                           ct.byref(st) if stats else None, _stream(stream)))
    return st.as_dict() if stats else None


def scoup_similarity_workspace_size(P: int, D: int, Q: int) -> int:
    return int(load().scoup_similarity_workspace_size(P, D, Q))


def scoup_similarity(features, text, out, feat_norm2=None, workspace=None, stream=None):
    """Cosine similarity out [P, Q] of bf16 features [P, D] to float32 text vectors [Q, D]."""
    import torch
    _need(features, torch.bfloat16, "features")
    _need(text, torch.float32, "text")
    _need(out, torch.float32, "out")
    _need(feat_norm2, torch.float32, "feat_norm2")
    P, D = features.shape
    Q = text.shape[0]
    if text.shape[1] != D or tuple(out.shape) != (P, Q):
        raise ValueError("shape mismatch")
    if workspace is None:
        workspace = torch.empty(scoup_similarity_workspace_size(P, D, Q), dtype=torch.uint8,
                                device=features.device)
    _need(workspace, torch.uint8, "workspace")
    check(load().scoup_similarity(_ptr(features), P, D, _ptr(feat_norm2), _ptr(text), Q, _ptr(out),
                                  _ptr(workspace), workspace.numel(), _stream(stream)))
    return workspace


def scoup_similarity_relevancy(features, text, n_canon: int, R, alpha: float = 10.0, feat_norm2=None,
                               workspace=None, stream=None):
    """Relevancy R [P, Q - n_canon] (Eq. 9) of bf16 features [P, D] for the
    float32 text vectors [Q, D] whose first n_canon rows are the canonical
    phrases, computed in the similarity GEMM's epilogue."""
    import torch
    _need(features, torch.bfloat16, "features")
    _need(text, torch.float32, "text")
    _need(R, torch.float32, "R")
    _need(feat_norm2, torch.float32, "feat_norm2")
    P, D = features.shape
    Q = text.shape[0]
    if text.shape[1] != D or tuple(R.shape) != (P, Q - n_canon):
        raise ValueError("shape mismatch")
    if workspace is None:
        workspace = torch.empty(scoup_similarity_workspace_size(P, D, Q), dtype=torch.uint8,
                                device=features.device)
    _need(workspace, torch.uint8, "workspace")
    check(load().scoup_similarity_relevancy(_ptr(features), P, D, _ptr(feat_norm2), _ptr(text), Q, int(n_canon),
                                            float(alpha), _ptr(R), _ptr(workspace), workspace.numel(),
                                            _stream(stream)))
    return workspace


def scoup_decode_query_workspace_size(P: int, C: int, D: int, Q: int) -> int:
    return int(load().scoup_decode_query_workspace_size(P, C, D, Q))


def scoup_decode_query(codes, codebook, text, out, n_canon: int = 0, alpha: float = 10.0, features=None,
                       feat_norm2=None, workspace=None, stream=None):
    """Eq. 8 decode with the App. B query in the same GEMM: features = codes @
    codebook (bf16 [P, D], or not written when None) and out = the cosine
    similarity [P, Q] to the float32 text vectors [Q, D] (n_canon = 0) or the
    relevancy [P, Q - n_canon] of Eq. 9 (n_canon canonical phrases first).
    Q is 16 or 32.  Returns the workspace."""
    import torch
    if codes.dtype not in (torch.float32, torch.bfloat16):
        raise TypeError("codes must be float32 or bfloat16")
    _need(codes, codes.dtype, "codes")
    _need(codebook, torch.float32, "codebook")
    _need(text, torch.float32, "text")
    _need(out, torch.float32, "out")
    _need(features, torch.bfloat16, "features")
    _need(feat_norm2, torch.float32, "feat_norm2")
    P, C = codes.shape
    D = codebook.shape[1]
    Q = text.shape[0]
    if codebook.shape[0] != C or text.shape[1] != D or tuple(out.shape) != (P, Q - int(n_canon)):
        raise ValueError("shape mismatch")
    if features is not None and tuple(features.shape) != (P, D):
        raise ValueError("features shape mismatch")
    if feat_norm2 is not None and feat_norm2.numel() < P:
        raise ValueError("feat_norm2 too short")
    if workspace is None:
        workspace = torch.empty(scoup_decode_query_workspace_size(P, C, D, Q), dtype=torch.uint8,
                                device=codes.device)
    _need(workspace, torch.uint8, "workspace")
    check(load().scoup_decode_query(_ptr(codes), 1 if codes.dtype == torch.bfloat16 else 0, P, C, _ptr(codebook),
                                    D, _ptr(text), Q, int(n_canon), float(alpha), _ptr(features),
                                    _ptr(feat_norm2), _ptr(out), _ptr(workspace), workspace.numel(),
                                    _stream(stream)))
    return workspace


def scoup_decode_backward(dF, codebook, dcodes, workspace=None, stream=None):
    """dcodes [P, C] = dF [P, D] @ codebook[C, D]^T on the tensor cores (bf16
    operands, FP32 accumulation); dF float32 or bf16.  Returns the workspace."""
    import torch
    if not isinstance(dF, torch.Tensor) or dF.dtype not in (torch.float32, torch.bfloat16):
        raise TypeError("dF must be a float32 or bfloat16 tensor")
    _need(dF, dF.dtype, "dF")
    _need(codebook, torch.float32, "codebook")
    _need(dcodes, torch.float32, "dcodes")
    P, D = dF.shape
    C = codebook.shape[0]
    if codebook.shape[1] != D or tuple(dcodes.shape) != (P, C):
        raise ValueError("shape mismatch")
    if workspace is None:
        workspace = torch.empty(int(load().scoup_decode_backward_workspace_size(P, C, D)), dtype=torch.uint8,
                                device=dF.device)
    _need(workspace, torch.uint8, "workspace")
    check(load().scoup_decode_backward(_ptr(dF), 1 if dF.dtype == torch.bfloat16 else 0, P, D, _ptr(codebook), C,
                                       _ptr(dcodes), _ptr(workspace), workspace.numel(), _stream(stream)))
    return workspace


def scoup_decode_backward_fp32(dF, codebook, dcodes, stream=None) -> None:
    """FP32 SIMT comparison form of scoup_decode_backward."""
    import torch
    for t, nm in ((dF, "dF"), (codebook, "codebook"), (dcodes, "dcodes")):
        _need(t, torch.float32, nm)
    P, D = dF.shape
    C = codebook.shape[0]
    if codebook.shape[1] != D or tuple(dcodes.shape) != (P, C):
        raise ValueError("shape mismatch")
    check(load().scoup_decode_backward_fp32(_ptr(dF), P, D, _ptr(codebook), C, _ptr(dcodes), _stream(stream)))


def scoup_region_l2_grad(F, region_map, code_idx, code_val, codebook, dF, loss=None, workspace=None, stream=None):
    """L2 loss of features F [P, D] (float32 or bf16) against the decoded codes
    of their regions and its gradient dF [P, D] (float32 or bf16); the loss is
    added to the float64 device scalar `loss` when given.  Returns the workspace."""
    import torch
    for t, nm in ((F, "F"), (dF, "dF")):
        if not isinstance(t, torch.Tensor) or t.dtype not in (torch.float32, torch.bfloat16):
            raise TypeError(f"{nm} must be a float32 or bfloat16 tensor")
        _need(t, t.dtype, nm)
    _need(region_map, torch.int32, "region_map")
    _need(code_idx, torch.int32, "code_idx")
    _need(code_val, torch.float32, "code_val")
    _need(codebook, torch.float32, "codebook")
    _need(loss, torch.float64, "loss")
    P, D = F.shape
    R, s = code_idx.shape
    C = codebook.shape[0]
    if tuple(dF.shape) != (P, D) or region_map.numel() != P or codebook.shape[1] != D or code_val.shape != code_idx.shape:
        raise ValueError("shape mismatch")
    if workspace is None:
        workspace = torch.empty(int(load().scoup_region_l2_grad_workspace_size(R, D)), dtype=torch.uint8,
                                device=F.device)
    _need(workspace, torch.uint8, "workspace")
    bf = lambda t: 1 if t.dtype == torch.bfloat16 else 0  # noqa: E731
    check(load().scoup_region_l2_grad(_ptr(F), bf(F), P, D, _ptr(region_map), _ptr(code_idx), _ptr(code_val), R, s,
                                      _ptr(codebook), C, _ptr(dF), bf(dF), _ptr(loss), _ptr(workspace),
                                      workspace.numel(), _stream(stream)))
    return workspace


def scoup_decode_fp32(codes, codebook, features, stream=None) -> None:
    """FP32 SIMT comparison form of scoup_decode: features [P, D] = codes [P, C] @ codebook [C, D]."""
    import torch
    for t, nm in ((codes, "codes"), (codebook, "codebook"), (features, "features")):
        _need(t, torch.float32, nm)
    P, C = codes.shape
    D = codebook.shape[1]
    if codebook.shape[0] != C or tuple(features.shape) != (P, D):
        raise ValueError("shape mismatch")
    check(load().scoup_decode_fp32(_ptr(codes), P, C, _ptr(codebook), D, _ptr(features), _stream(stream)))


def scoup_similarity_fp32(features, text, out, workspace=None, stream=None):
    """FP32 SIMT comparison form of scoup_similarity (float32 features)."""
    import torch
    for t, nm in ((features, "features"), (text, "text"), (out, "out")):
        _need(t, torch.float32, nm)
    P, D = features.shape
    Q = text.shape[0]
    if text.shape[1] != D or tuple(out.shape) != (P, Q):
        raise ValueError("shape mismatch")
    if workspace is None:
        workspace = torch.empty(scoup_similarity_workspace_size(P, D, Q), dtype=torch.uint8,
                                device=features.device)
    _need(workspace, torch.uint8, "workspace")
    check(load().scoup_similarity_fp32(_ptr(features), P, D, _ptr(text), Q, _ptr(out), _ptr(workspace),
                                       workspace.numel(), _stream(stream)))
    return workspace


def scoup_topk_entropy(accum, K: int, topk_idx, topk_val, entropy, comp=None, stream=None) -> None:
    """Eq. 6 Top-K of accum [n, C] plus the entropy [n] of every row's coefficients."""
    import torch
    for t, nm in ((accum, "accum"), (topk_val, "topk_val"), (entropy, "entropy"), (comp, "comp")):
        _need(t, torch.float32, nm)
    _need(topk_idx, torch.int32, "topk_idx")
    n, C = accum.shape
    check(load().scoup_topk_entropy(_ptr(accum), _ptr(comp), n, C, int(K), _ptr(topk_idx), _ptr(topk_val),
                                    _ptr(entropy), _stream(stream)))


def scoup_entropy_filter_workspace_size() -> int:
    return int(load().scoup_entropy_filter_workspace_size())


def scoup_entropy_filter(entropy, keep: int, topk_idx=None, topk_val=None, keep_mask=None, workspace=None,
                         stream=None):
    """Keep the `keep` lowest-entropy Gaussians; clear the others' Top-K rows
    (asynchronous on `stream`; capturable in a CUDA graph with a given workspace)."""
    import torch
    _need(entropy, torch.float32, "entropy")
    _need(topk_idx, torch.int32, "topk_idx")
    _need(topk_val, torch.float32, "topk_val")
    _need(keep_mask, torch.uint8, "keep_mask")
    if workspace is None:
        workspace = torch.empty(int(load().scoup_entropy_filter_workspace_size()), dtype=torch.uint8,
                                device=entropy.device)
        if stream is not None and hasattr(stream, "cuda_stream"):
            workspace.record_stream(stream)  # still in use by the kernels after this call returns
    K = int(topk_idx.shape[1]) if topk_idx is not None else 0
    check(load().scoup_entropy_filter(_ptr(entropy), entropy.numel(), int(keep), K, _ptr(topk_idx),
                                      _ptr(topk_val), _ptr(keep_mask), _ptr(workspace), workspace.numel(),
                                      _stream(stream)))


def scoup_relevancy(sim, n_canon: int, R, alpha: float = 10.0, stream=None) -> None:
    """Eq. 9 relevancy R [P, ncols - n_canon] from similarities sim [P, ncols] (canonical columns first)."""
    import torch
    _need(sim, torch.float32, "sim")
    _need(R, torch.float32, "R")
    P, ncols = sim.shape
    if tuple(R.shape) != (P, ncols - n_canon):
        raise ValueError("R must be [P, ncols - n_canon]")
    check(load().scoup_relevancy(_ptr(sim), P, ncols, int(n_canon), float(alpha), _ptr(R), _stream(stream)))


def scoup_selftest_red_throughput(buf, count: int, seed: int = 1, stream=None) -> None:
    """Enqueues `count` FP32 atomic additions to pseudo-random elements of the
    CUDA float32 tensor buf (whose size must be a power of two, >= 1024)."""
    import torch
    _need(buf, torch.float32, "buf")
    n = buf.numel()
    if n < 1024 or n & (n - 1) or n > (1 << 31):
        raise ValueError("buf must hold a power of two of floats, 2^10 .. 2^31")
    check(load().scoup_selftest_red_throughput(_ptr(buf), n.bit_length() - 1, int(count), int(seed) & 0xffffffff,
                                               _stream(stream)))


def scoup_selftest_gemm_timeout(stream=None) -> tuple:
    """Self-test of the tensor-core pipeline's bounded waits: (status code, message).
    SCOUP_ERR_TIMEOUT is the expected result."""
    import torch
    ws = torch.empty(49408, dtype=torch.uint8, device="cuda")
    rc = load().scoup_selftest_gemm_timeout(_ptr(ws), ws.numel(), _stream(stream))
    msg = load().scoup_last_error()
    return int(rc), (msg.decode() if msg else "")


def scoup_read_stats(workspace, stream=None) -> dict:
    st = Stats()
    check(load().scoup_read_stats(_ptr(workspace), workspace.numel(), ct.byref(st), _stream(stream)))
    return st.as_dict()


def scoup_profile_enable(enable: bool) -> None:
    check(load().scoup_profile_enable(1 if enable else 0))


def scoup_profile_read() -> dict:
    """{phase: (milliseconds, timed launch groups)} since the previous read."""
    ms = np.zeros(_lib.NUM_PHASES, np.float64)
    cnt = np.zeros(_lib.NUM_PHASES, np.int64)
    check(load().scoup_profile_read(ms.ctypes.data_as(ct.c_void_p), cnt.ctypes.data_as(ct.c_void_p),
                                    _lib.NUM_PHASES))
    return {name: (float(ms[i]), int(cnt[i])) for i, name in enumerate(_lib.PHASES) if cnt[i]}


def scoup_launch_count() -> int:
    return int(load().scoup_launch_count())


class Uplift:
    """Holds device copies of one uplift workload and a planned workspace.

    ``wl`` is any object with the fields of ``synth.UpliftWorkload`` (NumPy
    arrays); they are copied to the GPU once.  ``run()`` enqueues one full
    uplift (all views + Top-K) on the current stream.
    """

    def __init__(self, wl, device: str = "cuda", dup_capacity: Optional[int] = None,
                 headroom: float = 1.0, compensated: bool = False, topk: bool = True, chunked: bool = False):
        """chunked=True: run() uses the chunked form (SCOUP_UPLIFT_CHUNKED) and
        the workspace is sized for it."""
        import torch
        dev = torch.device(device)
        sc = wl.scene
        self.means = torch.as_tensor(sc.means, device=dev).contiguous()
        self.scales = torch.as_tensor(sc.scales, device=dev).contiguous()
        self.quats = torch.as_tensor(sc.quats, device=dev).contiguous()
        self.opacity = torch.as_tensor(sc.opacity, device=dev).contiguous()
        self.scene = scene_struct(self.means, self.scales, self.quats, self.opacity)
        self.cams = list(wl.cams)
        self.region_maps = torch.as_tensor(wl.region_maps, device=dev).contiguous()
        self.map_offsets = np.asarray(wl.map_offsets, np.int64)
        self.code_idx = torch.as_tensor(wl.code_idx, device=dev).contiguous()
        self.code_val = torch.as_tensor(wl.code_val, device=dev).contiguous()
        self.R_total = int(wl.code_idx.shape[0])
        self.s, self.C, self.K = int(wl.s), int(wl.C), int(wl.K)
        n = sc.n
        self.n = n
        maxw = max([c.width for c in self.cams] + [1])
        maxh = max([c.height for c in self.cams] + [1])
        extra = 8 * self.R_total * self.K + 1024 if self.s > self.K else 0
        if dup_capacity is None:
            probe = torch.empty(scoup_uplift_workspace_size(n, maxw, maxh, 0) + extra,
                                dtype=torch.uint8, device=dev)
            dup_capacity = int(scoup_uplift_plan(self.scene, self.cams, probe) * headroom) + 1
            del probe
        self.dup_capacity = dup_capacity
        self.chunked = bool(chunked)
        size = scoup_uplift_chunked_workspace_size if self.chunked else scoup_uplift_workspace_size
        self.workspace = torch.empty(size(n, maxw, maxh, dup_capacity) + extra, dtype=torch.uint8, device=dev)
        self.maxw, self.maxh, self.extra, self.device = maxw, maxh, extra, dev
        self._host_ws = None
        self.compensated = bool(compensated)
        self.accum = torch.empty(((2, n, self.C) if compensated else (n, self.C)), dtype=torch.float32,
                                 device=dev)
        self.topk_idx = torch.empty((n, self.K), dtype=torch.int32, device=dev) if topk else None
        self.topk_val = torch.empty((n, self.K), dtype=torch.float32, device=dev) if topk else None

    def run(self, stats: bool = True, accum_mode: int = 0, views=None, stream=None, topk: bool = True):
        """One uplift; topk=False (or an Uplift built with topk=False) accumulates only."""
        topk = topk and self.topk_idx is not None
        cams = self.cams if views is None else [self.cams[v] for v in views]
        offs = self.map_offsets if views is None else self.map_offsets[list(views)]
        if self.compensated:
            accum_mode |= SCOUP_ACCUM_COMPENSATED
        if self.chunked:
            accum_mode |= SCOUP_UPLIFT_CHUNKED
        return scoup_uplift(self.scene, cams, self.region_maps, offs, self.R_total, self.code_idx,
                            self.code_val, self.s, self.C, self.K, self.accum, accum_mode,
                            self.topk_idx if topk else None, self.topk_val if topk else None,
                            self.workspace, stats=stats, stream=stream)

    def run_host_maps(self, host_maps, stats: bool = True, accum_mode: int = 0, stream=None, topk: bool = True,
                      chunked: Optional[bool] = None):
        """One uplift with the region maps read from host memory (host_maps:
        a pinned CPU int32 tensor laid out like region_maps): the copies of
        the views' maps overlap the earlier views' compute.  chunked: the
        form (default: the Uplift's own)."""
        import torch
        topk = topk and self.topk_idx is not None
        chunked = self.chunked if chunked is None else bool(chunked)
        if self._host_ws is None:
            self._host_ws = {}
        if chunked not in self._host_ws:
            size = (scoup_uplift_host_maps_chunked_workspace_size if chunked
                    else scoup_uplift_host_maps_workspace_size)
            self._host_ws[chunked] = torch.empty(size(self.n, self.maxw, self.maxh, self.dup_capacity) + self.extra,
                                                 dtype=torch.uint8, device=self.device)
        if chunked:
            accum_mode |= SCOUP_UPLIFT_CHUNKED
        if self.compensated:
            accum_mode |= SCOUP_ACCUM_COMPENSATED
        return scoup_uplift_host_maps(self.scene, self.cams, host_maps, self.map_offsets, self.R_total,
                                      self.code_idx, self.code_val, self.s, self.C, self.K, self.accum, accum_mode,
                                      self.topk_idx if topk else None, self.topk_val if topk else None,
                                      self._host_ws[chunked], stats=stats, stream=stream)

    def accum_value(self):
        """The accumulator [n, C] (sum + compensation in the compensated form)."""
        if self.compensated:
            return self.accum[0].double() + self.accum[1].double()
        return self.accum


class LevelUplift:
    """L semantic levels (workloads sharing scene, cameras and map offsets) uplifted
    in one pass through scoup_uplift_levels.  accum is [n, L*C] (level l in
    columns l*C..); topk_idx / topk_val are [L, n, K]."""

    def __init__(self, wls, device: str = "cuda", compensated: bool = False, dup_capacity: Optional[int] = None):
        import torch
        dev = torch.device(device)
        self.wls = list(wls)
        self.L = len(self.wls)
        base = self.wls[0]
        self.base = Uplift(base, device=device, dup_capacity=dup_capacity, topk=False)
        self.C, self.K = int(base.C), int(base.K)
        n = base.scene.n
        self.compensated = bool(compensated)
        self.maps, self.ci, self.cv = [], [], []
        self.levels = (Level * self.L)()
        for l, wl in enumerate(self.wls):
            m = torch.as_tensor(wl.region_maps, device=dev).contiguous()
            ci = torch.as_tensor(wl.code_idx, device=dev).contiguous()
            cv = torch.as_tensor(wl.code_val, device=dev).contiguous()
            self.maps.append(m)
            self.ci.append(ci)
            self.cv.append(cv)
            self.levels[l].region_maps, self.levels[l].R_total = _ptr(m), int(wl.code_idx.shape[0])
            self.levels[l].code_idx, self.levels[l].code_val, self.levels[l].s = _ptr(ci), _ptr(cv), int(wl.s)
        shape = (2, n, self.L * self.C) if compensated else (n, self.L * self.C)
        self.accum = torch.empty(shape, dtype=torch.float32, device=dev)
        self.topk_idx = torch.empty((self.L, n, self.K), dtype=torch.int32, device=dev)
        self.topk_val = torch.empty((self.L, n, self.K), dtype=torch.float32, device=dev)

    def run(self, stats: bool = True, topk: bool = True, views=None, stream=None, accum_mode: int = 0):
        b = self.base
        cams = b.cams if views is None else [b.cams[v] for v in views]
        offs = np.ascontiguousarray((b.map_offsets if views is None else b.map_offsets[list(views)])[:max(1, len(cams))])
        ca = camera_array(cams)
        st = Stats()
        mode = accum_mode | (SCOUP_ACCUM_COMPENSATED if self.compensated else 0)
        check(load().scoup_uplift_levels(ct.byref(b.scene), ct.cast(ca, ct.c_void_p), len(cams),
                                         offs.ctypes.data_as(ct.c_void_p), ct.cast(self.levels, ct.c_void_p),
                                         self.L, self.C, self.K, _ptr(self.accum), mode,
                                         _ptr(self.topk_idx) if topk else None,
                                         _ptr(self.topk_val) if topk else None, _ptr(b.workspace),
                                         b.workspace.numel(), ct.byref(st) if stats else None, _stream(stream)))
        return st.as_dict() if stats else None

    def level_accum(self, l: int):
        a = self.accum[0] + self.accum[1] if self.compensated else self.accum
        return a[:, l * self.C:(l + 1) * self.C]


class BatchedUplift:
    """Many uplift workloads (scenes with their own views) run as one batch:
    a plan with per-lane workspaces, an optional autotuning pass and a CUDA
    graph replayed by ``run()``.  Every workload is copied to the GPU once;
    ``accum[b]``, ``topk_idx[b]``, ``topk_val[b]`` hold scene b's outputs."""

    def __init__(self, wls, device: str = "cuda", compensated: bool = False, stream=None):
        import torch
        dev = torch.device(device)
        self.device = dev
        self.wls = list(wls)
        if not self.wls:
            raise ValueError("empty batch")
        self.C, self.K = int(self.wls[0].C), int(self.wls[0].K)
        self.compensated = bool(compensated)
        self._keep = []
        self.accum, self.topk_idx, self.topk_val, self.scenes = [], [], [], []
        items = (BatchItem * len(self.wls))()
        for b, wl in enumerate(self.wls):
            if int(wl.C) != self.C or int(wl.K) != self.K:
                raise ValueError("C and K must be common to the batch")
            sc = wl.scene
            t = {k: torch.as_tensor(getattr(sc, k), device=dev).contiguous()
                 for k in ("means", "scales", "quats", "opacity")}
            sstruct = scene_struct(t["means"], t["scales"], t["quats"], t["opacity"])
            rm = torch.as_tensor(wl.region_maps, device=dev).contiguous()
            ci = torch.as_tensor(wl.code_idx, device=dev).contiguous()
            cv = torch.as_tensor(wl.code_val, device=dev).contiguous()
            cams = camera_array(wl.cams)
            offs = np.ascontiguousarray(np.asarray(wl.map_offsets, np.int64)[:max(1, len(wl.cams))])
            n = sc.n
            acc = torch.empty(((2, n, self.C) if compensated else (n, self.C)), dtype=torch.float32, device=dev)
            ti = torch.empty((n, self.K), dtype=torch.int32, device=dev)
            tv = torch.empty((n, self.K), dtype=torch.float32, device=dev)
            it = items[b]
            it.scene = sstruct
            it.cams = ct.cast(cams, ct.c_void_p)
            it.V = len(wl.cams)
            it.region_maps = _ptr(rm)
            it.map_offsets = offs.ctypes.data_as(ct.c_void_p)
            it.R_total = int(wl.code_idx.shape[0])
            it.code_idx, it.code_val, it.s = _ptr(ci), _ptr(cv), int(wl.s)
            it.accum, it.topk_idx, it.topk_val = _ptr(acc), _ptr(ti), _ptr(tv)
            self._keep += [t, sstruct, rm, ci, cv, cams, offs]
            self.accum.append(acc)
            self.topk_idx.append(ti)
            self.topk_val.append(tv)
            self.scenes.append(sstruct)
        self._items = items
        self.plan = ct.c_void_p()
        mode = SCOUP_ACCUM_COMPENSATED if compensated else 0
        check(load().scoup_plan_create(ct.cast(items, ct.c_void_p), len(self.wls), self.C, self.K, mode,
                                       ct.byref(self.plan), _stream(stream)))

    def autotune(self, sample_views: int = 4, stream=None) -> dict:
        check(load().scoup_autotune(self.plan, int(sample_views), _stream(stream)))
        return self.info()

    def set(self, lanes: int, warp_w: int) -> None:
        check(load().scoup_plan_set(self.plan, int(lanes), int(warp_w)))

    def set_chunk(self, chunk_views: int) -> None:
        """0: scenes on lanes; > 0: chunks of this many views, each composited
        by one persistent tile launch (scoup_plan_set_chunk)."""
        check(load().scoup_plan_set_chunk(self.plan, int(chunk_views)))

    def run(self, eager: bool = False, stream=None) -> None:
        check(load().scoup_uplift_batched(self.plan, SCOUP_BATCH_EAGER if eager else 0, _stream(stream)))

    def stats(self, stream=None) -> list:
        arr = (Stats * len(self.wls))()
        check(load().scoup_plan_stats(self.plan, ct.cast(arr, ct.c_void_p), _stream(stream)))
        return [arr[b].as_dict() for b in range(len(self.wls))]

    def info(self) -> dict:
        pi = PlanInfo()
        check(load().scoup_plan_info_get(self.plan, ct.byref(pi)))
        return {"lanes": pi.lanes, "warp_w": pi.warp_w, "tuned": bool(pi.tuned), "graph_kernels": pi.graph_kernels,
                "workspace_bytes": int(pi.workspace_bytes), "chunk_views": pi.chunk_views,
                "tune": [{"lanes": pi.tune[i].lanes, "warp_w": pi.tune[i].warp_w, "ms": float(pi.tune[i].ms),
                          "chunk_views": pi.tune[i].chunk_views} for i in range(pi.n_tune)]}

    def accum_value(self, b: int):
        if self.compensated:
            return self.accum[b][0].double() + self.accum[b][1].double()
        return self.accum[b]

    def close(self) -> None:
        if getattr(self, "plan", None) is not None and self.plan.value:
            load().scoup_plan_destroy(self.plan)
            self.plan = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


__all__ = ["ScoupError", "SCOUP_ACCUM_CONTINUE", "SCOUP_ACCUM_COMPENSATED", "SCOUP_UPLIFT_CHUNKED", "scene_struct", "camera_array", "scoup_version",
           "scoup_uplift_workspace_size", "scoup_uplift_chunked_workspace_size",
           "scoup_uplift_host_maps_chunked_workspace_size", "scoup_uplift_plan", "scoup_uplift", "scoup_topk",
           "scoup_read_stats", "scoup_uplift_noalloc", "scoup_uplift_noalloc_max_bytes",
           "scoup_profile_enable", "scoup_profile_read", "scoup_launch_count",
           "scoup_render", "scoup_render_backward", "Render", "Uplift",
           "scoup_decode_workspace_size", "scoup_decode", "scoup_similarity_workspace_size",
           "scoup_similarity", "scoup_decode_fp32", "scoup_similarity_fp32", "BatchedUplift",
           "SCOUP_BATCH_EAGER", "LevelUplift", "scoup_selftest_gemm_timeout", "scoup_selftest_red_throughput", "scoup_topk_entropy", "scoup_entropy_filter", "scoup_entropy_filter_workspace_size", "scoup_relevancy",
           "scoup_render_decode_workspace_size", "scoup_render_decode_fused",
           "scoup_uplift_host_maps_workspace_size", "scoup_uplift_host_maps",
           "scoup_similarity_relevancy", "scoup_decode_query", "scoup_decode_query_workspace_size", "scoup_decode_backward", "scoup_decode_backward_fp32",
           "scoup_region_l2_grad"]
