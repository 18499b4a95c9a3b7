"""Argument checks of the Python binding (no GPU: every case below is refused
before the library is called)."""
import numpy as np
import pytest
import torch

import paper_2605_13600_gb300 as gb


def test_host_maps_must_be_a_cpu_int32_tensor():
    scene = gb.Scene() if hasattr(gb, "Scene") else None
    cams = []
    for bad in (np.zeros(4, np.int32), torch.zeros(4, dtype=torch.float32), torch.zeros(8, dtype=torch.int32)[::2]):
        with pytest.raises(TypeError):
            gb.scoup_uplift_host_maps(scene, cams, bad, [0], 1, None, None, 1, 8, 1, None, 0, None, None, None)


def test_cuda_arrays_are_required():
    cpu = torch.zeros((4, 8), dtype=torch.float32)
    with pytest.raises(ValueError, match="CUDA"):
        gb.scoup_topk(cpu, 2, torch.zeros((4, 2), dtype=torch.int32), torch.zeros((4, 2)))
    with pytest.raises(TypeError):
        gb.scoup_topk(cpu.double(), 2, None, None)


def test_relevancy_shape_check():
    sim = torch.zeros((6, 10), dtype=torch.float32)
    with pytest.raises((ValueError, TypeError)):
        gb.scoup_relevancy(sim, 4, torch.zeros((6, 5), dtype=torch.float32))


def test_render_decode_fused_checks_types():
    f = torch.zeros((4, 16), dtype=torch.float16)
    with pytest.raises((TypeError, ValueError)):
        gb.scoup_render_decode_fused(None, None, None, 1, 8, None, torch.zeros((8, 16)), f, None, None, None, None)


@pytest.mark.parametrize("entry", ["scoup_uplift", "scoup_uplift_host_maps", "scoup_uplift_noalloc"])
@pytest.mark.parametrize("mode", [0, gb.SCOUP_ACCUM_COMPENSATED])
def test_uplift_refuses_a_short_accumulator(monkeypatch, entry, mode):
    """An accumulator shorter than n x C (2 n C when compensated) is refused in
    the binding, before the library sees a pointer it would write past."""
    def no_library():
        raise AssertionError("the library must not be called")
    monkeypatch.setattr(gb.scoup, "load", no_library)
    from paper_2605_13600_gb300 import _lib
    scene = _lib.Scene()
    scene.n = 10
    C = 8
    short = torch.zeros(10 * C * (2 if mode else 1) - 1, dtype=torch.float32)
    maps = torch.zeros(4, dtype=torch.int32)
    args = dict(scene=scene, cams=[], map_offsets=[0], R_total=1, code_idx=None, code_val=None, s=1, C=C,
                K=1, accum=short, accum_mode=mode, topk_idx=None, topk_val=None)
    fn = getattr(gb, entry)
    with pytest.raises(ValueError, match="accum is too small"):
        if entry == "scoup_uplift_host_maps":
            fn(host_region_maps=maps, workspace=None, **args)
        elif entry == "scoup_uplift":
            fn(region_maps=maps, workspace=None, **args)
        else:
            fn(region_maps=maps, **args)


def test_every_declared_entry_point_has_a_python_wrapper():
    """Each extern "C" function of include/*.h that takes device arrays is
    reachable from the package (its wrapper is exported)."""
    import os
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    names = set()
    for fn in os.listdir(os.path.join(root, "include")):
        if fn.endswith(".h"):
            src = re.sub(r"/\*.*?\*/", "", open(os.path.join(root, "include", fn)).read(), flags=re.S)
            names |= set(re.findall(r"\b(scoup_[a-z0-9_]+)\s*\(", src))
    host_only = {"scoup_last_error", "scoup_plan_create", "scoup_plan_destroy", "scoup_plan_set", "scoup_plan_set_chunk",
                 "scoup_plan_stats", "scoup_plan_info_get", "scoup_autotune", "scoup_uplift_batched",
                 "scoup_uplift_levels", "scoup_uplift_levels_workspace_size",
                 "scoup_region_l2_grad_workspace_size", "scoup_decode_backward_workspace_size",
                 "scoup_render_workspace_size", "scoup_render_backward_workspace_size"}
    missing = sorted(n for n in names - host_only if not hasattr(gb, n))
    assert not missing, missing
