"""scoup_uplift_noalloc: the uplift entry point for callers that cannot
allocate device memory (their host's memory manager owns every allocation
and hands out no scratch buffers).  Its scratch is a fixed array inside the
library.  These tests call it through the C ABI: twice in a row against
scoup_uplift with a caller-provided workspace and against the FP64 oracle,
in the continue and compensated accumulation modes, on a side stream, and
with a view whose tile lists do not fit the array's remainder
(SCOUP_ERR_CAPACITY, after which a normal call still succeeds).

The file name sorts last so that a run stopping at its first failure has
already run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import synth
from parity import ATOL_REL, RTOL, check_accum, check_topk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_13600_gb300 import build
    build.build()
    import paper_2605_13600_gb300 as gb
    return gb


def _noalloc(gb, up, accum, mode=0, stream=None):
    import torch
    ti = torch.empty_like(up.topk_idx)
    tv = torch.empty_like(up.topk_val)
    st = gb.scoup_uplift_noalloc(up.scene, up.cams, up.region_maps, up.map_offsets, up.R_total,
                                 up.code_idx, up.code_val, up.s, up.C, up.K, accum, mode, ti, tv,
                                 stream=stream)
    return st, ti, tv


def _compare(gb, up, wl, ref_acc, stream=None):
    import torch
    acc = torch.empty_like(up.accum)
    st, ti, tv = _noalloc(gb, up, acc, stream=stream)
    assert st["status"] == 0
    a = acc.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(a, ref_acc, rtol=RTOL, atol=1e-6 * np.abs(ref_acc).max())
    # Top-K sets and values checked the same way as against the oracle, with the
    # workspace result as the reference accumulator (ties within 1e-5 may swap)
    tk = check_topk(ti.cpu().numpy(), tv.cpu().numpy(), ref_acc, np.zeros_like(ref_acc), wl.K)
    assert tk["n_problems"] == 0, tk
    return st, acc, ti, tv


def test_noalloc_matches_workspace_entry_point_twice(gb):
    wl = synth.uplift_cfg1()
    up = gb.Uplift(wl)
    st_ref = up.run(stats=True)
    ref_acc = up.accum.cpu().numpy().astype(np.float64)
    assert gb.scoup_uplift_noalloc_max_bytes() == 32 << 20
    for _ in range(2):  # the second call starts from the first call's leftovers
        st, *_ = _compare(gb, up, wl, ref_acc)
        assert st["contributions"] == st_ref["contributions"]
        assert st["listed"] == st_ref["listed"]


def test_noalloc_matches_the_oracle(gb, oracle_lib, cfg1, cfg1_oracle):
    import torch
    up = gb.Uplift(cfg1)
    acc = torch.empty_like(up.accum)
    st, ti, tv = _noalloc(gb, up, acc)
    assert st["status"] == 0
    ora, risk = cfg1_oracle["acc"], cfg1_oracle["risk"]
    info = check_accum(acc.cpu().numpy(), ora, risk)
    assert info["n_bad"] == 0, info
    tk = check_topk(ti.cpu().numpy(), tv.cpu().numpy(), ora, risk, cfg1.K)
    assert tk["n_problems"] == 0, tk
    cnt = cfg1_oracle["counts"]
    assert abs(st["contributions"] - cnt["contributions"]) <= 2 * cnt["at_risk"]


def test_noalloc_continue_and_compensated_modes(gb):
    import torch
    wl = synth.uplift_cfg1()
    # continue: a second call adds the same views again on top of the first
    up = gb.Uplift(wl)
    up.run(stats=True)
    ref = up.accum.cpu().numpy().astype(np.float64)
    acc = torch.empty_like(up.accum)
    assert _noalloc(gb, up, acc)[0]["status"] == 0
    assert _noalloc(gb, up, acc, mode=gb.SCOUP_ACCUM_CONTINUE)[0]["status"] == 0
    np.testing.assert_allclose(acc.cpu().numpy(), 2 * ref, rtol=2 * RTOL, atol=2 * ATOL_REL * np.abs(ref).max())
    # compensated: sums and compensation terms against the workspace call's
    upc = gb.Uplift(wl, compensated=True)
    upc.run(stats=True)
    refc = upc.accum.cpu().numpy().astype(np.float64)
    accc = torch.empty_like(upc.accum)
    st, ti, tv = _noalloc(gb, upc, accc, mode=gb.SCOUP_ACCUM_COMPENSATED)
    assert st["status"] == 0
    got = accc.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(got[0] + got[1], refc[0] + refc[1], rtol=RTOL, atol=1e-6 * np.abs(refc[0]).max())
    # the compensation terms are rounding errors of the sums: tiny against them
    assert np.abs(got[1]).max() <= 1e-5 * np.abs(got[0]).max()


def test_noalloc_capacity_error_then_side_stream_call(gb):
    import torch
    budget = gb.scoup_uplift_noalloc_max_bytes()
    # the fixed part fits the array, the tile lists of the one view do not: the
    # Gaussians are so large that even the nearest 5% of them list more
    # (Gaussian, tile) pairs than the rest of the array holds
    big = synth.tiny_workload(43, n=60_000, width=1280, height=720, V=1, R=16, C=32, s=4, K=4,
                              log_scale_mean=-1.0)
    upb = gb.Uplift(big)  # plans its own workspace: the exact pair count of the view
    fixed = gb.scoup_uplift_workspace_size(big.scene.n, 1280, 720, 0)
    assert fixed < budget
    assert upb.dup_capacity * 8 > budget - fixed  # precondition: the lists overflow the remainder
    with pytest.raises(gb.ScoupError) as ei:
        _noalloc(gb, upb, upb.accum)
    assert ei.value.code == -4  # SCOUP_ERR_CAPACITY
    del upb
    # a normal call afterwards, on a side stream, reuses the array's leftovers
    wl = synth.uplift_cfg1()
    up = gb.Uplift(wl)
    up.run(stats=True)
    ref_acc = up.accum.cpu().numpy().astype(np.float64)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        _compare(gb, up, wl, ref_acc, stream=side)


def test_noalloc_rejects_scenes_beyond_its_array(gb):
    wl = synth.tiny_workload(41, n=400_000, width=64, height=48, V=1)
    up = gb.Uplift(wl, dup_capacity=16)
    with pytest.raises(gb.ScoupError) as ei:
        gb.scoup_uplift_noalloc(up.scene, up.cams, up.region_maps, up.map_offsets, up.R_total,
                                up.code_idx, up.code_val, up.s, up.C, up.K, up.accum, 0,
                                up.topk_idx, up.topk_val)
    assert ei.value.code == -1 and "fixed array" in str(ei.value)
