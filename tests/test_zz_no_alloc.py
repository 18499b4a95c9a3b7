"""scoup_uplift_noalloc: the uplift entry point for callers that cannot
allocate device memory (their host's memory manager owns every allocation
and hands out no scratch buffers).  Its scratch is a fixed array inside the
library; this test calls it twice in a row through the C ABI and checks both
results against scoup_uplift with a caller-provided workspace, at the parity
tolerances of the uplift tests.

The file name sorts last so that a run stopping at its first failure has
already run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import synth
from parity import RTOL, check_topk

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


def _compare(gb, up, wl, ref_acc, ref_idx, ref_val):
    import torch
    acc = torch.empty_like(up.accum)
    ti = torch.empty_like(up.topk_idx)
    tv = torch.empty_like(up.topk_val)
    st = gb.scoup_uplift_noalloc(up.scene, up.cams, up.region_maps, up.map_offsets, up.R_total,
                                 up.code_idx, up.code_val, up.s, up.C, up.K, acc, 0, ti, tv)
    assert st["status"] == 0
    a = acc.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(a, ref_acc, rtol=RTOL, atol=1e-6 * np.abs(ref_acc).max())
    # Top-K sets and values checked the same way as against the oracle, with the
    # workspace result as the reference accumulator (ties within 1e-5 may swap)
    tk = check_topk(ti.cpu().numpy(), tv.cpu().numpy(), ref_acc, np.zeros_like(ref_acc), wl.K)
    assert tk["n_problems"] == 0, tk
    return st


def test_noalloc_matches_workspace_entry_point_twice(gb):
    wl = synth.uplift_cfg1()
    up = gb.Uplift(wl)
    st_ref = up.run(stats=True)
    ref_acc = up.accum.cpu().numpy().astype(np.float64)
    ref_idx = up.topk_idx.cpu().numpy()
    ref_val = up.topk_val.cpu().numpy()
    assert gb.scoup_uplift_noalloc_max_bytes() == 32 << 20
    for _ in range(2):  # the second call starts from the first call's leftovers
        st = _compare(gb, up, wl, ref_acc, ref_idx, ref_val)
        assert st["contributions"] == st_ref["contributions"]
        assert st["listed"] == st_ref["listed"]


def test_noalloc_rejects_scenes_beyond_its_array(gb):
    wl = synth.tiny_workload(41, n=400_000, width=64, height=48, V=1)
    up = gb.Uplift(wl, dup_capacity=16)
    with pytest.raises(gb.ScoupError) as ei:
        gb.scoup_uplift_noalloc(up.scene, up.cams, up.region_maps, up.map_offsets, up.R_total,
                                up.code_idx, up.code_val, up.s, up.C, up.K, up.accum, 0,
                                up.topk_idx, up.topk_val)
    assert ei.value.code == -1 and "fixed array" in str(ei.value)
