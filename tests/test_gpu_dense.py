"""Dense feature uplift (Eq. 3) on the sparse-uplift kernels vs the FP64 oracle.

Each region's D-dimensional feature is written as a code over D + 1 atoms
(features in atoms 0..D-1, a constant 1 in atom D), so an accumulate-only
uplift yields sum e F_v(p) and Z_i = sum e in one pass; f_i is their ratio.
"""
import numpy as np
import pytest

import synth

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


@pytest.mark.parametrize("D", [48, 96])
def test_dense_uplift_matches_oracle(gb, oracle_lib, D):
    base = synth.tiny_workload(401 + D, n=1500, width=96, height=72, V=3, R=10, C=16, s=3, K=3, layout="blobs")
    wl = synth.dense_feature_codes(base, D=D, seed=D)
    up = gb.Uplift(wl, topk=False)
    st = up.run()
    assert st["status"] == 0
    ga = up.accum.cpu().numpy().astype(np.float64)
    acc, risk, cnt = oracle_lib.uplift(wl)
    # features are signed, so entries cancel: bound the error by the
    # magnitude sum e |F| (the same uplift of |codes|) and its risk
    wl_abs = synth.UpliftWorkload(wl.name + "_abs", wl.scene, wl.cams, wl.region_maps, wl.map_offsets,
                                  wl.code_idx, np.abs(wl.code_val), wl.C, wl.s, wl.K, wl.regions_per_view)
    mag, risk_abs, _ = oracle_lib.uplift(wl_abs)
    tol = 1e-4 * mag + risk_abs + 1e-6 * mag.max(axis=1, keepdims=True) + 1e-30
    err = np.abs(ga - acc)
    assert (err <= tol).all(), (np.argwhere(err > tol)[:3], float((err - tol).max()))
    # the normalised feature f_i = acc[:D] / Z_i (Eq. 3) on Gaussians whose stops are clear
    Z = acc[:, D]
    clear = (Z > 1e-6) & ~(risk_abs > 0).any(axis=1)
    f_ora = acc[clear, :D] / Z[clear, None]
    f_gpu = ga[clear, :D] / ga[clear, D:D + 1]
    f_tol = 2e-4 * mag[clear, :D] / Z[clear, None] + 1e-7
    assert (np.abs(f_gpu - f_ora) <= f_tol).all()


def test_dense_normaliser_is_weight_sum(gb):
    """Column D of the dense form equals the weights-only uplift (one-hot code)."""
    import torch
    base = synth.tiny_workload(450, n=800, width=64, height=48, V=2, R=6, C=16, s=3, K=3)
    wl = synth.dense_feature_codes(base, D=40, seed=3)
    up = gb.Uplift(wl, topk=False)
    up.run()
    one = synth.UpliftWorkload("weights_only", base.scene, base.cams, base.region_maps, base.map_offsets,
                               np.zeros((base.code_idx.shape[0], 1), np.int32),
                               np.ones((base.code_idx.shape[0], 1), np.float32), 1, 1, 1,
                               base.regions_per_view)
    uw = gb.Uplift(one, topk=False)
    uw.run()
    torch.testing.assert_close(up.accum[:, 40], uw.accum[:, 0], rtol=1e-5, atol=1e-7)
