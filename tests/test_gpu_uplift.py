"""GPU uplift (scoup_uplift through the C ABI) vs the FP64 oracle.

Element-by-element parity on seeded inputs small enough for the oracle
(cfg1: 10k Gaussians x 8 views; random scenes with ragged image sizes), edge
cases (empty scene, no views, all culled, unlabelled pixels, s > K, tiles
longer than one sort window), device-side error reporting, resume over
several calls, the chunked form (SCOUP_UPLIFT_CHUNKED: one persistent tile
launch per chunk of views) held to the same oracle with the counters of the
per-view form, and sampled rows of the full 1M-Gaussian x 200-view workload.
"""
import numpy as np
import pytest

import synth
from parity import check_accum, check_topk

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


def _run(gb, wl, **kw):
    up = gb.Uplift(wl, **kw)
    st = up.run(stats=True)
    return up, st


def _parity(gb, oracle_lib, wl, tag="", **kw):
    up, st = _run(gb, wl, **kw)
    acc, risk, cnt = oracle_lib.uplift(wl)
    ga = up.accum.cpu().numpy()
    info = check_accum(ga, acc, risk)
    assert info["n_bad"] == 0, (tag, info)
    tk = check_topk(up.topk_idx.cpu().numpy(), up.topk_val.cpu().numpy(), acc, risk, wl.K)
    assert tk["n_problems"] == 0, (tag, tk)
    # integer counters: equal except where a stop decision is at risk
    assert st["visible"] == cnt["visible"], (tag, st, cnt)
    assert st["duplicates"] == cnt["duplicates"], (tag, st, cnt)
    assert abs(st["contributions"] - cnt["contributions"]) <= 2 * cnt["at_risk"], (tag, st, cnt)
    # the GPU lists only (Gaussian, tile) pairs that can pass the alpha test somewhere in the
    # tile, so it examines at most the pairs the oracle examines over the full rectangles
    assert st["listed"] <= st["duplicates"], (tag, st)
    assert st["evaluated_pairs"] <= cnt["evaluated"] + 64 * cnt["at_risk"], (tag, st, cnt)
    return up, st, acc, risk, cnt, info, tk


def test_cfg1_parity(gb, oracle_lib, cfg1):
    up, st, acc, risk, cnt, info, tk = _parity(gb, oracle_lib, cfg1, "cfg1")
    assert cnt["contributions"] > 1_000_000
    assert info["max_rel_err"] < 1e-4
    print("cfg1", st, info, {k: tk[k] for k in ("n_set_diff", "n_tie_ok", "max_val_rel_err")})


@pytest.mark.parametrize("seed,W,H,n,V,R,C,s,K,lsm", [
    (31, 50, 37, 300, 3, 7, 16, 3, 3, -2.6),      # ragged tail in x and y
    (32, 33, 17, 500, 2, 5, 24, 4, 4, -2.2),
    (33, 130, 70, 2000, 4, 20, 64, 4, 4, -3.0),
    (34, 64, 48, 800, 2, 9, 32, 6, 3, -2.5),      # s > K: per-code Top-K first
    (35, 16, 16, 100, 1, 2, 8, 2, 8, -2.0),       # single tile, K = C
])
def test_random_scene_parity(gb, oracle_lib, seed, W, H, n, V, R, C, s, K, lsm):
    wl = synth.tiny_workload(seed, n=n, width=W, height=H, V=V, R=R, C=C, s=s, K=K,
                             log_scale_mean=lsm)
    _parity(gb, oracle_lib, wl, f"seed{seed}")


def test_long_tile_lists_use_several_windows(gb, oracle_lib):
    """Thousands of Gaussians over a 48x32 image: every tile list is longer
    than one ordering window, so several windows are composited per tile."""
    wl = synth.tiny_workload(36, n=6000, width=48, height=32, V=2, R=4, C=16, s=3, K=3,
                             log_scale_mean=-2.0)
    wl.scene.opacity[:] = np.minimum(wl.scene.opacity, 0.08)  # keep pixels open for long
    up, st, *_ = _parity(gb, oracle_lib, wl, "long")
    assert st["listed"] / (2 * 6) > 1500  # mean listed Gaussians per tile: several 256-key windows


def test_unlabelled_pixels(gb, oracle_lib):
    wl = synth.tiny_workload(37, n=400, width=40, height=40, V=2, R=5, C=12, s=3, K=3,
                             log_scale_mean=-2.5)
    maps = wl.region_maps.copy()
    maps[::3] = -1
    wl.region_maps = maps
    _parity(gb, oracle_lib, wl, "unlabelled")


def test_empty_inputs(gb, oracle_lib):
    import torch
    wl = synth.tiny_workload(38, n=50, width=32, height=32, V=2)
    # no views: accumulators stay zero, Top-K is all padding
    wl0 = synth.UpliftWorkload("noviews", wl.scene, [], np.zeros(1, np.int32), np.zeros(1, np.int64),
                               wl.code_idx, wl.code_val, wl.C, wl.s, wl.K)
    up = gb.Uplift(wl0, dup_capacity=16)
    st = up.run()
    assert st["contributions"] == 0
    assert (up.accum == 0).all() and (up.topk_idx == -1).all() and (up.topk_val == 0).all()
    # no Gaussians
    wln = synth.UpliftWorkload("empty", wl.scene.subset(np.arange(0)), wl.cams, wl.region_maps,
                               wl.map_offsets, wl.code_idx, wl.code_val, wl.C, wl.s, wl.K)
    up = gb.Uplift(wln, dup_capacity=16)
    assert up.run()["contributions"] == 0
    # everything behind the cameras
    far = wl.scene.subset(np.arange(wl.scene.n))
    far.means[:] = np.array([0.0, 0.0, 0.0], np.float32)
    cams = [synth.camera_at([0.0, 0.0, 0.1], 32, 32, target=(0.0, 0.0, 1.0))]
    wlb = synth.UpliftWorkload("culled", far, cams, wl.region_maps[:1024], wl.map_offsets[:2],
                               wl.code_idx, wl.code_val, wl.C, wl.s, wl.K)
    up = gb.Uplift(wlb, dup_capacity=16)
    st = up.run()
    assert st["visible"] == 0 and (up.topk_idx == -1).all()
    torch.cuda.synchronize()


def test_single_gaussian_closed_form(gb):
    """Same closed form as the oracle pin: sum of alpha over pixels with alpha >= 1/255."""
    import math
    from conftest import axis_camera, make_scene, single_region_workload
    f, s, z, o = 48.0, 0.125, 2.0, 0.3125
    cam = axis_camera(64, 48, f=f, z=z)
    scene = make_scene([0, 0, 0], [s, s, s], [1, 0, 0, 0], [o])
    wl = single_region_workload(scene, [cam], C=8, code_pairs=[(5, 1.0)], K=4)
    up, _ = _run(gb, wl)
    sigma2 = (f * s / z) ** 2 + 0.3
    ys, xs = np.mgrid[0:48, 0:64]
    a = o * np.exp(-0.5 * ((xs - 31.5) ** 2 + (ys - 23.5) ** 2) / sigma2)
    expect = a[a >= 1 / 255].sum()
    got = float(up.accum[0, 5])
    assert got == pytest.approx(expect, rel=1e-5)
    assert up.topk_idx[0].tolist() == [5, -1, -1, -1] and float(up.topk_val[0, 0]) == 1.0


@pytest.mark.parametrize("seed,V,W,H,n", [
    (41, 19, 120, 90, 3000),   # chunks of 8, 8 and 3 views on both lanes
    (42, 8, 64, 48, 800),      # exactly one chunk
    (43, 1, 50, 37, 300),      # one view, ragged tiles
    (44, 33, 40, 30, 600),     # five chunks: each lane reuses its view parts
])
def test_chunked_form_parity(gb, oracle_lib, seed, V, W, H, n):
    wl = synth.tiny_workload(seed, n=n, width=W, height=H, V=V, R=9, C=32, s=4, K=4, layout="blobs")
    _parity(gb, oracle_lib, wl, f"chunked seed{seed}", chunked=True)


def test_chunked_form_counters_equal_per_view_form(gb, cfg1):
    """Every counter is a count over the same per-view, per-tile work: the
    merge of the view parts' headers must reproduce the per-view form's."""
    _, a = _run(gb, cfg1)
    _, b = _run(gb, cfg1, chunked=True)
    assert a == b, (a, b)
    wl = synth.tiny_workload(45, n=2000, width=96, height=64, V=21, R=11, C=32, s=4, K=4, layout="blobs")
    _, a = _run(gb, wl)
    _, b = _run(gb, wl, chunked=True)
    assert a == b, (a, b)


def test_chunked_form_compensated_and_s_above_k(gb, oracle_lib):
    wl = synth.tiny_workload(46, n=1500, width=80, height=60, V=11, R=9, C=32, s=6, K=3, layout="blobs")
    up, st = _run(gb, wl, chunked=True, compensated=True)
    acc, risk, cnt = oracle_lib.uplift(wl)
    info = check_accum(up.accum_value().cpu().numpy(), acc, risk)
    assert info["n_bad"] == 0, info
    tk = check_topk(up.topk_idx.cpu().numpy(), up.topk_val.cpu().numpy(), acc, risk, wl.K)
    assert tk["n_problems"] == 0, tk


def test_chunked_form_resume_and_capacity(gb, cfg1):
    up = gb.Uplift(cfg1, chunked=True)
    up.run()
    one = up.accum.clone()
    up.run(views=range(0, 3))
    up.run(views=range(3, 8), accum_mode=1)
    np.testing.assert_allclose(up.accum.cpu().numpy(), one.cpu().numpy(), rtol=2e-6, atol=1e-7)
    small = gb.Uplift(cfg1, dup_capacity=1000, chunked=True)
    with pytest.raises(gb.ScoupError) as ei:
        small.run()
    assert ei.value.code == -4


def test_chunked_form_refuses_levels(gb, cfg1):
    lv = gb.LevelUplift([cfg1, cfg1])
    with pytest.raises(gb.ScoupError) as ei:
        lv.run(accum_mode=gb.SCOUP_UPLIFT_CHUNKED)
    assert ei.value.code == -1


def test_chunked_resume_matches_one_shot(gb, cfg1):
    up = gb.Uplift(cfg1)
    up.run()
    one = up.accum.clone()
    idx1 = up.topk_idx.clone()
    up.run(views=range(0, 3))
    up.run(views=range(3, 8), accum_mode=1)
    np.testing.assert_allclose(up.accum.cpu().numpy(), one.cpu().numpy(), rtol=2e-6, atol=1e-7)
    assert (up.topk_idx != idx1).sum().item() <= 4


def test_capacity_overflow_is_reported(gb, cfg1):
    up = gb.Uplift(cfg1, dup_capacity=1000)
    with pytest.raises(gb.ScoupError) as ei:
        up.run()
    assert ei.value.code == -4


def test_bad_region_id_is_reported(gb):
    wl = synth.tiny_workload(39, n=100, width=32, height=32, V=1, R=3)
    wl.region_maps = wl.region_maps.copy()
    wl.region_maps[100] = 999
    up = gb.Uplift(wl)
    with pytest.raises(gb.ScoupError) as ei:
        up.run()
    assert ei.value.code == -5


def test_topk_kernel_against_oracle(gb, oracle_lib):
    import torch
    rng = np.random.default_rng(5)
    for C, K in ((64, 4), (256, 8), (100, 7), (1000, 16), (24, 24)):
        acc = (rng.exponential(1.0, (3000, C)) * (rng.random((3000, C)) < 0.3)).astype(np.float32)
        acc[7] = 0
        acc[8, :5] = 2.0  # exact ties -> lower atom first
        a = torch.as_tensor(acc, device="cuda")
        ti = torch.empty((3000, K), dtype=torch.int32, device="cuda")
        tv = torch.empty((3000, K), dtype=torch.float32, device="cuda")
        gb.scoup_topk(a, K, ti, tv)
        oi, ov = oracle_lib.topk(acc.astype(np.float64), K)
        assert (ti.cpu().numpy() == oi).all()
        np.testing.assert_allclose(tv.cpu().numpy(), ov, rtol=2e-6, atol=1e-7)


def _cfg2_rows(wl, rng):
    """256 rows of the 1M-Gaussian workload: 128 seeded random Gaussians, 64
    whose view-0 means fall in the 16 tiles holding the most means (the longest
    tile lists), 64 in view-0 tiles with more than 4 regions (the pixels whose
    regions get no slot and scatter directly).  Chosen from the inputs alone."""
    import torch
    cam = wl.cams[0]
    vm = np.asarray(cam.viewmat, np.float64).reshape(3, 4)
    t = wl.scene.means.astype(np.float64) @ vm[:, :3].T + vm[:, 3]
    vis = t[:, 2] > 0.2
    mx = cam.fx * t[:, 0] / np.where(vis, t[:, 2], 1.0) + cam.cx - 0.5
    my = cam.fy * t[:, 1] / np.where(vis, t[:, 2], 1.0) + cam.cy - 0.5
    gx, gy = (cam.width + 15) // 16, (cam.height + 15) // 16
    inside = vis & (mx >= 0) & (mx < cam.width) & (my >= 0) & (my < cam.height)
    tile = np.where(inside, (my // 16).astype(np.int64) * gx + (mx // 16).astype(np.int64), -1)
    counts = np.bincount(tile[tile >= 0], minlength=gx * gy)
    dense = np.argsort(-counts)[:16]
    m = torch.as_tensor(wl.region_maps[:cam.width * cam.height]).reshape(cam.height, cam.width).cpu()
    pad = torch.full((gy * 16, gx * 16), -2, dtype=m.dtype)
    pad[:cam.height, :cam.width] = m
    blocks = pad.reshape(gy, 16, gx, 16).permute(0, 2, 1, 3).reshape(gx * gy, 256)
    srt = torch.sort(blocks, dim=1).values
    distinct = ((srt[:, 1:] != srt[:, :-1]) & (srt[:, 1:] >= 0)).sum(1) + (srt[:, 0] >= 0).long()
    many = np.nonzero(distinct.numpy() > 4)[0]
    picks = [rng.choice(wl.scene.n, 128, replace=False)]
    for t_ in dense:
        cand = np.nonzero(tile == t_)[0]
        picks.append(rng.choice(cand, min(4, len(cand)), replace=False))
    cand = np.nonzero(np.isin(tile, many))[0]
    assert len(many) > 0 and len(cand) >= 64
    picks.append(rng.choice(cand, 64, replace=False))
    return np.unique(np.concatenate(picks))


@pytest.mark.slow
@pytest.mark.parametrize("chunked", [True, False])
def test_cfg2_full_size_sampled_rows(gb, oracle_lib, chunked):
    """Full 1M-Gaussian x 200-view x 988x731 uplift in the benchmark's launch
    configuration (the chunked form) and in the per-view form; 256 rows
    (random, from the densest tiles and from tiles of more than 4 regions)
    checked against the oracle over all 200 views."""
    import torch
    wl = synth.uplift_cfg2(device="cuda")
    up = gb.Uplift(wl, chunked=chunked)
    st = up.run()
    assert st["status"] == 0 and st["contributions"] > 1e9
    acc_g = up.accum
    rows = _cfg2_rows(wl, np.random.default_rng(0))
    assert len(rows) >= 250
    acc, risk, cnt = oracle_lib.uplift(wl, rows=rows)
    ga = acc_g[torch.as_tensor(rows, device="cuda")].cpu().numpy()
    info = check_accum(ga, acc, risk)
    assert info["n_bad"] == 0, info
    tk = check_topk(up.topk_idx.cpu().numpy()[rows], up.topk_val.cpu().numpy()[rows], acc, risk, wl.K)
    assert tk["n_problems"] == 0, tk
    print("cfg2 sampled", info, st)


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("chunked", [False, True])
def test_host_region_maps(gb, oracle_lib, cfg1, cfg1_oracle, pinned, chunked):
    """scoup_uplift_host_maps: cfg1's 8 views staged from host memory through a
    4-slot device ring (every slot reused; in the chunked form one slot per
    view part) against the oracle, and against scoup_uplift on device maps
    (equal counters and Top-K; accumulators equal up to the order of FP32
    atomic additions)."""
    import torch
    up = gb.Uplift(cfg1, chunked=chunked)
    st_dev = up.run()
    acc_dev = up.accum.clone()
    idx_dev = up.topk_idx.clone()
    host = torch.as_tensor(np.asarray(cfg1.region_maps, np.int32)).contiguous()
    if pinned:
        host = host.pin_memory()
    st = up.run_host_maps(host)
    assert st["status"] == 0
    for k in ("visible", "duplicates", "evaluated_pairs", "contributions"):
        assert st[k] == st_dev[k], k
    info = check_accum(up.accum.cpu().numpy(), cfg1_oracle["acc"], cfg1_oracle["risk"])
    assert info["n_bad"] == 0, info
    tk = check_topk(up.topk_idx.cpu().numpy(), up.topk_val.cpu().numpy(), cfg1_oracle["acc"], cfg1_oracle["risk"],
                    cfg1.K)
    assert tk["n_problems"] == 0, tk
    np.testing.assert_allclose(up.accum.cpu().numpy(), acc_dev.cpu().numpy(), rtol=2e-6, atol=1e-7)
    assert (up.topk_idx != idx_dev).sum().item() <= 4


@pytest.mark.parametrize("chunked,V", [(False, 9), (True, 9), (True, 37)])
def test_host_region_maps_ragged_views(gb, oracle_lib, chunked, V):
    """Views of a ragged-size scene staged from host maps: nine views (the
    4-slot ring wraps twice; in the chunked form one chunk per lane), and 37
    views in the chunked form (five chunks: every lane's 8 slots refilled
    after the lane's previous drain)."""
    import torch
    wl = synth.tiny_workload(36, n=1500, width=70, height=45, V=V, R=12, C=32, s=4, K=4, log_scale_mean=-2.7)
    up = gb.Uplift(wl, chunked=chunked)
    st = up.run_host_maps(torch.as_tensor(np.asarray(wl.region_maps, np.int32)).contiguous().pin_memory())
    assert st["status"] == 0
    acc, risk, cnt = oracle_lib.uplift(wl)
    info = check_accum(up.accum.cpu().numpy(), acc, risk)
    assert info["n_bad"] == 0, info
    assert abs(st["contributions"] - cnt["contributions"]) <= 2 * cnt["at_risk"]


def _sheet_workload(n=1200, seed=61, opacity=0.05):
    """A fronto-parallel sheet: every Gaussian at exactly the same camera depth
    (3.0), spread over a few tiles around the image centre, so each of those
    tiles holds hundreds of keys in one depth bucket and the front-to-back
    order rests on the index tie-break alone."""
    from conftest import axis_camera, make_scene
    rng = np.random.default_rng(seed)
    means = np.zeros((n, 3))
    means[:, :2] = rng.uniform(-0.8, 0.8, size=(n, 2))
    scales = np.full((n, 3), 0.05)
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    scene = make_scene(means, scales, q, np.full(n, opacity))
    cam = axis_camera(width=64, height=48, f=50.0, z=3.0)
    maps, offs, rpv, R_tot = synth.scenes._pack_maps(synth.scenes._draw_seeds(rng, [cam], [5]), [cam], "cpu")
    ci, cv = synth.region_codes(rng, R_tot, 16, 3)
    return synth.UpliftWorkload("sheet", scene, [cam], maps, offs, ci, cv, 16, 3, 3, rpv)


def test_equal_depth_sheet_splits_buckets(gb, oracle_lib):
    """Hundreds of keys per tile at one depth: the ordering cuts windows out of
    a single oversize depth bucket (radix select on the keys, index
    tie-break); the result still matches the oracle's (depth, index) order."""
    wl = _sheet_workload()
    up, st, *_ = _parity(gb, oracle_lib, wl, "sheet")
    assert st["split_windows"] > 0, st
