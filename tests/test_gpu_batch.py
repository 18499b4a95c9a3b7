"""Batched uplift (many scenes, one plan, one CUDA graph) vs the FP64 oracle.

Every scene of a batch must give the results of its own plain uplift: the
batch only changes which streams the launches run on, the order of FP32
sums and the tile kernel's warp block shape.  The chunked form (one
persistent tile launch per chunk of views of several scenes) is held to the
same oracle, and its per-scene counters to those of the per-scene form.
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


def _uneven_batch():
    """Scenes of uneven size and resolution (C, s, K common)."""
    return [
        synth.tiny_workload(301, n=3000, width=160, height=120, V=5, R=12, C=64, s=4, K=4, layout="blobs"),
        synth.tiny_workload(302, n=200, width=33, height=17, V=3, R=4, C=64, s=4, K=4),
        synth.tiny_workload(303, n=6000, width=200, height=150, V=2, R=20, C=64, s=4, K=4, layout="blobs",
                            log_scale_mean=-3.5),
        synth.tiny_workload(304, n=800, width=64, height=48, V=7, R=6, C=64, s=4, K=4),
    ]


@pytest.fixture(scope="module")
def batch_oracle(oracle_lib):
    wls = _uneven_batch()
    out = []
    for wl in wls:
        acc, risk, cnt = oracle_lib.uplift(wl)
        out.append((acc, risk, cnt))
    return wls, out


def _check_batch(bu, wls, oracle_out, tag):
    stats = bu.stats()
    for b, (wl, (acc, risk, cnt)) in enumerate(zip(wls, oracle_out)):
        st = stats[b]
        assert st["status"] == 0, (tag, b, st)
        assert abs(st["contributions"] - cnt["contributions"]) <= 2 * cnt["at_risk"], (tag, b, st, cnt)
        info = check_accum(bu.accum_value(b).cpu().numpy(), acc, risk)
        assert info["n_bad"] == 0, (tag, b, info)
        tk = check_topk(bu.topk_idx[b].cpu().numpy(), bu.topk_val[b].cpu().numpy(), acc, risk, wl.K)
        assert tk["n_problems"] == 0, (tag, b, tk)


@pytest.mark.parametrize("lanes", [1, 2, 4])
def test_batch_graph_parity(gb, batch_oracle, lanes):
    wls, ora = batch_oracle
    bu = gb.BatchedUplift(wls)
    bu.set(lanes, 8)
    bu.run()
    _check_batch(bu, wls, ora, f"graph lanes={lanes}")
    info = bu.info()
    assert info["graph_kernels"] > 0
    # a replay of the captured graph recomputes everything from zero
    for acc in bu.accum:
        acc.fill_(123.0)
    bu.run()
    _check_batch(bu, wls, ora, f"replay lanes={lanes}")
    bu.close()


@pytest.mark.parametrize("warp_w", [4, 8, 16])
def test_batch_eager_warp_shapes(gb, batch_oracle, warp_w):
    wls, ora = batch_oracle
    bu = gb.BatchedUplift(wls)
    bu.set(2, warp_w)
    bu.run(eager=True)
    _check_batch(bu, wls, ora, f"eager warp_w={warp_w}")
    bu.close()


def test_batch_autotune(gb, batch_oracle):
    wls, ora = batch_oracle
    bu = gb.BatchedUplift(wls)
    info = bu.autotune(sample_views=2)
    # lanes {1, 2, 4} x warp blocks {8, 16, 4}, then chunks {4, 8, 16} x lanes {1, 2, 4}
    assert info["tuned"] and len(info["tune"]) == 18
    assert sorted((t["chunk_views"], t["lanes"]) for t in info["tune"][9:]) == [
        (c, l) for c in (4, 8, 16) for l in (1, 2, 4)]
    best = min(info["tune"], key=lambda t: t["ms"])
    assert (info["lanes"], info["warp_w"], info["chunk_views"]) == (best["lanes"], best["warp_w"],
                                                                    best["chunk_views"])
    bu.run()
    _check_batch(bu, wls, ora, "tuned")
    bu.close()


def test_batch_compensated(gb, batch_oracle):
    wls, ora = batch_oracle
    bu = gb.BatchedUplift(wls, compensated=True)
    bu.run()
    _check_batch(bu, wls, ora, "compensated")
    bu.close()


@pytest.mark.parametrize("chunk,lanes", [(1, 1), (3, 2), (4, 1), (16, 2), (64, 1)])
def test_batch_chunked_parity(gb, batch_oracle, chunk, lanes):
    """One persistent tile launch per chunk: chunks of one view, chunks that
    mix scenes, a chunk holding the whole batch; a graph replay recomputes
    everything from zero."""
    wls, ora = batch_oracle
    bu = gb.BatchedUplift(wls)
    bu.set(lanes, 8)
    bu.set_chunk(chunk)
    bu.run()
    _check_batch(bu, wls, ora, f"chunked {chunk}x{lanes}")
    info = bu.info()
    assert info["chunk_views"] == chunk and info["graph_kernels"] > 0
    for acc in bu.accum:
        acc.fill_(123.0)
    bu.run()
    _check_batch(bu, wls, ora, f"chunked replay {chunk}x{lanes}")
    bu.close()


def test_batch_chunked_counters_match_per_scene_form(gb, batch_oracle):
    """Every per-scene counter (visible, listed, evaluated, contributions,
    flushes, atomics, ...) is a count over the same per-view, per-tile work in
    both forms: the merge of the views' headers must give them exactly."""
    wls, _ = batch_oracle
    a = gb.BatchedUplift(wls)
    a.set(2, 8)
    a.run(eager=True)
    sa = a.stats()
    b = gb.BatchedUplift(wls)
    b.set(2, 8)
    b.set_chunk(5)
    b.run(eager=True)
    sb = b.stats()
    for k, (x, y) in enumerate(zip(sa, sb)):
        assert x == y, (k, x, y)
    a.close()
    b.close()


@pytest.mark.parametrize("warp_w", [4, 16])
def test_batch_chunked_eager_warp_shapes(gb, batch_oracle, warp_w):
    wls, ora = batch_oracle
    bu = gb.BatchedUplift(wls)
    bu.set(2, warp_w)
    bu.set_chunk(4)
    bu.run(eager=True)
    _check_batch(bu, wls, ora, f"chunked eager warp_w={warp_w}")
    bu.close()


def test_batch_chunked_compensated(gb, batch_oracle):
    wls, ora = batch_oracle
    bu = gb.BatchedUplift(wls, compensated=True)
    bu.set(2, 8)
    bu.set_chunk(3)
    bu.run()
    _check_batch(bu, wls, ora, "chunked compensated")
    bu.close()


def test_batch_chunk_argument_checked(gb, batch_oracle):
    wls, _ = batch_oracle
    bu = gb.BatchedUplift(wls)
    for bad in (-1, 65):
        with pytest.raises(gb.ScoupError):
            bu.set_chunk(bad)
    bu.close()


@pytest.mark.parametrize("chunk", [0, 2])
def test_batch_with_empty_scenes(gb, oracle_lib, chunk):
    """A scene with no Gaussians and a scene with no views ride along."""
    full = synth.tiny_workload(311, n=500, width=48, height=40, V=2, R=5, C=16, s=3, K=3)
    empty_n = synth.tiny_workload(312, n=1, width=48, height=40, V=2, R=5, C=16, s=3, K=3)
    empty_n.scene = empty_n.scene.subset(np.arange(0))
    no_views = synth.tiny_workload(313, n=300, width=48, height=40, V=1, R=5, C=16, s=3, K=3)
    no_views.cams = []
    no_views.map_offsets = no_views.map_offsets[:1]
    wls = [full, empty_n, no_views]
    bu = gb.BatchedUplift(wls)
    bu.set_chunk(chunk)
    bu.run()
    st = bu.stats()
    assert all(s["status"] == 0 for s in st)
    acc, risk, cnt = oracle_lib.uplift(full)
    assert check_accum(bu.accum[0].cpu().numpy(), acc, risk)["n_bad"] == 0
    assert bu.accum[1].numel() == 0
    assert (bu.accum[2] == 0).all() and (bu.topk_idx[2] == -1).all()
    bu.close()


@pytest.mark.parametrize("chunk", [None, 8])
def test_cfg3_full_size_scenes_sampled_rows(gb, oracle_lib, chunk):
    """Two scenes of the 16-scene batch at full size (342k Gaussians x 58
    views at 680 x 508 and 229k x 72 views at 832 x 622, C = 256, s = K = 8)
    in one autotuned batched graph (or the chunked form, 8 views per chunk on
    two lanes); 8 seeded rows per scene against the oracle."""
    import torch
    wls = [synth.uplift_cfg3_scene(b, device="cuda") for b in (9, 6)]
    bu = gb.BatchedUplift(wls)
    if chunk is None:
        bu.autotune(sample_views=2)
    else:
        bu.set(2, 8)
        bu.set_chunk(chunk)
    bu.run()
    stats = bu.stats()
    for b, wl in enumerate(wls):
        assert stats[b]["status"] == 0, (b, stats[b])
        rows = np.sort(np.random.default_rng(9 + b).choice(wl.scene.n, 8, replace=False))
        acc, risk, cnt = oracle_lib.uplift(wl, rows=rows)
        ga = bu.accum_value(b)[torch.as_tensor(rows, device="cuda")].cpu().numpy()
        info = check_accum(ga, acc, risk)
        assert info["n_bad"] == 0, (b, info)
        tk = check_topk(bu.topk_idx[b].cpu().numpy()[rows], bu.topk_val[b].cpu().numpy()[rows], acc, risk, wl.K)
        assert tk["n_problems"] == 0, (b, tk)
    bu.close()
