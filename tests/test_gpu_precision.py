"""Precision forms: error of every GPU result against the FP64 oracle.

  * uplift accumulator, plain FP32 atomics and the compensated (TwoSum) form;
  * Top-K coefficients of both forms;
  * sparse-code rendering (FP32 accumulate);
  * codebook decode, BF16 tensor cores and the FP32 SIMT comparison form;
  * cosine similarity to text vectors, BF16 and FP32.

Each comparison asserts its bound and records max / mean errors; with
SCOUP_PRECISION_REPORT=<path> set, the table is written there as JSON.
"""
import json
import os

import numpy as np
import pytest

import synth
from parity import check_accum, check_topk

pytestmark = pytest.mark.gpu

REPORT = {}


@pytest.fixture(scope="module")
def gb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_13600_gb300 import build
    build.build()
    import paper_2605_13600_gb300 as gb
    return gb


@pytest.fixture(scope="module", autouse=True)
def _write_report():
    yield
    path = os.environ.get("SCOUP_PRECISION_REPORT")
    if path and REPORT:
        with open(path, "w") as f:
            json.dump(REPORT, f, indent=1, sort_keys=True)


def _rel_stats(got, ref, floor):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    m = np.abs(ref) > floor
    rel = np.abs(got - ref)[m] / np.abs(ref)[m]
    return {"max_rel": float(rel.max()) if rel.size else 0.0, "mean_rel": float(rel.mean()) if rel.size else 0.0,
            "max_abs": float(np.abs(got - ref).max()) if got.size else 0.0, "n": int(m.sum())}


def test_uplift_plain_vs_compensated(gb, cfg1, cfg1_oracle):
    acc, risk = cfg1_oracle["acc"], cfg1_oracle["risk"]
    clear = ~(risk > 0)
    floor = 1e-6 * acc.max()
    out = {}
    for comp in (False, True):
        up = gb.Uplift(cfg1, compensated=comp)
        st = up.run()
        assert st["status"] == 0
        ga = up.accum_value().cpu().numpy()
        info = check_accum(ga, acc, risk)
        assert info["n_bad"] == 0, info
        tk = check_topk(up.topk_idx.cpu().numpy(), up.topk_val.cpu().numpy(), acc, risk, cfg1.K)
        assert tk["n_problems"] == 0, tk
        s = _rel_stats(np.where(clear, ga, acc), acc, floor)
        oidx, oval = cfg1_oracle["idx"], cfg1_oracle["val"]
        same = (np.sort(up.topk_idx.cpu().numpy(), 1) == np.sort(oidx, 1)).all(1)
        tv = _rel_stats(up.topk_val.cpu().numpy()[same], oval[same], 1e-6)
        out["compensated" if comp else "plain"] = (s, tv)
        REPORT[f"uplift_accum_{'compensated' if comp else 'plain'}"] = s
        REPORT[f"uplift_topk_val_{'compensated' if comp else 'plain'}"] = tv
    # On 8 views the summation error is small next to the per-term error of the
    # FP32 weights (an alpha near 0.99 amplifies its rounding into 1 - alpha
    # and into T of everything behind it), so both forms land close together.
    assert out["compensated"][0]["max_rel"] <= out["plain"][0]["max_rel"] * 1.05 + 1e-7
    assert out["compensated"][0]["mean_rel"] <= out["plain"][0]["mean_rel"] * 1.05 + 1e-8


def test_compensation_on_long_sums(gb, oracle_lib):
    """A summation-dominated case: one Gaussian seen head-on from the same
    camera V = 1000 times (one region, one-hot code), so each accumulator entry
    is the sum of V x (tiles) equal-sized partials.  The exact value is V times
    the oracle's single-view sum; the compensated form must stay at the
    per-term error level while the plain form drifts with V."""
    from conftest import axis_camera, make_scene, single_region_workload
    V = 1000
    scene = make_scene([0.0, 0.0, 0.0], [0.05, 0.05, 0.05], [1.0, 0.0, 0.0, 0.0], [0.3])
    cam = axis_camera(96, 96, f=300.0, z=2.0)
    wl1 = single_region_workload(scene, [cam], 4, [(1, 1.0)], 1)
    acc1, _, _ = oracle_lib.uplift(wl1)
    exact = V * acc1[0, 1]
    wl = single_region_workload(scene, [cam] * V, 4, [(1, 1.0)], 1)
    errs = {}
    for comp in (False, True):
        up = gb.Uplift(wl, compensated=comp)
        st = up.run()
        assert st["status"] == 0
        errs[comp] = abs(float(up.accum_value()[0, 1]) - exact) / exact
    REPORT["long_sum_1000_views_rel_err"] = {"plain": errs[False], "compensated": errs[True]}
    assert errs[True] <= 2e-6
    assert errs[True] <= errs[False]


def test_compensated_resume(gb, cfg1, cfg1_oracle):
    """The compensated form over two chunks of views (CONTINUE) equals one pass."""
    up = gb.Uplift(cfg1, compensated=True)
    up.run(views=range(0, 3))
    up.run(views=range(3, 8), accum_mode=gb.SCOUP_ACCUM_CONTINUE)
    info = check_accum(up.accum_value().cpu().numpy(), cfg1_oracle["acc"], cfg1_oracle["risk"])
    assert info["n_bad"] == 0, info


def test_render_error(gb, oracle_lib, cfg1, cfg1_oracle):
    idx = cfg1_oracle["idx"].astype(np.int32)
    val = cfg1_oracle["val"].astype(np.float32)
    r = gb.Render(cfg1.scene, idx, val, cfg1.C, cfg1.cams[:2])
    stats = []
    for v in range(2):
        (W, T, _), st = r.run(v)
        Wo, To, risk, _ = oracle_lib.render(cfg1.scene, idx, val.astype(np.float64), cfg1.C, cfg1.cams[v])
        ok = ~risk
        stats.append(_rel_stats(W.cpu().numpy()[ok], Wo[ok], 1e-6))
    s = {k: max(x[k] for x in stats) if k.startswith("max") else float(np.mean([x[k] for x in stats]))
         for k in stats[0]}
    REPORT["render_codes"] = s
    assert s["max_rel"] <= 1e-3


def test_decode_and_similarity_error(gb, oracle_lib):
    """BF16 tensor-core and FP32 SIMT decode + similarity on rendered-code-like
    inputs against FP64 (the 256 x 512 codebook and 32 text vectors of the
    1920x1080 render workload's recipe)."""
    import torch
    rng = np.random.default_rng(4)
    P, C, D, Q = 4096, 256, 512, 32
    codebook = synth.unit_rows(rng, C, D)
    text = synth.unit_rows(rng, Q, D)
    W = np.zeros((P, C), np.float32)
    for p in range(P):
        k = int(rng.integers(1, 25))
        j = rng.choice(C, size=k, replace=False)
        v = rng.random(k).astype(np.float32)
        W[p, j] = v / v.sum() * float(rng.uniform(0.05, 1.0))
    F64 = oracle_lib.decode(W.astype(np.float64), codebook)
    S64 = oracle_lib.similarity(F64, text)
    dev = torch.device("cuda:0")
    Wd, cbd, td = (torch.from_numpy(x).to(dev) for x in (W, codebook, text))
    fb = torch.empty((P, D), dtype=torch.bfloat16, device=dev)
    n2 = torch.empty((P,), dtype=torch.float32, device=dev)
    gb.scoup_decode(Wd, cbd, fb, n2)
    sb = torch.empty((P, Q), dtype=torch.float32, device=dev)
    gb.scoup_similarity(fb, td, sb, feat_norm2=n2)
    ff = torch.empty((P, D), dtype=torch.float32, device=dev)
    gb.scoup_decode_fp32(Wd, cbd, ff)
    sf = torch.empty((P, Q), dtype=torch.float32, device=dev)
    gb.scoup_similarity_fp32(ff, td, sf)
    torch.cuda.synchronize()
    fb_, ff_, sb_, sf_ = (x.float().cpu().numpy() for x in (fb, ff, sb, sf))

    def cos_rows(a, b):
        return (a * b).sum(1) / (np.linalg.norm(a, axis=1) * np.linalg.norm(b, axis=1))

    feat_cos_err_bf16 = 1.0 - cos_rows(fb_.astype(np.float64), F64)
    feat_cos_err_fp32 = 1.0 - cos_rows(ff_.astype(np.float64), F64)
    rep = {
        "decode_bf16_feature_cosine_err": {"max": float(feat_cos_err_bf16.max()),
                                           "mean": float(feat_cos_err_bf16.mean())},
        "decode_fp32_feature_cosine_err": {"max": float(feat_cos_err_fp32.max()),
                                           "mean": float(feat_cos_err_fp32.mean())},
        "decode_bf16_rel": _rel_stats(fb_, F64, 1e-3),
        "decode_fp32_rel": _rel_stats(ff_, F64, 1e-3),
        "decode_bf16_vs_fp32_max_abs": float(np.abs(fb_ - ff_).max()),
        "similarity_bf16_abs_err": {"max": float(np.abs(sb_ - S64).max()), "mean": float(np.abs(sb_ - S64).mean())},
        "similarity_fp32_abs_err": {"max": float(np.abs(sf_ - S64).max()), "mean": float(np.abs(sf_ - S64).mean())},
    }
    REPORT.update(rep)
    # decoded features within 2e-3 cosine error in BF16; FP32 to rounding level
    assert feat_cos_err_bf16.max() <= 2e-3
    assert feat_cos_err_fp32.max() <= 1e-6
    assert rep["decode_fp32_rel"]["max_rel"] <= 1e-4
    assert rep["similarity_fp32_abs_err"]["max"] <= 1e-5
    # BF16 similarity: four bf16 roundings (codes, codebook, features, text)
    assert rep["similarity_bf16_abs_err"]["max"] <= 4e-2 and rep["similarity_bf16_abs_err"]["mean"] <= 2e-3
