"""GPU sparse-code rendering (scoup_render, Eq. 7) vs the FP64 oracle.

Per pixel the dense C-vector, the final transmittance and the contribution
count are compared on seeded scenes with ragged image sizes, a one-hot round
trip, long tile lists (several windows), and Top-K codes from the oracle's
uplift.  Code rows up to 256 wide (Top-K up to 16) take the tensor-core
kernel; wider rows, and any shape with SCOUP_RENDER_SIMT=1, the SIMT kernel,
which is checked here on the same cases.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

RTOL = 1e-4


@pytest.fixture(scope="module")
def gb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_13600_gb300 import build
    build.build()
    import paper_2605_13600_gb300 as gb
    return gb


def check_render(What_g, T_g, What_o, T_o, risk):
    """Strict on pixels whose stop decision is clear, loose where it is at risk."""
    err = np.abs(What_g.astype(np.float64) - What_o)
    scale = np.abs(What_o).max(axis=-1, keepdims=True)
    tol = RTOL * np.abs(What_o) + 1e-6 * scale + 1e-7
    tol = np.where(risk[..., None], 1e-2 + tol, tol)
    bad = err > tol
    assert not bad.any(), (np.argwhere(bad)[:5], err[bad][:5], What_o[bad][:5])
    tT = np.where(risk, 1e-2, 1e-5 + 1e-4 * T_o)
    assert (np.abs(T_g - T_o) <= tT).all()
    ok = ~risk
    return float((err[ok] / np.maximum(np.abs(What_o[ok]), 1e-12))[What_o[ok] > 1e-6].max())


def _render_pair(gb, oracle_lib, scene, idx, val, C, cam):
    r = gb.Render(scene, idx, val, C, [cam])
    (W, T, last), st = r.run(0)
    Wo, To, risk, cnt = oracle_lib.render(scene, idx, val.astype(np.float64), C, cam)
    return W.cpu().numpy(), T.cpu().numpy(), last.cpu().numpy(), st, Wo, To, risk, cnt


@pytest.mark.parametrize("seed,W,H,n,C,K,lsm", [
    (51, 50, 37, 400, 16, 3, -2.5),
    (52, 64, 48, 1500, 64, 4, -2.8),
    (53, 33, 17, 300, 8, 8, -2.2),
    (54, 130, 70, 3000, 256, 8, -3.0),
])
def test_render_random_codes(gb, oracle_lib, seed, W, H, n, C, K, lsm):
    wl = synth.tiny_workload(seed, n=n, width=W, height=H, V=1, log_scale_mean=lsm)
    rng = np.random.default_rng(seed)
    idx, val = synth.sparse_topk_codes(rng, n, C, K)
    idx[::7, -1] = -1  # padded entries
    val[::7, -1] = 0.0
    Wg, Tg, lastg, st, Wo, To, risk, cnt = _render_pair(gb, oracle_lib, wl.scene, idx, val, C, wl.cams[0])
    rel = check_render(Wg, Tg, Wo, To, risk)
    assert abs(st["contributions"] - cnt["contributions"]) <= 2 * risk.sum()
    assert rel < RTOL
    assert (lastg >= 0).all()


@pytest.mark.parametrize("kernel", ["tensor", "simt"])
def test_render_one_hot_round_trip(gb, oracle_lib, monkeypatch, kernel):
    """Every Gaussian coded (j, 1): What(p) = (1 - T_final(p)) onehot_j.

    The SIMT kernel sums the weights in FP32 in list order (2e-6).  The
    tensor-core kernel splits each weight into two bf16 parts, which keep it
    to u^2 = 2^-16 relative (u = 2^-8; the code value 1 is exact in bf16),
    and sums the products in FP32 inside the MMA: the bound adds 2^-16 of the
    sum (1 - T)."""
    if kernel == "simt":
        monkeypatch.setenv("SCOUP_RENDER_SIMT", "1")
    wl = synth.tiny_workload(55, n=800, width=72, height=40, V=1, log_scale_mean=-2.6)
    n = wl.scene.n
    idx = np.full((n, 2), -1, np.int32)
    idx[:, 0] = 5
    val = np.zeros((n, 2), np.float32)
    val[:, 0] = 1.0
    Wg, Tg, *_ = _render_pair(gb, oracle_lib, wl.scene, idx, val, 12, wl.cams[0])
    atol = 2e-6 + (2.0 ** -16 * (1.0 - Tg) if kernel == "tensor" else 0.0)
    assert (np.abs(Wg[..., 5] - (1.0 - Tg)) <= atol).all()
    assert np.abs(np.delete(Wg, 5, axis=-1)).max() == 0.0


def test_render_long_lists(gb, oracle_lib):
    wl = synth.tiny_workload(56, n=6000, width=48, height=32, V=1, log_scale_mean=-2.0)
    wl.scene.opacity[:] = np.minimum(wl.scene.opacity, 0.06)
    rng = np.random.default_rng(56)
    idx, val = synth.sparse_topk_codes(rng, wl.scene.n, 32, 4)
    Wg, Tg, lastg, st, Wo, To, risk, cnt = _render_pair(gb, oracle_lib, wl.scene, idx, val, 32, wl.cams[0])
    check_render(Wg, Tg, Wo, To, risk)
    assert st["listed"] / 6 > 1500


def test_render_uplifted_codes(gb, oracle_lib, cfg1, cfg1_oracle):
    """Render cfg1's scene with the Top-K codes of the oracle's uplift (the
    paper's pipeline; the GPU uplift's own Top-K is checked against the same
    codes by the uplift parity tests)."""
    idx = cfg1_oracle["idx"].astype(np.int32)
    val = cfg1_oracle["val"].astype(np.float32)
    for v in (0, 5):
        Wg, Tg, lastg, st, Wo, To, risk, cnt = _render_pair(gb, oracle_lib, cfg1.scene, idx, val, cfg1.C,
                                                           cfg1.cams[v])
        check_render(Wg, Tg, Wo, To, risk)


@pytest.mark.parametrize("case", ["random", "long_lists"])
def test_render_bf16_output(gb, oracle_lib, case):
    """bf16 output: the FP32 row rounded once per window the pixel spans
    (relative error at most windows x 2^-8 on top of the FP32 tolerance)."""
    import torch
    if case == "random":
        wl = synth.tiny_workload(57, n=3000, width=130, height=70, V=1, log_scale_mean=-3.0)
        C, K = 256, 8
    else:
        wl = synth.tiny_workload(56, n=6000, width=48, height=32, V=1, log_scale_mean=-2.0)
        wl.scene.opacity[:] = np.minimum(wl.scene.opacity, 0.06)
        C, K = 32, 4
    rng = np.random.default_rng(57)
    idx, val = synth.sparse_topk_codes(rng, wl.scene.n, C, K)
    r = gb.Render(wl.scene, idx, val, C, [wl.cams[0]])
    (W32, T32, last), _ = r.run(0)
    outb = r.outputs(wl.cams[0], dtype=torch.bfloat16)
    (Wb, Tb, lastb), st = r.run(0, out=outb)
    assert st["status"] == 0
    Wo, To, risk, _ = oracle_lib.render(wl.scene, idx, val.astype(np.float64), C, wl.cams[0])
    windows = np.ceil(np.maximum(last.cpu().numpy(), 1) / 256.0)[..., None] + 1.0
    err = np.abs(Wb.float().cpu().numpy().astype(np.float64) - Wo)
    scale = np.abs(Wo).max(axis=-1, keepdims=True)
    tol = windows * 2.0 ** -8 * np.abs(Wo) + 1e-4 * np.abs(Wo) + 1e-6 * scale + 1e-7
    tol = np.where(risk[..., None], 1e-2 + tol, tol)
    assert (err <= tol).all(), float((err - tol).max())
    # transmittance and counts do not depend on the output type
    assert torch.equal(Tb, T32) and torch.equal(lastb, last)


def test_render_bf16_feeds_decode(gb):
    """bf16 rendered codes go to the decode without conversion (codes_dtype 1):
    the result equals decoding the same values handed over as float32 (which
    the decode rounds to the same bf16 numbers)."""
    import torch
    wl = synth.tiny_workload(58, n=2000, width=64, height=48, V=1)
    rng = np.random.default_rng(58)
    C, K, D = 64, 4, 32
    idx, val = synth.sparse_topk_codes(rng, wl.scene.n, C, K)
    B = torch.from_numpy(synth.unit_rows(rng, C, D)).cuda()
    r = gb.Render(wl.scene, idx, val, C, [wl.cams[0]])
    outb = r.outputs(wl.cams[0], dtype=torch.bfloat16)
    (Wb, _, _), _ = r.run(0, out=outb)
    P = wl.cams[0].width * wl.cams[0].height
    f_direct = torch.empty((P, D), dtype=torch.float32, device="cuda")
    f_conv = torch.empty((P, D), dtype=torch.float32, device="cuda")
    gb.scoup_decode(Wb.view(P, C), B, f_direct)
    gb.scoup_decode(Wb.view(P, C).float().contiguous(), B, f_conv)
    torch.cuda.synchronize()
    assert torch.equal(f_direct, f_conv)
    assert f_direct.abs().sum() > 0


@pytest.mark.parametrize("seed,W,H,n,C,K,lsm", [
    (52, 64, 48, 1500, 64, 4, -2.8),
    (54, 130, 70, 3000, 256, 8, -3.0),
])
def test_render_simt_kernel(gb, oracle_lib, monkeypatch, seed, W, H, n, C, K, lsm):
    """The SIMT kernel, selected by SCOUP_RENDER_SIMT=1, on the random-code cases."""
    monkeypatch.setenv("SCOUP_RENDER_SIMT", "1")
    test_render_random_codes(gb, oracle_lib, seed, W, H, n, C, K, lsm)


def test_render_wide_rows_and_largest_k(gb, oracle_lib):
    """C = 320 (wider than the tensor-core kernel takes: SIMT kernel) and
    C = 256 with K = 16 (the largest Top-K the tensor-core kernel stages)."""
    wl = synth.tiny_workload(59, n=2500, width=80, height=56, V=1, log_scale_mean=-2.8)
    rng = np.random.default_rng(59)
    for C, K in ((320, 8), (256, 16)):
        idx, val = synth.sparse_topk_codes(rng, wl.scene.n, C, K)
        Wg, Tg, lastg, st, Wo, To, risk, cnt = _render_pair(gb, oracle_lib, wl.scene, idx, val, C, wl.cams[0])
        check_render(Wg, Tg, Wo, To, risk)
        assert abs(st["contributions"] - cnt["contributions"]) <= 2 * risk.sum()


def test_render_repeated_atoms(gb, oracle_lib):
    """A code naming one atom twice adds both values (Eq. 7 over the sparse
    vector), and atom ids outside [0, C) or -1 add nothing."""
    wl = synth.tiny_workload(60, n=1200, width=64, height=40, V=1, log_scale_mean=-2.6)
    rng = np.random.default_rng(60)
    C, K = 48, 6
    idx, val = synth.sparse_topk_codes(rng, wl.scene.n, C, K)
    idx[::3, 1] = idx[::3, 0]            # repeated atom
    idx[::5, 2] = idx[::5, 0]
    val[::4, 3] = -val[::4, 3]           # a negative coefficient
    idx[::11, 4] = -1
    val[::11, 4] = 0.0
    Wg, Tg, lastg, st, Wo, To, risk, cnt = _render_pair(gb, oracle_lib, wl.scene, idx, val, C, wl.cams[0])
    err = np.abs(Wg.astype(np.float64) - Wo)
    mag, *_ = oracle_lib.render(wl.scene, idx, np.abs(val).astype(np.float64), C, wl.cams[0])
    tol = 1e-4 * mag + 1e-6 * mag.max(axis=-1, keepdims=True) + 1e-7
    tol = np.where(risk[..., None], 1e-2 + tol, tol)
    assert (err <= tol).all(), float((err - tol).max())


@pytest.mark.parametrize("out_dtype", ["bf16", "f32"])
def test_render_decode_fused(gb, oracle_lib, out_dtype):
    """scoup_render_decode_fused (Eq. 7 then Eq. 8 in one call) equals
    scoup_render with bf16 codes followed by scoup_decode bit for bit, and
    the oracle's decode of the oracle's render within the bf16 operand bound:
    |F - F_o| <= (2u + u^2 + 2e-4) sum_c |W_c| |B_cd| (+ u |F_o| for bf16
    features), u = 2^-8, 2e-4 covering the rendered codes' own tolerance."""
    import torch
    wl = synth.tiny_workload(61, n=2500, width=96, height=64, V=1, log_scale_mean=-2.8)
    rng = np.random.default_rng(61)
    C, K, D = 64, 8, 128
    idx, val = synth.sparse_topk_codes(rng, wl.scene.n, C, K)
    Bn = synth.unit_rows(rng, C, D)
    B = torch.from_numpy(Bn).cuda()
    cam = wl.cams[0]
    P = cam.width * cam.height
    fdt = torch.bfloat16 if out_dtype == "bf16" else torch.float32
    r = gb.Render(wl.scene, idx, val, C, [cam])
    Wb, T1, last1 = r.outputs(cam, dtype=torch.bfloat16)
    r.run(0, out=(Wb, T1, last1))
    f1 = torch.empty((P, D), dtype=fdt, device="cuda")
    n1 = torch.zeros((P,), dtype=torch.float32, device="cuda") if out_dtype == "bf16" else None
    gb.scoup_decode(Wb.view(P, C), B, f1, n1)
    f2 = torch.empty_like(f1)
    n2 = torch.zeros_like(n1) if n1 is not None else None
    T2, last2 = torch.empty_like(T1), torch.empty_like(last1)
    st = r.run_decode(0, B, f2, n2, T2, last2)
    torch.cuda.synchronize()
    assert st["status"] == 0 and st["contributions"] > 0
    assert torch.equal(f1, f2) and torch.equal(T1, T2) and torch.equal(last1, last2)
    if n1 is not None:
        assert torch.equal(n1, n2)
    Wo, To, risk, _ = oracle_lib.render(wl.scene, idx, val.astype(np.float64), C, cam)
    Fo = oracle_lib.decode(Wo.reshape(P, C), Bn)
    mag = np.abs(Wo.reshape(P, C)) @ np.abs(Bn.astype(np.float64))
    u = 2.0 ** -8
    bound = (2 * u + u * u + 2e-4) * mag + (u * np.abs(Fo) if out_dtype == "bf16" else 0.0) + 1e-6
    ok = ~risk.reshape(P)
    err = np.abs(f2.float().cpu().numpy().astype(np.float64) - Fo)
    assert (err[ok] <= bound[ok]).all(), float((err - bound)[ok].max())


def test_render_decode_fused_argument_checks(gb):
    import torch
    from paper_2605_13600_gb300._lib import ScoupError
    wl = synth.tiny_workload(62, n=300, width=40, height=24, V=1)
    rng = np.random.default_rng(62)
    idx, val = synth.sparse_topk_codes(rng, wl.scene.n, 12, 3)
    r = gb.Render(wl.scene, idx, val, 12, [wl.cams[0]])
    B = torch.from_numpy(synth.unit_rows(rng, 12, 32)).cuda()
    f = torch.empty((40 * 24, 32), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(ScoupError):  # C = 12 is not a multiple of 8 (the decode's limit)
        r.run_decode(0, B, f)


def test_cfg4_full_size_sampled_pixels(gb, oracle_lib):
    """The 1920 x 1080 render of the 1M-Gaussian scene (C = 256, K = 8: the
    benchmark's render configuration, seeded random K-sparse codes) at 48
    sampled pixels (the four corners and 44 random ones): What(p) and T_final
    against the oracle's front-to-back list of each pixel, Eq. 7 summed in
    FP64.  A pixel whose stop decision flips (T off by more than 1e-3
    relative) is at risk; at most two of the 48 may be."""
    import torch
    from concurrent.futures import ThreadPoolExecutor
    wl = synth.render_cfg4(n_views=1)
    cam = wl.cams[0]
    r = gb.Render(wl.scene, wl.topk_idx, wl.topk_val, wl.C, [cam])
    (W, T, last), st = r.run(0)
    assert st["status"] == 0
    rng = np.random.default_rng(401)
    pts = [(0, 0), (cam.width - 1, cam.height - 1), (cam.width - 1, 0), (0, cam.height - 1)]
    pts += [(int(x), int(y)) for x, y in zip(rng.integers(0, cam.width, 44), rng.integers(0, cam.height, 44))]
    xs = torch.tensor([p[0] for p in pts], device=W.device)
    ys = torch.tensor([p[1] for p in pts], device=W.device)
    Wg = W[ys, xs].double().cpu().numpy()
    Tg = T[ys, xs].double().cpu().numpy()
    with ThreadPoolExecutor(16) as ex:  # the oracle's C code runs without the GIL
        lists = list(ex.map(lambda p: oracle_lib.pixel_list(wl.scene, cam, p[0], p[1]), pts))
    flips = 0
    for k, (gids, e, _, To) in enumerate(lists):
        if abs(Tg[k] - To) > 1e-3 * max(To, 1e-4) + 1e-6:
            flips += 1
            continue
        wo = np.zeros(wl.C)
        for g, ee in zip(gids, e):
            for a in range(wl.K):
                j = int(wl.topk_idx[g, a])
                if j >= 0:
                    wo[j] += float(wl.topk_val[g, a]) * ee
        tol = 1e-4 * np.abs(wo) + 1e-6 * np.abs(wo).max() + 1e-7
        assert (np.abs(Wg[k] - wo) <= tol).all(), (pts[k], float(np.max(np.abs(Wg[k] - wo) - tol)))
        assert abs(Tg[k] - To) <= 1e-5 + 1e-4 * To
    assert flips <= 2


@pytest.mark.parametrize("kernel", ["tensor", "simt"])
def test_render_equal_depth_sheet(gb, oracle_lib, monkeypatch, kernel):
    """The fronto-parallel sheet of the uplift tests (every Gaussian at one
    depth): both render kernels cut their windows out of one oversize depth
    bucket and still composite in the oracle's (depth, index) order."""
    from test_gpu_uplift import _sheet_workload
    if kernel == "simt":
        monkeypatch.setenv("SCOUP_RENDER_SIMT", "1")
    wl = _sheet_workload()
    rng = np.random.default_rng(62)
    idx, val = synth.sparse_topk_codes(rng, wl.scene.n, 32, 4)
    Wg, Tg, lastg, st, Wo, To, risk, cnt = _render_pair(gb, oracle_lib, wl.scene, idx, val, 32, wl.cams[0])
    check_render(Wg, Tg, Wo, To, risk)
    assert st["split_windows"] > 0, st
    assert abs(st["contributions"] - cnt["contributions"]) <= 2 * risk.sum()
