"""GPU backward of the sparse-code rendering (scoup_render_backward) vs the
FP64 oracle's backward (itself pinned against finite differences and an
autograd restatement), directly and through the torch.autograd.Function."""
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


def _case(seed, n, W, H, C, K, lsm):
    wl = synth.tiny_workload(seed, n=n, width=W, height=H, V=1, log_scale_mean=lsm)
    rng = np.random.default_rng(seed)
    idx, val = synth.sparse_topk_codes(rng, n, C, K)
    g = rng.normal(size=(H, W, C)).astype(np.float32)
    return wl.scene, wl.cams[0], idx, val, g


def _compare(d_g, d_o, name):
    scale = np.abs(d_o).max()
    err = np.abs(d_g - d_o)
    tol = 2e-4 * np.abs(d_o) + 2e-5 * scale
    bad = err > tol
    assert not bad.any(), (name, np.argwhere(bad)[:5], d_g[bad][:5], d_o[bad][:5], scale)
    return float(err.max() / scale)


@pytest.mark.parametrize("seed,n,W,H,C,K,lsm", [
    (61, 300, 40, 32, 16, 3, -2.5),
    (62, 1500, 64, 48, 64, 8, -2.8),
    (63, 800, 33, 21, 32, 4, -2.2),
])
def test_backward_matches_oracle(gb, oracle_lib, seed, n, W, H, C, K, lsm):
    import torch
    scene, cam, idx, val, g = _case(seed, n, W, H, C, K, lsm)
    # a pixel whose stop decision is at risk may drop or add one contribution on the
    # GPU: give it no gradient on both sides so the comparison covers clear pixels only
    _, _, risk, _ = oracle_lib.render(scene, idx, val.astype(np.float64), C, cam)
    g[risk] = 0.0
    r = gb.Render(scene, idx, val, C, [cam])
    d_val = torch.zeros((n, K), dtype=torch.float32, device="cuda")
    d_op = torch.zeros(n, dtype=torch.float32, device="cuda")
    gb.scoup_render_backward(r.scene, r.topk_idx, r.topk_val, K, C, cam, torch.as_tensor(g, device="cuda"),
                             d_val, d_op, r.workspace)
    dv_o, do_o = oracle_lib.render_backward(scene, idx, val.astype(np.float64), C, cam, g.astype(np.float64))
    _compare(d_val.cpu().numpy(), dv_o, "d_val")
    _compare(d_op.cpu().numpy(), do_o, "d_opacity")


def test_autograd_function(gb, oracle_lib):
    import torch
    from paper_2605_13600_gb300.autograd import SparseRender
    scene, cam, idx, val, _ = _case(64, 700, 48, 40, 24, 4, -2.6)
    rng = np.random.default_rng(1)
    cb = torch.as_tensor(rng.normal(size=(24, 10)).astype(np.float32), device="cuda")
    target = torch.as_tensor(rng.normal(size=(40, 48, 10)).astype(np.float32), device="cuda")
    Wo, _, risk, _ = oracle_lib.render(scene, idx, val.astype(np.float64), 24, cam)
    keep = torch.as_tensor(~risk, device="cuda").float()[..., None]
    r = gb.Render(scene, idx, val, 24, [cam])
    op = torch.as_tensor(scene.opacity, device="cuda").clone().requires_grad_(True)
    tv = torch.as_tensor(val, device="cuda").clone().requires_grad_(True)
    W = SparseRender.apply(op, tv, r, 0)
    loss = (keep * (W @ cb - target) ** 2).sum()
    loss.backward()
    # the oracle's gradient input comes from its own forward render, in FP64
    cb64 = cb.cpu().numpy().astype(np.float64)
    keep64 = (~risk).astype(np.float64)[..., None]
    g = keep64 * 2.0 * (Wo @ cb64 - target.cpu().numpy().astype(np.float64)) @ cb64.T
    dv_o, do_o = oracle_lib.render_backward(scene, idx, val.astype(np.float64), 24, cam, g)
    _compare(tv.grad.cpu().numpy(), dv_o, "d_val")
    _compare(op.grad.cpu().numpy(), do_o, "d_opacity")


def test_cfg5_full_size_backward(gb, oracle_lib):
    """The benchmark's backward configuration (500k Gaussians, an 800 x 600
    view, C = 256, K = 8; seeded N(0, 1) gradient, zero at pixels whose stop
    decision is at risk) against the oracle's FP64 backward of the whole
    view.  d_val sums many signed FP32 terms: its bound adds 1e-5 of the sum
    of the terms' magnitudes, which the oracle gives exactly as d_val of |g|."""
    import torch
    wl = synth.render_cfg5()
    cam = wl.cams[0]
    n, C, K = wl.scene.n, wl.C, wl.K
    idx, val = wl.topk_idx, wl.topk_val
    rng = np.random.default_rng(501)
    g = rng.standard_normal((cam.height, cam.width, C), dtype=np.float32)
    _, _, risk, _ = oracle_lib.render(wl.scene, idx, val.astype(np.float64), C, cam)
    g[risk] = 0.0
    r = gb.Render(wl.scene, idx, val, C, [cam])
    d_val = torch.zeros((n, K), dtype=torch.float32, device="cuda")
    d_op = torch.zeros(n, dtype=torch.float32, device="cuda")
    gb.scoup_render_backward(r.scene, r.topk_idx, r.topk_val, K, C, cam, torch.as_tensor(g, device="cuda"),
                             d_val, d_op, r.workspace)
    g64 = g.astype(np.float64)
    dv_o, do_o = oracle_lib.render_backward(wl.scene, idx, val.astype(np.float64), C, cam, g64)
    dv_mag, _ = oracle_lib.render_backward(wl.scene, idx, np.abs(val).astype(np.float64), C, cam, np.abs(g64))
    dv_g = d_val.cpu().numpy()
    tol = 2e-4 * np.abs(dv_o) + 2e-5 * np.abs(dv_o).max() + 1e-5 * dv_mag
    assert (np.abs(dv_g - dv_o) <= tol).all(), float(np.max(np.abs(dv_g - dv_o) - tol))
    _compare(d_op.cpu().numpy(), do_o, "d_opacity")
    assert np.abs(dv_o).max() > 0 and np.abs(do_o).max() > 0
