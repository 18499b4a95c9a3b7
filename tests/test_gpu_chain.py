"""The differentiable render's loss chain on the GPU (the 500k-Gaussian,
800 x 600 differentiable-render workload): render (Eq. 7) -> decode (Eq. 8, bf16 tensor cores) -> L2 loss against
the decoded region codes -> dL/dF -> dL/dWhat = dL/dF C^T (tensor cores) ->
render backward.  Each new piece is checked against FP64 NumPy within the
bound its roundings imply; the whole chain against the oracle's FP64 chain
(oracle render, decode and render backward; the loss gradient by NumPy)
within the same bounds carried through the linear backward.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

U = 2.0 ** -8  # unit roundoff of bf16


@pytest.fixture(scope="module")
def gb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_13600_gb300 import build
    build.build()
    import paper_2605_13600_gb300 as gb
    return gb


@pytest.mark.parametrize("P,C,D", [(5000, 256, 512), (333, 64, 96), (1, 16, 8)])
def test_decode_backward_against_fp64(gb, P, C, D):
    """dL/dWhat = G C^T: the bf16 form within the operand roundings (both
    operands to bf16, FP32 accumulation), f32 and bf16 inputs; the FP32 SIMT
    form within FP32 accumulation."""
    import torch
    rng = np.random.default_rng(P + C)
    G = rng.normal(size=(P, D)).astype(np.float32)
    Cb = synth.unit_rows(rng, C, D)
    dev = torch.device("cuda:0")
    Gd, Cd = torch.from_numpy(G).to(dev), torch.from_numpy(Cb).to(dev)
    want = G.astype(np.float64) @ Cb.astype(np.float64).T
    mag = np.abs(G.astype(np.float64)) @ np.abs(Cb.astype(np.float64)).T
    out = torch.empty((P, C), dtype=torch.float32, device=dev)
    gb.scoup_decode_backward(Gd, Cd, out)
    err = np.abs(out.cpu().numpy() - want)
    assert (err <= (2 * U + U * U + 2.0 ** -22 * D) * mag + 1e-30).all(), float((err / (mag + 1e-30)).max())
    # bf16 input: the gradient already rounded, only the codebook is
    Gb = Gd.to(torch.bfloat16)
    want_b = Gb.float().cpu().numpy().astype(np.float64) @ Cb.astype(np.float64).T
    gb.scoup_decode_backward(Gb, Cd, out)
    err = np.abs(out.cpu().numpy() - want_b)
    assert (err <= (U + 2.0 ** -22 * D) * mag * (1 + U) + 1e-30).all()
    gb.scoup_decode_backward_fp32(Gd, Cd, out)
    err = np.abs(out.cpu().numpy() - want)
    assert (err <= 2.0 ** -22 * D * mag + 1e-30).all()


@pytest.mark.parametrize("out_bf16", [False, True])
def test_region_l2_grad_against_fp64(gb, out_bf16):
    """Targets are the decoded region codes; unlabelled pixels carry no loss
    and no gradient; a bad region id is reported."""
    import torch
    rng = np.random.default_rng(81)
    P, D, C, R, s = 3001, 96, 40, 17, 5
    F = rng.normal(size=(P, D)).astype(np.float32)
    rmap = rng.integers(0, R, size=P).astype(np.int32)
    rmap[::9] = -1
    ci, cv = synth.region_codes(rng, R, C, s)
    ci[3, -1] = -1  # a padded entry
    cv[3, -1] = 0.0
    Cb = synth.unit_rows(rng, C, D)
    tgt = np.zeros((R, D))
    for r in range(R):
        for j, v in zip(ci[r], cv[r]):
            if j >= 0:
                tgt[r] += float(v) * Cb[j].astype(np.float64)
    lab = rmap >= 0
    diff = np.where(lab[:, None], F.astype(np.float64) - tgt[np.maximum(rmap, 0)], 0.0)
    dev = torch.device("cuda:0")
    dF = torch.empty((P, D), dtype=torch.bfloat16 if out_bf16 else torch.float32, device=dev)
    loss = torch.zeros((), dtype=torch.float64, device=dev)
    ws = gb.scoup_region_l2_grad(torch.from_numpy(F).to(dev), torch.from_numpy(rmap).to(dev),
                                 torch.from_numpy(ci).to(dev), torch.from_numpy(cv).to(dev),
                                 torch.from_numpy(Cb).to(dev), dF, loss)
    torch.cuda.synchronize()
    assert gb.scoup_read_stats(ws)["status"] == 0
    got = dF.float().cpu().numpy().astype(np.float64)
    # target in FP32 from s products: within 2^-22 s |code| |C| of FP64
    slack = 2.0 ** -21 * s + (U if out_bf16 else 2.0 ** -23)
    assert (np.abs(got - 2 * diff) <= slack * (2 * np.abs(diff) + 2.0) + 1e-7).all()
    assert (got[~lab] == 0).all()
    assert abs(float(loss.item()) - float((diff ** 2).sum())) <= 1e-5 * float((diff ** 2).sum())
    # a region id past the table is reported, not read
    bad = torch.from_numpy(rmap).to(dev)
    bad[7] = R
    ws = gb.scoup_region_l2_grad(torch.from_numpy(F).to(dev), bad, torch.from_numpy(ci).to(dev),
                                 torch.from_numpy(cv).to(dev), torch.from_numpy(Cb).to(dev), dF, None)
    torch.cuda.synchronize()
    with pytest.raises(gb.ScoupError) as ei:
        gb.scoup_read_stats(ws)
    assert ei.value.code == -5


def _chain_workload():
    """A small scene with its own uplift: 2500 blob Gaussians, 3 views at
    80x60, 12 regions per view, C = 32, s = 4, K = 4, and a 32 x 64 codebook."""
    return synth.uplift_cfg5(n=2500, V=3, width=80, height=60, R=12, C=32, s=4, K=4, D=64, seed=85)


def test_loss_chain_matches_oracle(gb, oracle_lib):
    """The whole chain on one view with the oracle's own Top-K codes: GPU
    d_val and d_opacity against the oracle's FP64 chain, within the bf16
    roundings of the decode, the loss gradient and the backward GEMM carried
    through the backward (which is linear in the upstream gradient)."""
    import torch
    from paper_2605_13600_gb300.autograd import SparseDecode, SparseRender
    wl, cb = _chain_workload()
    acc, _, _ = oracle_lib.uplift(wl)
    idx, val = oracle_lib.topk(acc, wl.K)
    idx, val = idx.astype(np.int32), val.astype(np.float32)
    cam = wl.cams[0]
    H, W, C, D, n = cam.height, cam.width, wl.C, cb.shape[1], wl.scene.n
    Wo, To, risk, _ = oracle_lib.render(wl.scene, idx, val.astype(np.float64), C, cam)
    # pixels whose stop decision is at risk get no target on either side
    rmap = wl.region_maps[:H * W].copy()
    rmap[risk.reshape(-1)] = -1
    lab = (rmap >= 0).reshape(H, W)
    cb64 = cb.astype(np.float64)
    tgt = np.zeros((int(wl.code_idx.shape[0]), D))
    for r in range(tgt.shape[0]):
        for j, v in zip(wl.code_idx[r], wl.code_val[r]):
            if j >= 0:
                tgt[r] += float(v) * cb64[j]
    F = Wo.reshape(-1, C) @ cb64
    Fs = np.where(lab.reshape(-1, 1), tgt[np.maximum(rmap, 0)], 0.0)
    dF = np.where(lab.reshape(-1, 1), 2.0 * (F - Fs), 0.0)
    g = (dF @ cb64.T).reshape(H, W, C)
    dv_o, do_o = oracle_lib.render_backward(wl.scene, idx, val.astype(np.float64), C, cam, g)

    # ---- GPU: render -> decode -> loss -> backward GEMM -> render backward ----
    dev = torch.device("cuda:0")
    r = gb.Render(wl.scene, idx, val, C, [cam])
    op = torch.as_tensor(wl.scene.opacity, device=dev).clone().requires_grad_(True)
    tv = torch.as_tensor(val, device=dev).clone().requires_grad_(True)
    cbd = torch.from_numpy(cb).to(dev)
    Wg = SparseRender.apply(op, tv, r, 0)
    Fg = SparseDecode.apply(Wg.reshape(-1, C), cbd)
    dFg = torch.empty((H * W, D), dtype=torch.bfloat16, device=dev)
    loss = torch.zeros((), dtype=torch.float64, device=dev)
    gb.scoup_region_l2_grad(Fg.detach(), torch.from_numpy(rmap).to(dev), torch.from_numpy(wl.code_idx).to(dev),
                            torch.from_numpy(wl.code_val).to(dev), cbd, dFg, loss)
    Fg.backward(dFg.float())
    torch.cuda.synchronize()

    # ---- bound on |g_gpu - g| per pixel and atom, then through the backward ----
    A = np.abs(Wo.reshape(-1, C)) @ np.abs(cb64)
    A += (1e-4 * np.abs(Wo.reshape(-1, C)) + 1e-6 * np.abs(Wo).max()) @ np.abs(cb64)  # FP32 render
    eF = A * (2 * U + U * U + 2.0 ** -22 * C) + U * (np.abs(F) + A) + 1e-7  # decode: bf16 operands, bf16 output
    diff = np.abs(F - Fs)[lab.reshape(-1)]
    eL = eF[lab.reshape(-1)]
    want_loss = float((diff ** 2).sum())
    assert abs(float(loss.item()) - want_loss) <= float((2 * diff * eL + eL ** 2).sum()) + 1e-6 * want_loss
    dFm = np.where(lab.reshape(-1, 1), 2.0 * eF * (1 + U) + U * np.abs(dF), 0.0)  # dF to bf16
    dg = ((dFm + (U + 2.0 ** -22 * D) * (np.abs(dF) + dFm)) @ np.abs(cb64).T).reshape(H, W, C)
    bnd_val, _ = oracle_lib.render_backward(wl.scene, idx, val.astype(np.float64), C, cam, dg)
    gmax = np.broadcast_to(dg.max(axis=-1, keepdims=True), dg.shape).copy()
    bnd_e, _ = oracle_lib.render_backward(wl.scene, idx, val.astype(np.float64), C, cam, gmax)
    terms_val, _ = oracle_lib.render_backward(wl.scene, idx, val.astype(np.float64), C, cam, np.abs(g))
    o = wl.scene.opacity.astype(np.float64)
    tol_val = bnd_val + 2e-4 * np.abs(dv_o) + 2e-5 * np.abs(dv_o).max() + 1e-5 * terms_val
    tol_op = 2.0 / o * bnd_e[:, 0] + 2e-4 * np.abs(do_o) + 2e-5 * np.abs(do_o).max()
    dv_g = tv.grad.cpu().numpy().astype(np.float64)
    do_g = op.grad.cpu().numpy().astype(np.float64)
    assert (np.abs(dv_g - dv_o) <= tol_val).all(), float(np.max(np.abs(dv_g - dv_o) - tol_val))
    assert (np.abs(do_g - do_o) <= tol_op).all(), float(np.max(np.abs(do_g - do_o) - tol_op))
    # the bound is a fraction of the gradient it guards, not vacuous
    assert np.median(bnd_val[np.abs(dv_o) > 0] / np.abs(dv_o[np.abs(dv_o) > 0])) < 0.2
