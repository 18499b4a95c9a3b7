"""Pins of the oracle's backward through Eq. 7 (no GPU).

The loss is L = sum_p |What(p) C - F*(p)|^2 (Eq. 8 decode against a
per-pixel target).  The oracle's analytic gradient w.r.t. the Top-K values
and the opacities is checked against (a) central finite differences of the
oracle's own forward render and (b) an FP64 PyTorch autograd restatement of
Eqs. 2 and 7 over the same front-to-back lists.
"""
import numpy as np
import pytest

from conftest import make_scene


def _setup(seed=21, n=60, W=32, H=24, K=3, C=8, D=6):
    import synth
    rng = np.random.default_rng(seed)
    scene = synth.gaussians(rng, n, "uniform", log_scale_mean=-2.3)
    scene.means *= 0.6
    cam = synth.camera_at([0.3, -2.5, 0.8], W, H, 60.0)
    idx, val = synth.sparse_topk_codes(rng, n, C, K)
    idx[3, 2] = -1
    val[3, 2] = 0.0
    cb = rng.normal(size=(C, D)).astype(np.float32)
    target = rng.normal(size=(H, W, D))
    return scene, cam, idx, val.astype(np.float64), cb, target


def _loss(oracle_lib, scene, cam, idx, val, cb, target, C):
    What, T, risk, cnt = oracle_lib.render(scene, idx, val, C, cam)
    F = What @ cb.astype(np.float64)
    return float(((F - target) ** 2).sum()), What, cnt


def _grad(oracle_lib, scene, cam, idx, val, cb, target, C):
    L, What, _ = _loss(oracle_lib, scene, cam, idx, val, cb, target, C)
    g = 2.0 * (What @ cb.astype(np.float64) - target) @ cb.astype(np.float64).T
    return oracle_lib.render_backward(scene, idx, val, C, cam, g)


def test_backward_values_fd(oracle_lib):
    scene, cam, idx, val, cb, target = _setup()
    C = 8
    d_val, _ = _grad(oracle_lib, scene, cam, idx, val, cb, target, C)
    assert np.abs(d_val).max() > 0
    h = 1e-3  # L is quadratic in the values: central differences are exact up to rounding
    rng = np.random.default_rng(0)
    for i in rng.choice(scene.n, 15, replace=False):
        for k in range(idx.shape[1]):
            vp, vm = val.copy(), val.copy()
            vp[i, k] += h
            vm[i, k] -= h
            Lp = _loss(oracle_lib, scene, cam, idx, vp, cb, target, C)[0]
            Lm = _loss(oracle_lib, scene, cam, idx, vm, cb, target, C)[0]
            fd = (Lp - Lm) / (2 * h)
            assert d_val[i, k] == pytest.approx(fd, rel=1e-8, abs=1e-9)


def test_backward_opacity_fd(oracle_lib):
    scene, cam, idx, val, cb, target = _setup()
    C = 8
    _, d_op = _grad(oracle_lib, scene, cam, idx, val, cb, target, C)
    L0, _, cnt0 = _loss(oracle_lib, scene, cam, idx, val, cb, target, C)
    checked = 0
    for i in range(scene.n):
        o = scene.opacity[i]
        if not (0.05 < o < 0.9):
            continue
        op = np.nextafter(o, np.float32(2), dtype=np.float32)
        om = np.nextafter(o, np.float32(0), dtype=np.float32)
        for _ in range(63):
            op = np.nextafter(op, np.float32(2), dtype=np.float32)
            om = np.nextafter(om, np.float32(0), dtype=np.float32)
        sp, sm = scene.subset(np.arange(scene.n)), scene.subset(np.arange(scene.n))
        sp.opacity[i] = op
        sm.opacity[i] = om
        Lp, _, cp = _loss(oracle_lib, sp, cam, idx, val, cb, target, C)
        Lm, _, cm = _loss(oracle_lib, sm, cam, idx, val, cb, target, C)
        if cp != cnt0 or cm != cnt0:
            continue  # a discrete decision moved; the derivative is not defined there
        fd = (Lp - Lm) / (float(op) - float(om))
        assert d_op[i] == pytest.approx(fd, rel=1e-5, abs=1e-6)
        checked += 1
    assert checked >= 10


def test_backward_matches_autograd(oracle_lib):
    torch = pytest.importorskip("torch")
    scene, cam, idx, val, cb, target = _setup(seed=22, n=50, W=24, H=20)
    C = 8
    d_val, d_op = _grad(oracle_lib, scene, cam, idx, val, cb, target, C)
    proj = [oracle_lib.project(scene, cam, i) for i in range(scene.n)]
    val_t = torch.tensor(val, dtype=torch.float64, requires_grad=True)
    op_t = torch.tensor(scene.opacity.astype(np.float64), requires_grad=True)
    cb_t = torch.tensor(cb.astype(np.float64))
    idx_t = torch.tensor(idx.astype(np.int64))
    loss = torch.zeros((), dtype=torch.float64)
    for y in range(cam.height):
        for x in range(cam.width):
            gids, _, _, _ = oracle_lib.pixel_list(scene, cam, x, y)
            Wp = torch.zeros(C, dtype=torch.float64)
            T = torch.ones((), dtype=torch.float64)
            for g in gids.tolist():
                p = proj[g]
                dx, dy = p.mx64 - x, p.my64 - y
                G = np.exp(-0.5 * (p.ca64 * dx * dx + p.cc64 * dy * dy) - p.cb64 * dx * dy)
                alpha = torch.clamp(op_t[g] * G, max=0.99)
                w = torch.zeros(C, dtype=torch.float64)
                valid = idx_t[g] >= 0
                w = w.index_add(0, idx_t[g][valid], val_t[g][valid])
                Wp = Wp + alpha * T * w
                T = T * (1 - alpha)
            loss = loss + ((Wp @ cb_t - torch.tensor(target[y, x])) ** 2).sum()
    loss.backward()
    np.testing.assert_allclose(d_val, val_t.grad.numpy(), rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(d_op, op_t.grad.numpy(), rtol=1e-9, atol=1e-12)
