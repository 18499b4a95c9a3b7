"""Pins of the FP64 oracle against facts fixed outside it (no GPU).

Each test checks the oracle against a closed form, an independent library
construction, brute force or an invariant, so that a dropped term, a wrong
sign or index, or a transposed operand in the oracle fails at least one:

* projection / EWA covariance  -> SciPy rotation + finite-difference Jacobian
* alpha, mean offset, scatter  -> single-Gaussian closed form
* compositing order            -> two-Gaussian occlusion, 0.99 stack with stop
* telescoping                  -> sum_i e_i(p) = 1 - T_final(p)
* tile binning + depth sort    -> brute-force per-pixel candidate scan
* scatter indexing             -> per-pixel lists x region codes, linearity,
                                  permutation and view-order invariance
* Top-K (Eq. 6)                -> full NumPy sort
* render (Eq. 7)               -> round trip of a one-hot scene
* decode / similarity          -> NumPy matmul / cosine
"""
import json
import math
import os

import numpy as np
import pytest

from conftest import axis_camera, make_scene, single_region_workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# projection
# --------------------------------------------------------------------------

def _independent_projection(mean, scale, quat, cam):
    """EWA 2D covariance from SciPy's rotation and a finite-difference
    Jacobian of the pinhole map (x, y, z) -> (fx x/z + cx, fy y/z + cy)."""
    from scipy.spatial.transform import Rotation
    vm = np.asarray(cam.viewmat, np.float64).reshape(3, 4)
    Rv, tv = vm[:, :3], vm[:, 3]
    mean = np.asarray(mean, np.float64)
    t = Rv @ mean + tv
    w, x, y, z = np.asarray(quat, np.float64)
    Rq = Rotation.from_quat([x, y, z, w]).as_matrix()
    S3 = Rq @ np.diag(np.asarray(scale, np.float64) ** 2) @ Rq.T
    limx = 1.3 * cam.width / (2 * cam.fx)
    limy = 1.3 * cam.height / (2 * cam.fy)
    tc = np.array([np.clip(t[0] / t[2], -limx, limx) * t[2],
                   np.clip(t[1] / t[2], -limy, limy) * t[2], t[2]])

    def pi(u):
        return np.array([cam.fx * u[0] / u[2] + cam.cx, cam.fy * u[1] / u[2] + cam.cy])

    J = np.zeros((2, 3))
    for k in range(3):
        h = 1e-5 * max(1.0, abs(tc[k]))
        e = np.zeros(3)
        e[k] = h
        J[:, k] = (pi(tc + e) - pi(tc - e)) / (2 * h)
    S2 = J @ Rv @ S3 @ Rv.T @ J.T + 0.3 * np.eye(2)
    mean2d = pi(t) - 0.5
    return t, S2, mean2d


def _random_cam(rng, W=320, H=240):
    import synth
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    return synth.camera_at(3.0 * d, W, H, 60.0)


def test_projection_matches_independent_ewa(oracle_lib):
    rng = np.random.default_rng(11)
    checked = 0
    for trial in range(300):
        cam = _random_cam(rng)
        mean = rng.uniform(-1.0, 1.0, 3)
        scale = np.exp(rng.normal(-3.0, 0.7, 3))
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        scene = make_scene(mean, scale, q, [0.5])
        p = oracle_lib.project(scene, cam, 0)
        t, S2, m2 = _independent_projection(scene.means[0], scene.scales[0], scene.quats[0], cam)
        if t[2] <= 0.2 + 1e-6:
            assert p.visible == 0
            continue
        if not p.visible:
            continue  # off-screen rectangle
        checked += 1
        conic = np.linalg.inv(S2)
        np.testing.assert_allclose([p.ca64, p.cb64, p.cc64], [conic[0, 0], conic[0, 1], conic[1, 1]],
                                   rtol=1e-6, atol=1e-9 * np.abs(conic).max())
        np.testing.assert_allclose([p.mx64, p.my64], m2, rtol=1e-10, atol=1e-9)
        # binary32 decision path agrees with FP64 to binary32 accuracy
        assert abs(p.qa - (-0.5 * conic[0, 0])) <= 1e-4 * abs(conic).max()
        assert abs(p.qb - (-conic[0, 1])) <= 1e-4 * abs(conic).max()
        assert abs(p.qc - (-0.5 * conic[1, 1])) <= 1e-4 * abs(conic).max()
        assert abs(p.mx - m2[0]) <= 1e-5 * max(1.0, abs(m2[0]))
        assert abs(p.depth - t[2]) <= 1e-6 * t[2]
        # radius from the largest eigenvalue with the 0.1 floor of the 3DGS bound
        a, b, c = S2[0, 0], S2[0, 1], S2[1, 1]
        mid = 0.5 * (a + c)
        lam = mid + math.sqrt(max(0.1, mid * mid - (a * c - b * b)))
        r = 3.0 * math.sqrt(lam)
        if mid * mid - (a * c - b * b) > 0.1:
            assert abs(lam - np.linalg.eigvalsh(S2).max()) <= 1e-9 * lam
        if abs(r - round(r)) > 1e-3:
            assert p.radius == math.ceil(r)
        # rectangle: tiles overlapping [m - r, m + r], clamped to the grid
        gx, gy = (cam.width + 15) // 16, (cam.height + 15) // 16
        for lo_hi, expect in (((p.rect[0], p.rect[2]), (m2[0], gx)), ((p.rect[1], p.rect[3]), (m2[1], gy))):
            m, g = expect
            lo = min(g, max(0, math.floor((m - p.radius) / 16)))
            hi = min(g, max(0, math.floor((m + p.radius + 15) / 16)))
            edge = min(abs((m - p.radius) / 16 - round((m - p.radius) / 16)),
                       abs((m + p.radius + 15) / 16 - round((m + p.radius + 15) / 16)))
            if edge > 1e-4:
                assert lo_hi == (lo, hi)
    assert checked > 150


def test_projection_clamped_jacobian(oracle_lib):
    """Off-axis Gaussians: the Jacobian is taken at the tangent clamped to
    1.3 x the half field of view, per axis (x uses the width, y the height)."""
    cam = axis_camera(64, 48, f=40.0, z=2.0)
    # lim_x = 1.3 * 32 / 40 = 1.04, lim_y = 1.3 * 24 / 40 = 0.78
    for mean, axis in (([3.0, 0.2, 0.0], 0), ([1.8, 0.1, 0.0], None), ([0.1, 1.9, 0.0], 1)):
        scene = make_scene(mean, [0.9, 0.5, 0.7], [0.9, 0.1, 0.3, 0.2], [0.5])
        scene.quats /= np.linalg.norm(scene.quats, axis=1, keepdims=True)
        p = oracle_lib.project(scene, cam, 0)
        t, S2, m2 = _independent_projection(scene.means[0], scene.scales[0], scene.quats[0], cam)
        if axis == 0:
            assert t[0] / t[2] > 1.04
        if axis == 1:
            assert t[1] / t[2] > 0.78
        assert p.visible == 1
        conic = np.linalg.inv(S2)
        np.testing.assert_allclose([p.ca64, p.cb64, p.cc64], [conic[0, 0], conic[0, 1], conic[1, 1]], rtol=1e-6)
        np.testing.assert_allclose([p.qa, p.qb, p.qc], [-0.5 * conic[0, 0], -conic[0, 1], -0.5 * conic[1, 1]],
                                   rtol=1e-4, atol=1e-6 * np.abs(conic).max())


def test_near_plane_cull(oracle_lib):
    cam = axis_camera(64, 48, f=48.0, z=0.0)
    for zc, vis in ((0.19, 0), (0.2, 0), (0.25, 1)):
        scene = make_scene([0.0, 0.0, zc], [0.01] * 3, [1, 0, 0, 0], [0.5])
        assert oracle_lib.project(scene, cam, 0).visible == vis


# --------------------------------------------------------------------------
# compositing closed forms
# --------------------------------------------------------------------------

def _iso_alpha(o, sigma2, mx, my, W, H):
    ys, xs = np.mgrid[0:H, 0:W]
    return o * np.exp(-0.5 * ((xs - mx) ** 2 + (ys - my) ** 2) / sigma2)


def test_single_gaussian_closed_form(oracle_lib):
    """Isotropic Gaussian on the optical axis: Sigma2 = (f s / z)^2 I + 0.3 I,
    mean at (cx - 0.5, cy - 0.5); with o < 0.35 every pixel with
    alpha >= 1/255 lies inside the 3-sigma rectangle, so the one-region
    one-hot uplift is the sum of the closed-form alphas."""
    f, s, z, o = 48.0, 0.125, 2.0, 0.3125
    W, H = 64, 48
    cam = axis_camera(W, H, f=f, z=z)
    scene = make_scene([0, 0, 0], [s, s, s], [1, 0, 0, 0], [o])
    wl = single_region_workload(scene, [cam], C=8, code_pairs=[(5, 1.0)], K=4)
    acc, risk, cnt = oracle_lib.uplift(wl)
    sigma2 = (f * s / z) ** 2 + 0.3
    a = _iso_alpha(o, sigma2, W / 2 - 0.5, H / 2 - 0.5, W, H)
    assert np.min(np.abs(a * 255.0 - 1.0)) > 1e-6
    keep = a >= 1.0 / 255.0
    assert acc[0, 5] == pytest.approx(a[keep].sum(), rel=1e-12)
    assert np.count_nonzero(acc) == 1 and not risk.any()
    assert cnt["contributions"] == int(keep.sum())
    idx, val = oracle_lib.topk(acc, 4)
    assert idx[0].tolist() == [5, -1, -1, -1] and val[0].tolist() == [1.0, 0.0, 0.0, 0.0]


def test_anisotropic_rotated_closed_form(oracle_lib):
    """Rotation theta about the optical axis, scales (sx, sy, sz), on axis:
    Sigma2 = (f/z)^2 R_theta diag(sx^2, sy^2) R_theta^T + 0.3 I."""
    f, z, o, th = 40.0, 2.5, 0.3, 0.6
    sx, sy, sz = 0.2, 0.08, 0.3
    W, H = 64, 64
    cam = axis_camera(W, H, f=f, z=z, cx=32.5, cy=31.5)
    q = [math.cos(th / 2), 0.0, 0.0, math.sin(th / 2)]
    scene = make_scene([0, 0, 0], [sx, sy, sz], q, [o])
    s32 = scene.scales[0].astype(np.float64)
    q32 = scene.quats[0].astype(np.float64)
    th32 = 2 * math.atan2(q32[3], q32[0])
    R2 = np.array([[math.cos(th32), -math.sin(th32)], [math.sin(th32), math.cos(th32)]])
    S2 = (f / z) ** 2 * R2 @ np.diag([s32[0] ** 2, s32[1] ** 2]) @ R2.T + 0.3 * np.eye(2)
    inv = np.linalg.inv(S2)
    ys, xs = np.mgrid[0:H, 0:W]
    d = np.stack([xs - 32.0, ys - 31.0], -1)
    a = float(scene.opacity[0]) * np.exp(-0.5 * np.einsum("...i,ij,...j->...", d, inv, d))
    p = oracle_lib.project(scene, cam, 0)
    np.testing.assert_allclose([p.ca64, p.cb64, p.cc64], [inv[0, 0], inv[0, 1], inv[1, 1]], rtol=1e-9)
    wl = single_region_workload(scene, [cam], C=4, code_pairs=[(2, 1.0)], K=1)
    acc, _, _ = oracle_lib.uplift(wl)
    keep = a >= 1.0 / 255.0
    assert acc[0, 2] == pytest.approx(a[keep].sum(), rel=1e-11)


def test_two_gaussian_occlusion(oracle_lib):
    """Front Gaussian (depth 2) over back Gaussian (depth 3): e1 = a1, e2 = a2 (1 - a1)."""
    f, W, H = 48.0, 64, 48
    cam = axis_camera(W, H, f=f, z=2.0, cx=32.5, cy=24.5)
    s1, s2, o1, o2 = 0.125, 0.25, 0.5, 0.75
    scene = make_scene([[0, 0, 1.0], [0, 0, 0]], [[s2] * 3, [s1] * 3], [[1, 0, 0, 0]] * 2, [o2, o1])
    sig1 = (f * s1 / 2.0) ** 2 + 0.3
    sig2 = (f * s2 / 3.0) ** 2 + 0.3
    a1 = _iso_alpha(o1, sig1, 32.0, 24.0, W, H)
    a2 = _iso_alpha(o2, sig2, 32.0, 24.0, W, H)
    gold = json.load(open(os.path.join(GOLDEN, "compositing_pins.json")))["two_gaussian_centre"]
    checked = 0
    for (x, y) in [(32, 24), (30, 25), (35, 20), (28, 28), (40, 24)]:
        gids, e, al, T = oracle_lib.pixel_list(scene, cam, x, y)
        if a1[y, x] >= 1 / 255 and a2[y, x] >= 1 / 255:
            assert gids.tolist() == [1, 0]  # gid 1 is in front
            np.testing.assert_allclose(e, [a1[y, x], a2[y, x] * (1 - a1[y, x])], rtol=1e-12)
            checked += 1
        if (x, y) == (32, 24):
            np.testing.assert_allclose(e, gold["e"], rtol=1e-12)
            assert T == pytest.approx(gold["T_final"], rel=1e-12)
    assert checked >= 4


def test_stop_rule_stack(oracle_lib):
    """Centre pixel of three stacked Gaussians with alpha 0.99 (capped),
    0.9, 0.95: T goes 1 -> 0.01 -> 1e-3, and the third would bring it to
    5e-5 < 1e-4, so it is excluded (stop before the Gaussian)."""
    gold = json.load(open(os.path.join(GOLDEN, "compositing_pins.json")))["stack_stop"]
    cam = axis_camera(32, 32, f=32.0, z=2.0, cx=16.5, cy=16.5)
    scene = make_scene([[0, 0, 0], [0, 0, 1.0], [0, 0, 2.0]], [[0.1] * 3] * 3,
                       [[1, 0, 0, 0]] * 3, [0.999, 0.9, 0.95])
    gids, e, al, T = oracle_lib.pixel_list(scene, cam, 16, 16)
    assert gids.tolist() == gold["gids"]
    np.testing.assert_allclose(al, gold["alpha"], rtol=1e-7)
    np.testing.assert_allclose(e, gold["e"], rtol=1e-7)
    assert T == pytest.approx(gold["T_final"], rel=1e-6)


def test_telescoping_sum(oracle_lib):
    """sum_i e_i(p) = 1 - T_final(p) for every pixel (Eq. 2 telescopes)."""
    import synth
    for seed in (3, 4):
        wl = synth.tiny_workload(seed, n=300, width=40, height=32, V=1, log_scale_mean=-2.5)
        cam = wl.cams[0]
        worst = 0.0
        for y in range(cam.height):
            for x in range(cam.width):
                _, e, _, T = oracle_lib.pixel_list(wl.scene, cam, x, y)
                worst = max(worst, abs(e.sum() - (1.0 - T)))
        assert worst < 1e-12


def test_brute_force_matches_tile_lists(oracle_lib):
    """Per-pixel O(N) candidate scan == tile-binned lists, bit for bit."""
    import synth
    for seed, (W, H) in ((5, (16, 16)), (6, (48, 40)), (7, (64, 48))):
        wl = synth.tiny_workload(seed, n=50, width=W, height=H, V=1, log_scale_mean=-2.0)
        cam = wl.cams[0]
        for y in range(0, H, 3):
            for x in range(0, W, 3):
                a = oracle_lib.pixel_list(wl.scene, cam, x, y, brute=False)
                b = oracle_lib.pixel_list(wl.scene, cam, x, y, brute=True)
                assert a[0].tolist() == b[0].tolist()
                assert np.array_equal(a[1], b[1]) and a[3] == b[3]


# --------------------------------------------------------------------------
# uplift scatter (Eq. 5, Algorithm 1)
# --------------------------------------------------------------------------

def test_uplift_equals_pixel_lists(oracle_lib):
    """acc[i, j] = sum over views and pixels of c_j(region(p)) e_i(v, p)."""
    import synth
    wl = synth.tiny_workload(8, n=120, width=32, height=32, V=2, R=5, C=12, s=3, K=3)
    acc, _, cnt = oracle_lib.uplift(wl)
    ref = np.zeros_like(acc)
    n_contrib = 0
    for v, cam in enumerate(wl.cams):
        rmap = wl.region_map(v)
        for y in range(cam.height):
            for x in range(cam.width):
                gids, e, _, _ = oracle_lib.pixel_list(wl.scene, cam, x, y)
                n_contrib += gids.size
                r = rmap[y, x]
                for g, ev in zip(gids, e):
                    for j, c in zip(wl.code_idx[r], wl.code_val[r]):
                        ref[g, j] += float(c) * ev
    np.testing.assert_allclose(acc, ref, rtol=1e-12, atol=1e-15)
    assert cnt["contributions"] == n_contrib


def test_uplift_weights_only_and_linearity(oracle_lib):
    """One-hot codes give Z_i = sum e_i; the uplift is linear in the codes."""
    import synth
    base = synth.tiny_workload(9, n=150, width=40, height=32, V=2, R=4, C=10, s=2, K=4)
    z_wl = single_region_workload(base.scene, base.cams, 10, [(3, 1.0)], 4)
    Z, _, _ = oracle_lib.uplift(z_wl)
    assert np.count_nonzero(Z[:, [0, 1, 2, 4, 5, 6, 7, 8, 9]]) == 0
    mix = single_region_workload(base.scene, base.cams, 10, [(3, 0.25), (7, 0.5), (1, 2.0)], 4)
    acc, _, _ = oracle_lib.uplift(mix)
    np.testing.assert_allclose(acc[:, 3], 0.25 * Z[:, 3], rtol=1e-12, atol=0)
    np.testing.assert_allclose(acc[:, 7], 0.5 * Z[:, 3], rtol=1e-12, atol=0)
    np.testing.assert_allclose(acc[:, 1], 2.0 * Z[:, 3], rtol=1e-12, atol=0)
    # a code with more than K entries keeps its K largest (ties to the lower atom)
    many = single_region_workload(base.scene, base.cams, 10, [(3, 0.25), (7, 0.5), (1, 2.0), (9, 0.5)], 2)
    acc2, _, _ = oracle_lib.uplift(many)
    assert np.count_nonzero(acc2[:, [3, 9]]) == 0
    np.testing.assert_allclose(acc2[:, 7], 0.5 * Z[:, 3], rtol=1e-12, atol=0)


def test_uplift_permutation_and_view_order(oracle_lib):
    import synth
    wl = synth.tiny_workload(10, n=200, width=48, height=40, V=3, R=6, C=16, s=3, K=3)
    acc, _, _ = oracle_lib.uplift(wl)
    perm = np.random.default_rng(0).permutation(wl.scene.n)
    wl_p = synth.UpliftWorkload(wl.name, wl.scene.subset(perm), wl.cams, wl.region_maps,
                                wl.map_offsets, wl.code_idx, wl.code_val, wl.C, wl.s, wl.K)
    acc_p, _, _ = oracle_lib.uplift(wl_p)
    np.testing.assert_allclose(acc_p, acc[perm], rtol=1e-12, atol=1e-15)
    acc_r, _, _ = oracle_lib.uplift(wl, views=[2, 1, 0])
    np.testing.assert_allclose(acc_r, acc, rtol=1e-12, atol=1e-15)
    rows = np.array([5, 17, 42, 199, 0])
    acc_rows, _, _ = oracle_lib.uplift(wl, rows=rows)
    np.testing.assert_allclose(acc_rows, acc[rows], rtol=1e-12, atol=1e-15)


def test_unlabelled_pixels_occlude_but_do_not_scatter(oracle_lib):
    import synth
    wl = synth.tiny_workload(12, n=150, width=40, height=32, V=1, R=4, C=8, s=2, K=2)
    acc, _, _ = oracle_lib.uplift(wl)
    masked = wl.region_maps.copy().reshape(32, 40)
    masked[:, :20] = -1
    wl_m = synth.UpliftWorkload(wl.name, wl.scene, wl.cams, masked.reshape(-1), wl.map_offsets,
                                wl.code_idx, wl.code_val, wl.C, wl.s, wl.K)
    acc_m, _, _ = oracle_lib.uplift(wl_m)
    ref = np.zeros_like(acc)
    for y in range(32):
        for x in range(20, 40):
            gids, e, _, _ = oracle_lib.pixel_list(wl.scene, wl.cams[0], x, y)
            r = masked[y, x]
            for g, ev in zip(gids, e):
                for j, c in zip(wl.code_idx[r], wl.code_val[r]):
                    ref[g, j] += float(c) * ev
    np.testing.assert_allclose(acc_m, ref, rtol=1e-12, atol=1e-15)
    assert (acc_m <= acc + 1e-15).all()


# --------------------------------------------------------------------------
# Top-K (Eq. 6)
# --------------------------------------------------------------------------

def test_topk_matches_full_sort(oracle_lib):
    rng = np.random.default_rng(1)
    n, C = 400, 32
    acc = rng.exponential(1.0, (n, C)) * (rng.random((n, C)) < 0.4)
    acc[5] = 0.0                       # empty row
    acc[6, :] = 0.0
    acc[6, [3, 9]] = [2.0, 2.0]        # tie -> lower index first
    acc[7, :4] = [-1.0, 0.5, 0.0, 0.25]  # negatives are never kept
    for K in (1, 4, 8, 40):
        idx, val = oracle_lib.topk(acc, K)
        for i in range(n):
            pos = np.nonzero(acc[i] > 0)[0]
            order = pos[np.lexsort((pos, -acc[i, pos]))][:K]
            exp_idx = np.full(K, -1)
            exp_idx[:order.size] = order
            assert idx[i].tolist() == exp_idx.tolist()
            if order.size:
                assert val[i].sum() == pytest.approx(1.0, abs=1e-14)
                np.testing.assert_allclose(val[i, :order.size], acc[i, order] / acc[i, order].sum(), rtol=1e-14)
            assert (val[i, order.size:] == 0).all()
    idx, _ = oracle_lib.topk(acc, 2)
    assert idx[6].tolist() == [3, 9] and idx[5].tolist() == [-1, -1]


# --------------------------------------------------------------------------
# render (Eq. 7), decode (Eq. 8), similarity
# --------------------------------------------------------------------------

def test_round_trip_one_hot(oracle_lib):
    """One region per view with a one-hot code j: every visible Gaussian
    uplifts to (j, 1) and renders back to (1 - T_final) onehot_j."""
    import synth
    base = synth.tiny_workload(13, n=200, width=48, height=40, V=3, C=12)
    wl = single_region_workload(base.scene, base.cams, 12, [(7, 1.0)], 3)
    acc, _, _ = oracle_lib.uplift(wl)
    idx, val = oracle_lib.topk(acc, 3)
    hit = acc.sum(1) > 0
    assert hit.sum() > 20
    assert (idx[hit, 0] == 7).all() and (val[hit, 0] == 1.0).all() and (idx[hit, 1:] == -1).all()
    What, T, risk, _ = oracle_lib.render(base.scene, idx, val, 12, base.cams[0])
    np.testing.assert_allclose(What[..., 7], 1.0 - T, rtol=0, atol=1e-12)
    assert np.abs(np.delete(What, 7, axis=-1)).max() == 0.0


def test_render_reduces_to_weight_sum(oracle_lib):
    """K = 1, C = 1, w^ = 1: What(p) = sum_i e_i(p) = 1 - T_final(p)."""
    import synth
    wl = synth.tiny_workload(14, n=250, width=40, height=32, V=1, log_scale_mean=-2.5)
    idx = np.zeros((wl.scene.n, 1), np.int32)
    val = np.ones((wl.scene.n, 1))
    What, T, _, cnt = oracle_lib.render(wl.scene, idx, val, 1, wl.cams[0])
    np.testing.assert_allclose(What[..., 0], 1.0 - T, atol=1e-12)
    assert cnt["contributions"] > 0


def test_decode_and_similarity(oracle_lib):
    rng = np.random.default_rng(2)
    What = rng.random((7, 9, 16))
    cb = rng.normal(size=(16, 24)).astype(np.float32)
    F = oracle_lib.decode(What, cb)
    np.testing.assert_allclose(F, What @ cb.astype(np.float64), rtol=1e-12)
    text = rng.normal(size=(5, 24)).astype(np.float32)
    F[0, 0] = 0.0
    S = oracle_lib.similarity(F, text)
    t64 = text.astype(np.float64)
    ref = (F @ t64.T) / (np.linalg.norm(F, axis=-1, keepdims=True) * np.linalg.norm(t64, axis=-1))
    ref[0, 0] = 0.0
    np.testing.assert_allclose(S, ref, rtol=1e-12, atol=1e-15)
    # single atom: F = e C[j], cos(F, C[j]) = 1
    W1 = np.zeros((1, 16))
    W1[0, 4] = 0.37
    F1 = oracle_lib.decode(W1, cb)
    np.testing.assert_allclose(F1[0], 0.37 * cb[4].astype(np.float64), rtol=1e-12)
    assert oracle_lib.similarity(F1, cb[4:5])[0, 0] == pytest.approx(1.0, abs=1e-12)
