"""Seeded input generators: determinism and the stated distributions (no GPU)."""
import numpy as np

import synth


def test_voronoi_exact_and_ties():
    seeds = np.array([[2, 2], [6, 2], [4, 6]])
    m = synth.voronoi_map(seeds, 9, 8)
    # brute force with explicit tie-breaking to the lower seed index
    ref = np.zeros((8, 9), np.int32)
    for y in range(8):
        for x in range(9):
            d = [(x - sx) ** 2 + (y - sy) ** 2 for sx, sy in seeds]
            ref[y, x] = int(np.argmin(d))
    assert (m == ref).all()
    assert m[2, 4] == 0  # equidistant from seeds 0 and 1


def test_codes_are_convex_and_distinct():
    rng = np.random.default_rng(0)
    idx, val = synth.region_codes(rng, 500, 64, 8)
    assert (val >= 0).all()
    np.testing.assert_allclose(val.sum(1), 1.0, rtol=1e-6)
    assert all(len(set(r)) == 8 for r in idx.tolist())


def test_cameras_orthonormal_and_look_at_origin():
    for cam in synth.fibonacci_cameras(8, 3.0, 160, 120) + synth.band_cameras(
            np.random.default_rng(1), 5, 3.0, 988, 731):
        vm = cam.viewmat.reshape(3, 4).astype(np.float64)
        R, t = vm[:, :3], vm[:, 3]
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-6)
        assert np.linalg.det(R) > 0.99
        np.testing.assert_allclose(t, [0.0, 0.0, 3.0], atol=1e-5)  # origin straight ahead


def test_cfg1_deterministic():
    a, b = synth.uplift_cfg1(), synth.uplift_cfg1()
    assert np.array_equal(a.scene.means, b.scene.means)
    assert np.array_equal(a.region_maps, b.region_maps)
    assert a.region_maps.max() == 8 * 32 - 1 and a.region_maps.min() == 0
    assert a.scene.n == 10_000 and a.V == 8 and (a.C, a.s, a.K) == (64, 4, 4)
