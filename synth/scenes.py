"""Seeded synthetic stand-ins for the paper's pretrained 3DGS scenes and SAM/CLIP codes.

The paper evaluates on LERF-OVS, Mip-NeRF360 and 3D-OVS scenes (Sec. 5); none of
them (nor SAM/CLIP weights) is available, so every input here is drawn from a
NumPy ``default_rng(seed)`` (PCG64) with the shapes and value distributions of
those workloads:

* Gaussians (Sec. 3): means uniform in [-1, 1]^3 or 64 clustered blobs
  (sigma 0.2), linear scales exp(N(-4, 0.5)) per axis, unit quaternions
  normalize(N(0, 1)^4) in (w, x, y, z) order, opacity sigmoid(N(0, 1.5)).
* Pinhole cameras looking at the origin, world-to-camera 3x4 row-major,
  camera x right / y down / z forward, fx = fy = W / (2 tan(fov_x / 2)),
  principal point at the image centre.
* Region maps (Sec. 4.1): a Voronoi partition per view, seeds at integer pixel
  positions, nearest seed by integer squared distance, ties to the lower seed
  index.  Computed with exact integer arithmetic so CPU and GPU agree bit for
  bit.
* Sparse region codes (Eq. 4): s distinct atoms per region, Dirichlet(1)
  coefficients (nonnegative, summing to one).

Nothing here implements the uplift itself.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

__all__ = [
    "Scene", "Camera", "UpliftWorkload", "RenderWorkload",
    "gaussians", "look_at", "camera_at", "fibonacci_cameras", "band_cameras",
    "voronoi_map", "region_codes", "sparse_topk_codes", "unit_rows",
    "tiny_workload", "uplift_cfg1", "uplift_cfg2", "uplift_cfg3_scene",
    "render_cfg4", "render_cfg5", "uplift_cfg5", "dense_feature_codes", "level_workloads",
]


@dataclass
class Scene:
    means: np.ndarray      # float32 [n, 3]
    scales: np.ndarray     # float32 [n, 3]  (linear, already exp'ed)
    quats: np.ndarray      # float32 [n, 4]  (w, x, y, z), unit norm
    opacity: np.ndarray    # float32 [n]     (already sigmoid'ed)

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        return Scene(self.means[idx].copy(), self.scales[idx].copy(),
                     self.quats[idx].copy(), self.opacity[idx].copy())


@dataclass
class Camera:
    viewmat: np.ndarray    # float32 [12], world->camera 3x4 row-major
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int

    def as_array(self) -> np.ndarray:
        """16 float32 values: viewmat[12], fx, fy, cx, cy."""
        return np.concatenate([self.viewmat.astype(np.float32),
                               np.array([self.fx, self.fy, self.cx, self.cy], np.float32)])


@dataclass
class UpliftWorkload:
    name: str
    scene: Scene
    cams: List[Camera]
    region_maps: np.ndarray   # int32, packed sum_v H_v*W_v, global code-table rows, -1 = none
    map_offsets: np.ndarray   # int64 [V+1]
    code_idx: np.ndarray      # int32 [R_total, s], -1 = padding
    code_val: np.ndarray      # float32 [R_total, s]
    C: int
    s: int
    K: int
    regions_per_view: List[int] = field(default_factory=list)

    @property
    def V(self) -> int:
        return len(self.cams)

    def region_map(self, v: int) -> np.ndarray:
        c = self.cams[v]
        return self.region_maps[self.map_offsets[v]:self.map_offsets[v + 1]].reshape(c.height, c.width)


@dataclass
class RenderWorkload:
    name: str
    scene: Scene
    cams: List[Camera]
    topk_idx: np.ndarray      # int32 [n, K], -1 = padding
    topk_val: np.ndarray      # float32 [n, K]
    C: int
    K: int
    codebook: Optional[np.ndarray] = None  # float32 [C, D], unit-norm rows
    text: Optional[np.ndarray] = None      # float32 [Q, D], unit-norm rows


# ----------------------------------------------------------------------------
# Gaussians
# ----------------------------------------------------------------------------

def gaussians(rng: np.random.Generator, n: int, layout: str = "uniform",
              n_blobs: int = 64, blob_sigma: float = 0.2,
              log_scale_mean: float = -4.0, log_scale_std: float = 0.5,
              opacity_logit_std: float = 1.5) -> Scene:
    if layout == "uniform":
        means = rng.uniform(-1.0, 1.0, size=(n, 3))
    elif layout == "blobs":
        centres = rng.uniform(-1.0, 1.0, size=(n_blobs, 3))
        which = rng.integers(0, n_blobs, size=n)
        means = centres[which] + rng.normal(0.0, blob_sigma, size=(n, 3))
    else:
        raise ValueError(layout)
    scales = np.exp(rng.normal(log_scale_mean, log_scale_std, size=(n, 3)))
    q = rng.normal(0.0, 1.0, size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    opacity = 1.0 / (1.0 + np.exp(-rng.normal(0.0, opacity_logit_std, size=n)))
    return Scene(means.astype(np.float32), scales.astype(np.float32),
                 q.astype(np.float32), opacity.astype(np.float32))


# ----------------------------------------------------------------------------
# Cameras
# ----------------------------------------------------------------------------

def look_at(position, target=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """World->camera 3x4 (row-major) for a camera at `position` looking at
    `target`; camera axes x right, y down, z forward."""
    c = np.asarray(position, np.float64)
    f = np.asarray(target, np.float64) - c
    f /= np.linalg.norm(f)
    u = np.asarray(up, np.float64)
    if abs(np.dot(f, u / np.linalg.norm(u))) > 0.999:
        u = np.array([0.0, 1.0, 0.0])
    x = np.cross(f, u)
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    R = np.stack([x, y, f])
    t = -R @ c
    return np.concatenate([R, t[:, None]], axis=1).reshape(12)


def camera_at(position, width: int, height: int, fov_x_deg: float = 60.0,
              target=(0.0, 0.0, 0.0)) -> Camera:
    f = width / (2.0 * math.tan(math.radians(fov_x_deg) / 2.0))
    return Camera(look_at(position, target).astype(np.float32), float(np.float32(f)),
                  float(np.float32(f)), float(np.float32(width / 2.0)),
                  float(np.float32(height / 2.0)), int(width), int(height))


def fibonacci_cameras(V: int, radius: float, width: int, height: int,
                      fov_x_deg: float = 60.0) -> List[Camera]:
    golden = math.pi * (3.0 - math.sqrt(5.0))
    cams = []
    for i in range(V):
        z = 1.0 - 2.0 * (i + 0.5) / V
        rr = math.sqrt(max(0.0, 1.0 - z * z))
        th = golden * i
        pos = radius * np.array([rr * math.cos(th), rr * math.sin(th), z])
        cams.append(camera_at(pos, width, height, fov_x_deg))
    return cams


def band_cameras(rng: np.random.Generator, V: int, radius: float, width: int,
                 height: int, fov_x_deg: float = 60.0,
                 elev_deg=(-20.0, 30.0)) -> List[Camera]:
    elev = np.radians(rng.uniform(elev_deg[0], elev_deg[1], size=V))
    cams = []
    for k in range(V):
        az = 2.0 * math.pi * k / V
        pos = radius * np.array([math.cos(elev[k]) * math.cos(az),
                                 math.cos(elev[k]) * math.sin(az),
                                 math.sin(elev[k])])
        cams.append(camera_at(pos, width, height, fov_x_deg))
    return cams


# ----------------------------------------------------------------------------
# Region maps and codes
# ----------------------------------------------------------------------------

def voronoi_map(seeds_xy: np.ndarray, width: int, height: int, device: str = "cpu") -> np.ndarray:
    """Nearest-seed label per pixel (int32 [H, W]); exact integer arithmetic:
    key = d2 * R + seed_index, the minimum key gives the nearest seed with ties
    going to the lower index."""
    import torch
    R = int(seeds_xy.shape[0])
    sx = torch.as_tensor(seeds_xy[:, 0].astype(np.int64), device=device)
    sy = torch.as_tensor(seeds_xy[:, 1].astype(np.int64), device=device)
    sidx = torch.arange(R, device=device, dtype=torch.int64)
    out = torch.empty(height * width, dtype=torch.int64, device=device)
    xs_all = torch.arange(width, device=device, dtype=torch.int64)
    # chunking only bounds memory: the integer keys make the result independent of it
    budget = (1 << 26) if str(device).startswith("cuda") else (1 << 22)
    rows_per_chunk = max(1, budget // max(1, width * R))
    for y0 in range(0, height, rows_per_chunk):
        y1 = min(height, y0 + rows_per_chunk)
        ys = torch.arange(y0, y1, device=device, dtype=torch.int64)
        px = xs_all.repeat(y1 - y0)
        py = ys.repeat_interleave(width)
        d2 = (px[:, None] - sx[None, :]) ** 2 + (py[:, None] - sy[None, :]) ** 2
        key = d2 * R + sidx[None, :]
        out[y0 * width:y1 * width] = key.min(dim=1).values % R
    return out.to(torch.int32).cpu().numpy().reshape(height, width)


def region_codes(rng: np.random.Generator, R: int, C: int, s: int):
    """s distinct atoms per region with Dirichlet(1) weights (Eq. 4)."""
    idx = np.argsort(rng.random((R, C)), axis=1)[:, :s].astype(np.int32)
    w = rng.exponential(1.0, size=(R, s))
    w /= w.sum(axis=1, keepdims=True)
    return idx, w.astype(np.float32)


def sparse_topk_codes(rng: np.random.Generator, n: int, C: int, K: int):
    """Random K-sparse per-Gaussian codes (distinct atoms, Dirichlet(1) values)."""
    return region_codes(rng, n, C, K)


def unit_rows(rng: np.random.Generator, rows: int, dim: int) -> np.ndarray:
    x = rng.normal(0.0, 1.0, size=(rows, dim))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    return x.astype(np.float32)


def dense_feature_codes(wl: "UpliftWorkload", D: int = 512, seed: int = 7) -> "UpliftWorkload":
    """The same views and regions with a dense D-dimensional unit feature per
    region (a synthetic stand-in for per-mask CLIP features) written as a code
    over C = D + 1 atoms: atoms 0..D-1 carry the feature, atom D carries 1, so
    an accumulate-only uplift gives sum e F in columns 0..D-1 and Z in column D
    (dense feature uplift, Eq. 3, as the same aggregation)."""
    rng = np.random.default_rng(seed)
    R = int(wl.code_idx.shape[0])
    feats = unit_rows(rng, R, D)
    ci = np.tile(np.arange(D + 1, dtype=np.int32), (R, 1))
    cv = np.concatenate([feats, np.ones((R, 1), np.float32)], axis=1)
    out = UpliftWorkload(f"{wl.name}_dense{D}", wl.scene, wl.cams, wl.region_maps, wl.map_offsets,
                         ci, cv, D + 1, D + 1, D + 1, wl.regions_per_view)
    out.region_features = feats
    return out


def level_workloads(base: "UpliftWorkload", R_levels=(8, 32, 128), seed: int = 11,
                    device: str = "cpu") -> List["UpliftWorkload"]:
    """Semantic levels over the scene and views of `base` (coarse to fine, like
    SAM's whole / part / subpart masks): the finest level partitions every
    view into R_levels[-1] Voronoi regions; level l merges them into
    R_levels[l] groups (fine local id * R_l // R_fine), so the levels nest.
    Each level has its own Dirichlet codes (base C, s, K)."""
    rng = np.random.default_rng(seed)
    R_fine = int(R_levels[-1])
    seeds = _draw_seeds(rng, base.cams, [R_fine] * len(base.cams))
    local = [voronoi_map(sd, c.width, c.height, device=device).reshape(-1) for sd, c in zip(seeds, base.cams)]
    offs = np.zeros(len(base.cams) + 1, np.int64)
    for v, c in enumerate(base.cams):
        offs[v + 1] = offs[v] + c.width * c.height
    out = []
    for l, R in enumerate(R_levels):
        R = int(R)
        maps = np.concatenate([(m.astype(np.int64) * R // R_fine + v * R).astype(np.int32)
                               for v, m in enumerate(local)]) if local else np.zeros(0, np.int32)
        ci, cv = region_codes(rng, R * len(base.cams), base.C, base.s)
        out.append(UpliftWorkload(f"{base.name}_level{l}", base.scene, base.cams, maps, offs, ci, cv,
                                  base.C, base.s, base.K, [R] * len(base.cams)))
    return out


def _draw_seeds(rng, cams, R_per_view):
    return [np.stack([rng.integers(0, cam.width, size=R), rng.integers(0, cam.height, size=R)], axis=1)
            for cam, R in zip(cams, R_per_view)]


def _pack_maps(seeds, cams, device):
    maps, offs, rpv = [], [0], []
    base = 0
    for cam, sd in zip(cams, seeds):
        m = voronoi_map(sd, cam.width, cam.height, device=device)
        maps.append((m + base).astype(np.int32).reshape(-1))
        offs.append(offs[-1] + cam.width * cam.height)
        rpv.append(int(sd.shape[0]))
        base += int(sd.shape[0])
    return np.concatenate(maps), np.array(offs, np.int64), rpv, base


# ----------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------

def tiny_workload(seed: int, n: int = 200, width: int = 48, height: int = 40,
                  V: int = 2, R: int = 6, C: int = 16, s: int = 3, K: int = 3,
                  layout: str = "uniform", radius: float = 3.0,
                  log_scale_mean: float = -3.0, fov_x_deg: float = 60.0) -> UpliftWorkload:
    """Small random scenes for brute-force and parity checks."""
    rng = np.random.default_rng(seed)
    scene = gaussians(rng, n, layout, log_scale_mean=log_scale_mean, n_blobs=4)
    cams = band_cameras(rng, V, radius, width, height, fov_x_deg)
    maps, offs, rpv, R_tot = _pack_maps(_draw_seeds(rng, cams, [R] * V), cams, "cpu")
    ci, cv = region_codes(rng, R_tot, C, s)
    return UpliftWorkload(f"tiny{seed}", scene, cams, maps, offs, ci, cv, C, s, K, rpv)


def uplift_cfg1() -> UpliftWorkload:
    """10k uniform Gaussians, 8 Fibonacci-sphere views at 160x120, 32 regions
    per view, C=64, s=4, K=4 (seed 1)."""
    rng = np.random.default_rng(1)
    scene = gaussians(rng, 10_000, "uniform")
    cams = fibonacci_cameras(8, 3.0, 160, 120, 60.0)
    maps, offs, rpv, R_tot = _pack_maps(_draw_seeds(rng, cams, [32] * 8), cams, "cpu")
    ci, cv = region_codes(rng, R_tot, 64, 4)
    return UpliftWorkload("cfg1_tiny_10k_8v_160x120", scene, cams, maps, offs, ci, cv, 64, 4, 4, rpv)


def uplift_cfg2(device: str = "cpu", n: int = 1_000_000, V: int = 200) -> UpliftWorkload:
    """1M Gaussians in 64 blobs, 200 sphere-band views at 988x731, 200 regions
    per view, C=256, s=8, K=8 (seed 2).  `n`/`V` shrink it for bounded samples."""
    rng = np.random.default_rng(2)
    scene = gaussians(rng, 1_000_000, "blobs")
    cams = band_cameras(rng, 200, 3.0, 988, 731, 60.0)
    seeds = _draw_seeds(rng, cams, [200] * 200)
    ci, cv = region_codes(rng, 200 * 200, 256, 8)
    maps, offs, rpv, R_tot = _pack_maps(seeds[:V], cams[:V], device)
    if n < scene.n:
        scene = scene.subset(np.arange(n))
    return UpliftWorkload("cfg2_paper_1M_200v_988x731", scene, cams[:V], maps, offs,
                          ci[:R_tot], cv[:R_tot], 256, 8, 8, rpv)


def uplift_cfg3_scene(b: int, device: str = "cpu") -> UpliftWorkload:
    """Scene b of the 16-scene batch: N log-uniform in [2e5, 2e6], V in
    {50..300}, width in {640..1296} (multiple of 8), H = 0.747 W clamped to
    [480, 968]; C=256, s=8, K=8 (seed 300 + b)."""
    rng = np.random.default_rng(300 + b)
    n = int(math.floor(math.exp(rng.uniform(math.log(2e5), math.log(2e6)))))
    V = int(rng.integers(50, 301))
    width = int(rng.integers(640, 1297)) // 8 * 8
    height = int(min(968, max(480, round(0.747 * width))))
    scene = gaussians(rng, n, "blobs")
    cams = band_cameras(rng, V, 3.0, width, height, 60.0)
    seeds = _draw_seeds(rng, cams, [200] * V)
    ci, cv = region_codes(rng, 200 * V, 256, 8)
    maps, offs, rpv, R_tot = _pack_maps(seeds, cams, device)
    return UpliftWorkload(f"cfg3_scene{b}_{n}_{V}v_{width}x{height}", scene, cams, maps, offs,
                          ci, cv, 256, 8, 8, rpv)


def render_cfg4(topk_idx: Optional[np.ndarray] = None, topk_val: Optional[np.ndarray] = None,
                n_views: int = 64) -> RenderWorkload:
    """cfg2's 1M Gaussians with K=8 codes rendered to 64 band views at
    1920x1080; 256x512 unit-norm codebook and 32 unit text vectors (seed 4).
    Without a Top-K from the uplift, random K-sparse codes stand in."""
    scene = gaussians(np.random.default_rng(2), 1_000_000, "blobs")
    rng = np.random.default_rng(4)
    cams = band_cameras(rng, 64, 3.0, 1920, 1080, 60.0)[:n_views]
    codebook = unit_rows(rng, 256, 512)
    text = unit_rows(rng, 32, 512)
    if topk_idx is None:
        topk_idx, topk_val = sparse_topk_codes(rng, scene.n, 256, 8)
    return RenderWorkload("cfg4_render_1M_64v_1920x1080", scene, cams, topk_idx, topk_val,
                          256, 8, codebook, text)


def uplift_cfg5(n: int = 500_000, V: int = 32, width: int = 800, height: int = 600, R: int = 200,
                C: int = 256, s: int = 8, K: int = 8, D: int = 512, seed: int = 5, device: str = "cpu"):
    """The differentiable-render workload with its own uplift inputs: n blob
    Gaussians, V band views, R Voronoi regions per view with s-sparse codes
    over C atoms, Top-K of K (the Top-K comes from uplifting these inputs),
    and a C x D unit-norm codebook.  The loss targets are the decoded region
    codes, F*(p) = code_{r(p)} C.  Returns (UpliftWorkload, codebook)."""
    rng = np.random.default_rng(seed)
    scene = gaussians(rng, n, "blobs")
    cams = band_cameras(rng, V, 3.0, width, height, 60.0)
    maps, offs, rpv, R_tot = _pack_maps(_draw_seeds(rng, cams, [R] * V), cams, device)
    ci, cv = region_codes(rng, R_tot, C, s)
    codebook = unit_rows(rng, C, D)
    wl = UpliftWorkload(f"cfg5_diff_render_{n}_{V}v_{width}x{height}", scene, cams, maps, offs, ci, cv, C, s, K, rpv)
    return wl, codebook


def render_cfg5(n: int = 500_000, V: int = 32) -> RenderWorkload:
    """500k blob Gaussians, 32 band views at 800x600, K=8 of C=256 (seed 5),
    random K-sparse codes (for backward checks that need no uplift; the
    benchmark's differentiable-render leg uses uplift_cfg5's own uplift)."""
    rng = np.random.default_rng(5)
    scene = gaussians(rng, n, "blobs")
    cams = band_cameras(rng, V, 3.0, 800, 600, 60.0)
    idx, val = sparse_topk_codes(rng, n, 256, 8)
    codebook = unit_rows(rng, 256, 512)
    return RenderWorkload("cfg5_diff_render_500k_32v_800x600", scene, cams, idx, val, 256, 8, codebook)
