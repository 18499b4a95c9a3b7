"""FP64 CPU oracle for SCOUP sparse code uplift -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library (``paper_2605_13600_gb300``) and never imports it.

The C source (``scoup_oracle.c``) restates the paper's definitions:
Eq. 2 (front-to-back compositing weights), Eq. 5 and Algorithm 1 (sparse
coefficient uplift), Eq. 6 (Top-K + L1 normalisation), Eq. 7 (sparse
coefficient rendering), Eq. 8 (codebook decode), cosine similarity (App. B)
and the gradient of an L2 feature loss through Eq. 7 (derived from Eqs. 2, 7).
Its header explains which discrete decisions are taken in binary32 and why.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "scoup_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

STOP_MARGIN = 1e-2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no contraction of a*b+c, IEEE semantics)."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
                os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "scoup_oracle.h"))):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-frounding-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


class Camera(ct.Structure):
    _fields_ = [("viewmat", ct.c_float * 12), ("fx", ct.c_float), ("fy", ct.c_float),
                ("cx", ct.c_float), ("cy", ct.c_float), ("width", ct.c_int32),
                ("height", ct.c_int32)]


class Counts(ct.Structure):
    _fields_ = [("visible", ct.c_int64), ("duplicates", ct.c_int64), ("evaluated", ct.c_int64),
                ("contributions", ct.c_int64), ("at_risk", ct.c_int64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class Proj(ct.Structure):
    _fields_ = [("visible", ct.c_int32), ("rect", ct.c_int32 * 4), ("depth", ct.c_float),
                ("mx", ct.c_float), ("my", ct.c_float), ("qa", ct.c_float), ("qb", ct.c_float),
                ("qc", ct.c_float), ("radius", ct.c_float), ("mx64", ct.c_double),
                ("my64", ct.c_double), ("ca64", ct.c_double), ("cb64", ct.c_double),
                ("cc64", ct.c_double)]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ct.CDLL(_LIB)
        P = ct.c_void_p
        i64, i32 = ct.c_int64, ct.c_int
        lib.orc_project.argtypes = [P, P, P, ct.POINTER(Camera), ct.POINTER(Proj)]
        lib.orc_project.restype = None
        lib.orc_power_f32.argtypes = [ct.POINTER(Proj), i32, i32]
        lib.orc_power_f32.restype = ct.c_float
        lib.orc_pixel_list.argtypes = [P, P, P, P, i64, ct.POINTER(Camera), i32, i32, i32, i32,
                                       P, P, P, P]
        lib.orc_pixel_list.restype = i32
        lib.orc_uplift.argtypes = [P, P, P, P, i64, P, i32, P, P, P, P, i32, i32, i32, P, i64,
                                   P, P, ct.POINTER(Counts), i32]
        lib.orc_uplift.restype = i32
        lib.orc_topk.argtypes = [P, i64, i32, i32, P, P]
        lib.orc_topk.restype = i32
        lib.orc_render.argtypes = [P, P, P, P, i64, P, P, i32, i32, ct.POINTER(Camera), P, P, P,
                                   ct.POINTER(Counts), i32]
        lib.orc_render.restype = i32
        lib.orc_decode.argtypes = [P, i64, i32, P, i32, P]
        lib.orc_decode.restype = None
        lib.orc_similarity.argtypes = [P, i64, i32, P, i32, P]
        lib.orc_similarity.restype = None
        lib.orc_entropy.argtypes = [P, i64, i32, P]
        lib.orc_entropy.restype = None
        lib.orc_entropy_filter.argtypes = [P, i64, i64, P]
        lib.orc_entropy_filter.restype = None
        lib.orc_relevancy.argtypes = [P, P, i64, i32, ct.c_double, P]
        lib.orc_relevancy.restype = None
        lib.orc_render_backward.argtypes = [P, P, P, P, i64, P, P, i32, i32, ct.POINTER(Camera),
                                            P, P, P]
        lib.orc_render_backward.restype = i32
        _lib = lib
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ct.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def camera(cam) -> Camera:
    c = Camera()
    for k in range(12):
        c.viewmat[k] = float(cam.viewmat[k])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def _scene(scene):
    return _f32(scene.means), _f32(scene.scales), _f32(scene.quats), _f32(scene.opacity)


def project(scene, cam, i: int) -> Proj:
    """Projection of Gaussian i (binary32 decision path + FP64 value path)."""
    lib = _load()
    m, s, q, _ = _scene(scene)
    out = Proj()
    lib.orc_project(_p(m[i]), _p(s[i]), _p(q[i]), ct.byref(camera(cam)), ct.byref(out))
    return out


def power_f32(proj: Proj, x: int, y: int) -> float:
    return float(_load().orc_power_f32(ct.byref(proj), int(x), int(y)))


def pixel_list(scene, cam, x: int, y: int, brute: bool = False, cap: int = 1 << 16):
    """(gids, e, alpha, T_final) of pixel (x, y), front to back."""
    lib = _load()
    m, s, q, o = _scene(scene)
    gid = np.zeros(cap, np.int32)
    e = np.zeros(cap, np.float64)
    al = np.zeros(cap, np.float64)
    T = np.zeros(1, np.float64)
    nh = lib.orc_pixel_list(_p(m), _p(s), _p(q), _p(o), scene.n, ct.byref(camera(cam)), int(x),
                            int(y), int(brute), cap, _p(gid), _p(e), _p(al), _p(T))
    if nh < 0:
        raise RuntimeError("orc_pixel_list failed")
    return gid[:nh].copy(), e[:nh].copy(), al[:nh].copy(), float(T[0])


def uplift(wl, rows: Optional[Sequence[int]] = None, nthreads: int = 0, views=None):
    """Raw uplift accumulators (Eq. 5 without Z_i).

    Returns (acc [n or len(rows), C] FP64, risk [same] FP64, counts dict)."""
    lib = _load()
    m, s, q, o = _scene(wl.scene)
    vsel = list(range(wl.V)) if views is None else list(views)
    cams = (Camera * max(1, len(vsel)))()
    offs = np.zeros(len(vsel) + 1, np.int64)
    maps = []
    for k, v in enumerate(vsel):
        cams[k] = camera(wl.cams[v])
        mv = wl.region_maps[wl.map_offsets[v]:wl.map_offsets[v + 1]]
        maps.append(mv)
        offs[k + 1] = offs[k] + mv.size
    maps = _i32(np.concatenate(maps) if maps else np.zeros(1, np.int32))
    rows_a = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    nout = wl.scene.n if rows_a is None else rows_a.size
    acc = np.zeros((nout, wl.C), np.float64)
    risk = np.zeros((nout, wl.C), np.float64)
    cnt = Counts()
    ci, cv = _i32(wl.code_idx), _f32(wl.code_val)
    rc = lib.orc_uplift(_p(m), _p(s), _p(q), _p(o), wl.scene.n, ct.cast(cams, ct.c_void_p),
                        len(vsel), _p(maps), _p(offs), _p(ci), _p(cv), wl.s, wl.C, wl.K,
                        _p(rows_a), 0 if rows_a is None else rows_a.size, _p(acc), _p(risk),
                        ct.byref(cnt), int(nthreads))
    if rc != 0:
        raise RuntimeError("orc_uplift failed")
    return acc, risk, cnt.as_dict()


def topk(acc: np.ndarray, K: int):
    lib = _load()
    a = _f64(acc)
    n, C = a.shape
    idx = np.zeros((n, K), np.int32)
    val = np.zeros((n, K), np.float64)
    if lib.orc_topk(_p(a), n, C, K, _p(idx), _p(val)) != 0:
        raise RuntimeError("orc_topk failed")
    return idx, val


def render(scene, topk_idx, topk_val, C: int, cam, nthreads: int = 0):
    """(What [H, W, C], T_final [H, W], risk [H, W] bool, counts) for one view (Eq. 7)."""
    lib = _load()
    m, s, q, o = _scene(scene)
    ti, tv = _i32(topk_idx), _f64(topk_val)
    K = ti.shape[1]
    H, W = cam.height, cam.width
    What = np.zeros((H, W, C), np.float64)
    T = np.zeros((H, W), np.float64)
    risk = np.zeros((H, W), np.uint8)
    cnt = Counts()
    rc = lib.orc_render(_p(m), _p(s), _p(q), _p(o), scene.n, _p(ti), _p(tv), K, C,
                        ct.byref(camera(cam)), _p(What), _p(T), _p(risk), ct.byref(cnt),
                        int(nthreads))
    if rc != 0:
        raise RuntimeError("orc_render failed")
    return What, T, risk.astype(bool), cnt.as_dict()


def decode(What: np.ndarray, codebook: np.ndarray) -> np.ndarray:
    lib = _load()
    Wh = _f64(What).reshape(-1, What.shape[-1])
    cb = _f32(codebook)
    P, C = Wh.shape
    D = cb.shape[1]
    F = np.zeros((P, D), np.float64)
    lib.orc_decode(_p(Wh), P, C, _p(cb), D, _p(F))
    return F.reshape(What.shape[:-1] + (D,))


def similarity(F: np.ndarray, text: np.ndarray) -> np.ndarray:
    lib = _load()
    Fm = _f64(F).reshape(-1, F.shape[-1])
    t = _f32(text)
    P, D = Fm.shape
    Q = t.shape[0]
    out = np.zeros((P, Q), np.float64)
    lib.orc_similarity(_p(Fm), P, D, _p(t), Q, _p(out))
    return out.reshape(F.shape[:-1] + (Q,))


def entropy(acc: np.ndarray) -> np.ndarray:
    """H_i = -sum p log p of each row's positive coefficients (0 for empty rows)."""
    lib = _load()
    a = _f64(acc)
    n, C = a.shape
    H = np.zeros(n, np.float64)
    lib.orc_entropy(_p(a), n, C, _p(H))
    return H


def entropy_filter(H: np.ndarray, keep: int) -> np.ndarray:
    """uint8 mask of the `keep` lowest-entropy rows (ties to the lower index)."""
    lib = _load()
    h = _f64(H)
    m = np.zeros(h.shape[0], np.uint8)
    lib.orc_entropy_filter(_p(h), h.shape[0], int(keep), _p(m))
    return m


def relevancy(s_query: np.ndarray, s_canon: np.ndarray, alpha: float = 10.0) -> np.ndarray:
    """Eq. 9 relevancy from query similarities [P] and canonical similarities [P, k]."""
    lib = _load()
    q = _f64(s_query).reshape(-1)
    c = _f64(s_canon).reshape(q.shape[0], -1)
    R = np.zeros(q.shape[0], np.float64)
    lib.orc_relevancy(_p(q), _p(c), q.shape[0], c.shape[1], float(alpha), _p(R))
    return R


def render_backward(scene, topk_idx, topk_val, C: int, cam, dL_dWhat: np.ndarray):
    """(d_val [n, K], d_opacity [n]) through Eq. 7 for one view."""
    lib = _load()
    m, s, q, o = _scene(scene)
    ti, tv = _i32(topk_idx), _f64(topk_val)
    K = ti.shape[1]
    g = _f64(dL_dWhat)
    dv = np.zeros((scene.n, K), np.float64)
    do = np.zeros(scene.n, np.float64)
    rc = lib.orc_render_backward(_p(m), _p(s), _p(q), _p(o), scene.n, _p(ti), _p(tv), K, C,
                                 ct.byref(camera(cam)), _p(g), _p(dv), _p(do))
    if rc != 0:
        raise RuntimeError("orc_render_backward failed")
    return dv, do
