"""The C-ABI library loads, exports every declared symbol, and validates
arguments on the host (no GPU needed: every call here fails validation
before any CUDA call)."""
import ctypes as ct
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2605_13600_gb300 import build
    build.build()
    from paper_2605_13600_gb300 import _lib
    return _lib


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(scoup_[a-z0-9_]+)\s*\(", src))
    return names


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert {"scoup_uplift", "scoup_topk", "scoup_version"} <= names
    raw = ct.CDLL(lib.LIB_PATH)
    for nm in sorted(names):
        assert hasattr(raw, nm), nm
        assert nm in lib.PROTOS, f"binding lacks {nm}"


def test_version_and_sizes(lib):
    L = lib.load()
    assert b"sm_103a" in L.scoup_version()
    assert L.scoup_uplift_workspace_size(-1, 10, 10, 0) == 0
    assert L.scoup_uplift_workspace_size(10, 0, 10, 0) == 0
    a = L.scoup_uplift_workspace_size(1000, 160, 120, 0)
    b = L.scoup_uplift_workspace_size(1000, 160, 120, 100)
    assert b - a == 2 * 800 and a > 1000 * 32  # two view pipelines, 8 bytes per pair each


def _call_uplift(lib, **kw):
    L = lib.load()
    sc = lib.Scene()
    sc.n = kw.get("n", 4)
    fake = ct.c_void_p(0x10000)  # never dereferenced: validation fails first
    sc.means = sc.scales = sc.opacity = fake
    sc.quats = kw.get("quats", fake)
    cams = (lib.Camera * 1)()
    cams[0].fx = cams[0].fy = kw.get("fx", 100.0)
    cams[0].width, cams[0].height = kw.get("wh", (32, 32))
    offs = (ct.c_int64 * 1)(0)
    st = lib.Stats()
    rc = L.scoup_uplift(ct.byref(sc), ct.cast(cams, ct.c_void_p), kw.get("V", 1), fake,
                        ct.cast(offs, ct.c_void_p), 4, fake, fake, kw.get("s", 2), kw.get("C", 8),
                        kw.get("K", 2), kw.get("accum", fake), kw.get("mode", 0), fake, fake,
                        kw.get("ws", fake), kw.get("ws_bytes", 1 << 30), ct.byref(st), None)
    return rc, L.scoup_last_error().decode()


@pytest.mark.parametrize("kw,frag", [
    ({"K": 0}, "K=0"), ({"K": 9}, "K=9"), ({"C": 2000, "K": 2}, "C=2000"), ({"s": 0}, "s=0"),
    ({"s": 1025}, "s=1025"), ({"V": -1}, "V=-1"), ({"n": -5}, "n=-5"), ({"mode": 8}, "accum_mode"),
    ({"wh": (0, 10)}, "bad size"), ({"fx": 0.0}, "focal"), ({"accum": None}, "accum"),
    ({"ws": None}, "workspace"), ({"ws_bytes": 16}, "workspace too small"),
    ({"quats": ct.c_void_p(0x10004)}, "aligned"),
])
def test_uplift_rejects_bad_arguments(lib, kw, frag):
    rc, msg = _call_uplift(lib, **kw)
    expect = lib.SCOUP_ERR_OOM if frag == "workspace too small" else lib.SCOUP_ERR_INVALID_ARG
    assert rc == expect, msg
    assert frag in msg


def test_topk_rejects_bad_arguments(lib):
    L = lib.load()
    fake = ct.c_void_p(0x10000)
    assert L.scoup_topk(fake, 10, 8, 9, fake, fake, None) == lib.SCOUP_ERR_INVALID_ARG
    assert L.scoup_topk(None, 10, 8, 2, fake, fake, None) == lib.SCOUP_ERR_INVALID_ARG
    assert L.scoup_topk(fake, -1, 8, 2, fake, fake, None) == lib.SCOUP_ERR_INVALID_ARG


def test_render_decode_fused_sizes_and_checks(lib):
    """Workspace layout of scoup_render_decode_fused (decode workspace, bf16
    codes, render workspace) and its host-side argument checks."""
    L = lib.load()
    n, W, H, C, D, dup = 1000, 160, 120, 64, 128, 500
    P = W * H
    al = lambda x: (x + 255) // 256 * 256
    want = al(L.scoup_decode_workspace_size(P, C, D)) + al(P * C * 2) + L.scoup_uplift_workspace_size(n, W, H, dup)
    assert L.scoup_render_decode_workspace_size(n, W, H, C, D, dup) == want
    assert L.scoup_render_decode_workspace_size(n, 0, H, C, D, dup) == 0
    assert L.scoup_render_decode_workspace_size(n, W, H, C, 0, dup) == 0
    sc = lib.Scene()
    sc.n = 4
    fake = ct.c_void_p(0x10000)  # never dereferenced: validation fails first
    sc.means = sc.scales = sc.quats = sc.opacity = fake
    cams = (lib.Camera * 1)()
    cams[0].fx = cams[0].fy = 100.0
    cams[0].width, cams[0].height = W, H
    for kw, frag in (({"C": 12}, "C=12"), ({"D": 40}, "D=40"), ({"ws_bytes": 1024}, "workspace too small")):
        rc = L.scoup_render_decode_fused(ct.byref(sc), fake, fake, 4, kw.get("C", C), ct.cast(cams, ct.POINTER(lib.Camera)),
                                         fake, kw.get("D", D), fake, 1, None, None, None, fake,
                                         kw.get("ws_bytes", 1 << 30), None, None)
        assert rc != 0 and frag in L.scoup_last_error().decode(), (kw, L.scoup_last_error())


def test_chunked_form_sizes_and_checks(lib):
    """Workspace layout of the chunked form (SCOUP_UPLIFT_CHUNKED): the scene
    part, then 2 x 8 view parts each holding dup_capacity 8-byte keys; with
    host maps a 16-slot staging ring in front.  A workspace below the chunked
    layout is refused before any device work."""
    L = lib.load()
    n, W, H, dup = 1000, 160, 120, 100
    al = lambda x: (x + 255) // 256 * 256
    a = L.scoup_uplift_chunked_workspace_size(n, W, H, 0)
    b = L.scoup_uplift_chunked_workspace_size(n, W, H, dup)
    assert b - a == 16 * al(8 * dup)
    assert a > L.scoup_uplift_workspace_size(n, W, H, 0)  # 16 view parts against 2
    assert L.scoup_uplift_host_maps_chunked_workspace_size(n, W, H, dup) == al(16 * W * H * 4) + b
    for bad in ((-1, W, H, dup), (n, 0, H, dup), (n, W, H, -1)):
        assert L.scoup_uplift_chunked_workspace_size(*bad) == 0
        assert L.scoup_uplift_host_maps_chunked_workspace_size(*bad) == 0
    # a per-view sized workspace does not hold the chunked layout
    ws_bytes = L.scoup_uplift_workspace_size(4, 32, 32, 10)
    rc, msg = _call_uplift(lib, n=4, mode=4, wh=(32, 32), ws_bytes=ws_bytes)
    assert rc == lib.SCOUP_ERR_OOM and "chunked form" in msg, msg


def test_uplift_host_maps_sizes_and_checks(lib):
    """Workspace layout of scoup_uplift_host_maps (a 4-slot staging ring of
    view maps, then a scoup_uplift workspace) and its host-side checks."""
    L = lib.load()
    n, W, H, dup = 1000, 160, 120, 500
    al = lambda x: (x + 255) // 256 * 256
    assert L.scoup_uplift_host_maps_workspace_size(n, W, H, dup) == al(4 * W * H * 4) + L.scoup_uplift_workspace_size(n, W, H, dup)
    assert L.scoup_uplift_host_maps_workspace_size(n, 0, H, dup) == 0
    sc = lib.Scene()
    sc.n = 4
    fake = ct.c_void_p(0x10000)  # never dereferenced: validation fails first
    sc.means = sc.scales = sc.quats = sc.opacity = fake
    cams = (lib.Camera * 1)()
    cams[0].fx = cams[0].fy = 100.0
    offs = (ct.c_int64 * 1)(0)
    for wh, ws_bytes, frag in (((0, 10), 1 << 30, "bad size"), ((W, H), 1024, "staging ring")):
        cams[0].width, cams[0].height = wh
        rc = L.scoup_uplift_host_maps(ct.byref(sc), ct.cast(cams, ct.c_void_p), 1, fake, ct.cast(offs, ct.c_void_p),
                                      4, fake, fake, 2, 8, 2, fake, 0, fake, fake, fake, ws_bytes, None, None)
        assert rc != 0 and frag in L.scoup_last_error().decode(), (wh, L.scoup_last_error())


def test_relevancy_rejects_bad_alpha(lib):
    """Eq. 9's minimum over canonical phrases is taken at the largest canonical
    similarity, which needs alpha > 0: zero, negative and non-finite alphas
    are refused before any launch."""
    L = lib.load()
    fake = ct.c_void_p(0x10000)
    for a in (0.0, -1.0, float("inf"), float("nan")):
        assert L.scoup_relevancy(fake, 10, 8, 2, a, fake, None) != 0
        assert "alpha" in L.scoup_last_error().decode()
    assert L.scoup_relevancy(fake, 10, 2, 2, 10.0, fake, None) != 0  # no query column


def test_red_throughput_rejects_bad_arguments(lib):
    f = lib.load().scoup_selftest_red_throughput
    assert f(None, 20, 10, 1, None) == lib.SCOUP_ERR_INVALID_ARG
    assert f(ct.c_void_p(256), 9, 10, 1, None) == lib.SCOUP_ERR_INVALID_ARG
    assert f(ct.c_void_p(256), 32, 10, 1, None) == lib.SCOUP_ERR_INVALID_ARG
    assert f(ct.c_void_p(256), 20, -1, 1, None) == lib.SCOUP_ERR_INVALID_ARG


def test_similarity_relevancy_rejects_bad_arguments(lib):
    f = lib.load().scoup_similarity_relevancy
    buf = ct.c_void_p(256)
    # Q must be 16 or 32; Q - n_canon a multiple of 4; alpha positive
    assert f(buf, 10, 512, None, buf, 28, 4, 10.0, buf, buf, 1 << 20, None) == lib.SCOUP_ERR_INVALID_ARG
    assert f(buf, 10, 512, None, buf, 32, 3, 10.0, buf, buf, 1 << 20, None) == lib.SCOUP_ERR_INVALID_ARG
    assert f(buf, 10, 512, None, buf, 32, 0, 10.0, buf, buf, 1 << 20, None) == lib.SCOUP_ERR_INVALID_ARG
    assert f(buf, 10, 512, None, buf, 32, 4, 0.0, buf, buf, 1 << 20, None) == lib.SCOUP_ERR_INVALID_ARG


def test_decode_query_rejects_bad_arguments(lib):
    """Argument checks of the decode with the query unit, before any device work."""
    f = lib.load().scoup_decode_query
    buf = ct.c_void_p(256)
    ws = 1 << 30
    # scoup_decode_query(codes, codes_dtype, P, C, codebook, D, text, Q, n_canon, alpha,
    #                    features, feat_norm2, out, workspace, ws_bytes, stream)
    ok = dict(Q=32, n_canon=0, alpha=10.0, C=256, D=512, dt=1)

    def call(**kw):
        a = dict(ok, **kw)
        return f(buf, a["dt"], 10, a["C"], buf, a["D"], buf, a["Q"], a["n_canon"], a["alpha"], None, None, buf,
                 buf, ws, None)
    assert call(Q=48) == lib.SCOUP_ERR_INVALID_ARG              # one 16- or 32-column unit
    assert call(Q=24) == lib.SCOUP_ERR_INVALID_ARG
    assert call(n_canon=3) == lib.SCOUP_ERR_INVALID_ARG         # Q - n_canon a multiple of 4
    assert call(n_canon=32) == lib.SCOUP_ERR_INVALID_ARG        # at least one query
    assert call(n_canon=4, alpha=0.0) == lib.SCOUP_ERR_INVALID_ARG
    assert call(C=12) == lib.SCOUP_ERR_INVALID_ARG              # C a multiple of 8
    assert call(D=40) == lib.SCOUP_ERR_INVALID_ARG              # D a multiple of 16
    assert call(dt=2) == lib.SCOUP_ERR_INVALID_ARG
    # misaligned output, and a workspace that is too small
    assert f(buf, 1, 10, 256, buf, 512, buf, 32, 0, 10.0, None, None, ct.c_void_p(260), buf, ws, None) == \
        lib.SCOUP_ERR_INVALID_ARG
    need = lib.load().scoup_decode_query_workspace_size(10, 256, 512, 32)
    assert need > 0
    assert f(buf, 1, 10, 256, buf, 512, buf, 32, 0, 10.0, None, None, buf, buf, need - 1, None) == \
        lib.SCOUP_ERR_OOM
