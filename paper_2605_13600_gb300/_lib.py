"""ctypes loader for libscoup.so (the C ABI declared in include/scoup.h).

Raises immediately if the shared library is missing: there is no CPU or
PyTorch fallback for any entry point.
"""
from __future__ import annotations

import ctypes as ct
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libscoup.so")

SCOUP_OK = 0
SCOUP_ERR_INVALID_ARG = -1
SCOUP_ERR_CUDA = -2
SCOUP_ERR_OOM = -3
SCOUP_ERR_CAPACITY = -4
SCOUP_ERR_DEVICE_CHECK = -5
SCOUP_ERR_TIMEOUT = -6

SCOUP_ACCUM_CONTINUE = 1
SCOUP_ACCUM_COMPENSATED = 2
SCOUP_UPLIFT_CHUNKED = 4


class ScoupError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"scoup error {code}: {msg}")
        self.code = code


class Scene(ct.Structure):
    _fields_ = [("n", ct.c_int64), ("means", ct.c_void_p), ("scales", ct.c_void_p),
                ("quats", ct.c_void_p), ("opacity", ct.c_void_p)]


class Camera(ct.Structure):
    _fields_ = [("viewmat", ct.c_float * 12), ("fx", ct.c_float), ("fy", ct.c_float),
                ("cx", ct.c_float), ("cy", ct.c_float), ("width", ct.c_int32),
                ("height", ct.c_int32)]


class Stats(ct.Structure):
    _fields_ = [("visible", ct.c_int64), ("duplicates", ct.c_int64),
                ("evaluated_pairs", ct.c_int64), ("contributions", ct.c_int64),
                ("flushes", ct.c_int64), ("atomics", ct.c_int64), ("listed", ct.c_int64),
                ("status", ct.c_int32),
                ("max_dups_view", ct.c_int32), ("split_windows", ct.c_int64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class Level(ct.Structure):
    _fields_ = [("region_maps", ct.c_void_p), ("R_total", ct.c_int32), ("code_idx", ct.c_void_p),
                ("code_val", ct.c_void_p), ("s", ct.c_int32)]


class BatchItem(ct.Structure):
    _fields_ = [("scene", Scene), ("cams", ct.c_void_p), ("V", ct.c_int32), ("region_maps", ct.c_void_p),
                ("map_offsets", ct.c_void_p), ("R_total", ct.c_int32), ("code_idx", ct.c_void_p),
                ("code_val", ct.c_void_p), ("s", ct.c_int32), ("accum", ct.c_void_p),
                ("topk_idx", ct.c_void_p), ("topk_val", ct.c_void_p)]


class TuneEntry(ct.Structure):
    _fields_ = [("lanes", ct.c_int32), ("warp_w", ct.c_int32), ("ms", ct.c_float), ("chunk_views", ct.c_int32)]


SCOUP_MAX_TUNE = 24
SCOUP_MAX_CHUNK_VIEWS = 64
SCOUP_BATCH_EAGER = 1


class PlanInfo(ct.Structure):
    _fields_ = [("lanes", ct.c_int32), ("warp_w", ct.c_int32), ("tuned", ct.c_int32),
                ("graph_kernels", ct.c_int32), ("workspace_bytes", ct.c_int64), ("n_tune", ct.c_int32),
                ("tune", TuneEntry * SCOUP_MAX_TUNE), ("chunk_views", ct.c_int32)]


_lib = None

P = ct.c_void_p
I32 = ct.c_int32
I64 = ct.c_int64
SZ = ct.c_size_t

# name -> (restype, argtypes); every entry point of include/scoup.h
PROTOS = {
    "scoup_version": (ct.c_char_p, []),
    "scoup_last_error": (ct.c_char_p, []),
    "scoup_uplift_workspace_size": (SZ, [I64, I32, I32, I64]),
    "scoup_uplift_chunked_workspace_size": (SZ, [I64, I32, I32, I64]),
    "scoup_uplift_host_maps_chunked_workspace_size": (SZ, [I64, I32, I32, I64]),
    "scoup_uplift_plan": (ct.c_int, [ct.POINTER(Scene), P, I32, P, SZ, ct.POINTER(I64), P]),
    "scoup_uplift": (ct.c_int, [ct.POINTER(Scene), P, I32, P, P, I32, P, P, I32, I32, I32, P, I32,
                                P, P, P, SZ, ct.POINTER(Stats), P]),
    "scoup_uplift_host_maps_workspace_size": (SZ, [I64, I32, I32, I64]),
    "scoup_uplift_host_maps": (ct.c_int, [ct.POINTER(Scene), P, I32, P, P, I32, P, P, I32, I32, I32, P, I32,
                                          P, P, P, SZ, ct.POINTER(Stats), P]),
    "scoup_topk": (ct.c_int, [P, I64, I32, I32, P, P, P]),
    "scoup_uplift_levels": (ct.c_int, [ct.POINTER(Scene), P, I32, P, P, I32, I32, I32, P, I32, P, P, P, SZ,
                                       ct.POINTER(Stats), P]),
    "scoup_render": (ct.c_int, [ct.POINTER(Scene), P, P, I32, I32, ct.POINTER(Camera), P, I32, P, P, P, SZ,
                                ct.POINTER(Stats), P]),
    "scoup_render_backward": (ct.c_int, [ct.POINTER(Scene), P, P, I32, I32, ct.POINTER(Camera), P, P, P, P,
                                         SZ, ct.POINTER(Stats), P]),
    "scoup_read_stats": (ct.c_int, [P, SZ, ct.POINTER(Stats), P]),
    "scoup_decode_workspace_size": (SZ, [I64, I32, I32]),
    "scoup_decode": (ct.c_int, [P, I32, I64, I32, P, I32, P, I32, P, P, SZ, P]),
    "scoup_render_decode_workspace_size": (SZ, [I64, I32, I32, I32, I32, I64]),
    "scoup_render_decode_fused": (ct.c_int, [ct.POINTER(Scene), P, P, I32, I32, ct.POINTER(Camera), P, I32, P, I32,
                                             P, P, P, P, SZ, ct.POINTER(Stats), P]),
    "scoup_similarity_workspace_size": (SZ, [I64, I32, I32]),
    "scoup_similarity": (ct.c_int, [P, I64, I32, P, P, I32, P, P, SZ, P]),
    "scoup_decode_fp32": (ct.c_int, [P, I64, I32, P, I32, P, P]),
    "scoup_topk_entropy": (ct.c_int, [P, P, I64, I32, I32, P, P, P, P]),
    "scoup_entropy_filter_workspace_size": (SZ, []),
    "scoup_entropy_filter": (ct.c_int, [P, I64, I64, I32, P, P, P, P, SZ, P]),
    "scoup_relevancy": (ct.c_int, [P, I64, I32, I32, ct.c_float, P, P]),
    "scoup_similarity_fp32": (ct.c_int, [P, I64, I32, P, I32, P, P, SZ, P]),
    "scoup_uplift_noalloc_max_bytes": (SZ, []),
    "scoup_uplift_noalloc": (ct.c_int, [ct.POINTER(Scene), P, I32, P, P, I32, P, P, I32, I32, I32, P, I32,
                                        P, P, ct.POINTER(Stats), P]),
    "scoup_plan_create": (ct.c_int, [P, I32, I32, I32, I32, ct.POINTER(ct.c_void_p), P]),
    "scoup_plan_set": (ct.c_int, [P, I32, I32]),
    "scoup_plan_set_chunk": (ct.c_int, [P, I32]),
    "scoup_autotune": (ct.c_int, [P, I32, P]),
    "scoup_uplift_batched": (ct.c_int, [P, I32, P]),
    "scoup_plan_stats": (ct.c_int, [P, P, P]),
    "scoup_plan_info_get": (ct.c_int, [P, ct.POINTER(PlanInfo)]),
    "scoup_plan_destroy": (ct.c_int, [P]),
    "scoup_selftest_gemm_timeout": (ct.c_int, [P, SZ, P]),
    "scoup_similarity_relevancy": (ct.c_int, [P, ct.c_int64, ct.c_int32, P, P, ct.c_int32, ct.c_int32, ct.c_float,
                                              P, P, SZ, P]),
    "scoup_decode_query_workspace_size": (SZ, [ct.c_int64, ct.c_int32, ct.c_int32, ct.c_int32]),
    "scoup_decode_query": (ct.c_int, [P, ct.c_int32, ct.c_int64, ct.c_int32, P, ct.c_int32, P, ct.c_int32,
                                      ct.c_int32, ct.c_float, P, P, P, P, SZ, P]),
    "scoup_decode_backward_workspace_size": (SZ, [ct.c_int64, ct.c_int32, ct.c_int32]),
    "scoup_decode_backward": (ct.c_int, [P, ct.c_int32, ct.c_int64, ct.c_int32, P, ct.c_int32, P, P, SZ, P]),
    "scoup_decode_backward_fp32": (ct.c_int, [P, ct.c_int64, ct.c_int32, P, ct.c_int32, P, P]),
    "scoup_region_l2_grad_workspace_size": (SZ, [ct.c_int32, ct.c_int32]),
    "scoup_region_l2_grad": (ct.c_int, [P, ct.c_int32, ct.c_int64, ct.c_int32, P, P, P, ct.c_int32, ct.c_int32,
                                        P, ct.c_int32, P, ct.c_int32, P, P, SZ, P]),
    "scoup_selftest_red_throughput": (ct.c_int, [P, ct.c_int32, ct.c_int64, ct.c_uint32, P]),
    "scoup_profile_enable": (ct.c_int, [I32]),
    "scoup_profile_read": (ct.c_int, [P, P, I32]),
    "scoup_launch_count": (I64, []),
}

PHASES = ["reorder", "preprocess", "binning", "uplift_tiles", "topk", "code_topk", "render",
          "render_bwd", "decode", "similarity"]
NUM_PHASES = 16


def load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2605_13600_gb300.build.build() "
                              "(nvcc, sm_103a); there is no fallback implementation")
        lib = ct.CDLL(LIB_PATH)
        for name, (res, args) in PROTOS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(rc: int) -> None:
    if rc != SCOUP_OK:
        msg = load().scoup_last_error()
        raise ScoupError(rc, msg.decode() if msg else "")
