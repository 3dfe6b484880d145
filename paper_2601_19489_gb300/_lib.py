"""ctypes binding of libgs.so (include/gs.h).

Argument marshalling only: every function here forwards to the C entry point
of the same name.  The library is loaded from this package directory; if it
is missing it is built with nvcc, and if that is impossible the import fails
loudly — there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgs.so")

GS_MAX_VIEWS = 16
GS_NG_FEAT = 32
GS_NG_HIDDEN = 32
GS_NG_CHILDREN = 10
GS_TILE = 16
GS_BUCKET = 32

GS_OK, GS_ERR_ARG, GS_ERR_CAPACITY, GS_ERR_CUDA, GS_ERR_TIMEOUT, GS_ERR_INTERNAL = 0, -1, -2, -3, -4, -5

(GS_WS_RECORDS, GS_WS_TILES_TOUCHED, GS_WS_RECTS, GS_WS_DEPTH_ORDER, GS_WS_INST_TILE,
 GS_WS_INST_GID, GS_WS_TILE_RANGES, GS_WS_N_CONTRIB, GS_WS_GRAD2D, GS_WS_STATUS, GS_WS_BIN) = range(11)

EXPORTS = (
    "gs_plan_create", "gs_plan_create_tuned", "gs_plan_destroy", "gs_plan_workspace_bytes", "gs_plan_pixels",
    "gs_workspace_view", "gs_read_status", "gs_error_string", "gs_preprocess", "gs_bin_sort",
    "gs_render_fwd", "gs_render_bwd", "gs_render_bwd_blend", "gs_preprocess_bwd",
    "gs_loss_scratch_floats", "gs_loss", "gs_adam_step",
    "gs_adam_step_multi", "gs_adam_step_multi_dev", "gs_preprocess_bwd_adam", "gs_sort_scratch_bytes",
    "gs_sort_pairs_u32", "gs_sort_pairs_u32_noalloc",
    "gs_ng_workspace_bytes", "gs_ng_decode_fwd", "gs_ng_decode_preprocess", "gs_ng_decode_bwd",
    "gs_ng_read_status", "gs_ng_wait_probe",
    "gs_densify_scratch_bytes", "gs_densify_score", "gs_densify_plan", "gs_densify_apply",
    "gs_pose_init", "gs_plan_set_pose", "gs_pose_step",
)

GS_DENSIFY_PRUNE, GS_DENSIFY_KEEP, GS_DENSIFY_CLONE, GS_DENSIFY_SPLIT = 0, 1, 2, 3

GS_POSE_SLOTS = 256
GS_POSE_STATE_DOUBLES = 32 + 8 * GS_POSE_SLOTS


class GsCamera(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float),
                ("cy", ctypes.c_float), ("w2c", ctypes.c_float * 12), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("near_z", ctypes.c_float)]


class GsParams(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("sh_degree", ctypes.c_int32),
                ("means", ctypes.c_void_p), ("log_scales", ctypes.c_void_p),
                ("quats", ctypes.c_void_p), ("opacity_logits", ctypes.c_void_p),
                ("sh", ctypes.c_void_p)]


class GsTuning(ctypes.Structure):
    _fields_ = [("bucket", ctypes.c_int32), ("bwd_warps", ctypes.c_int32), ("bwd_chains", ctypes.c_int32),
                ("bbox_3sigma", ctypes.c_int32), ("bwd_per_pixel", ctypes.c_int32), ("bin_radix", ctypes.c_int32),
                ("fwd_pixels", ctypes.c_int32)]


class GsAdamHparams(ctypes.Structure):
    _fields_ = [("lr_means", ctypes.c_float), ("lr_log_scales", ctypes.c_float), ("lr_quats", ctypes.c_float),
                ("lr_opacity", ctypes.c_float), ("lr_sh_dc", ctypes.c_float), ("lr_sh_rest", ctypes.c_float),
                ("b1", ctypes.c_float), ("b2", ctypes.c_float), ("eps", ctypes.c_float),
                ("visible_only", ctypes.c_int32)]


class GsDensifyRules(ctypes.Structure):
    _fields_ = [("tau_plus", ctypes.c_float), ("tau_minus", ctypes.c_float), ("min_opacity", ctypes.c_float),
                ("percent_dense", ctypes.c_float), ("extent", ctypes.c_float), ("k_views", ctypes.c_int32)]


class GsPoseHparams(ctypes.Structure):
    _fields_ = [("lr_rot", ctypes.c_double), ("lr_trans", ctypes.c_double), ("b1", ctypes.c_double),
                ("b2", ctypes.c_double), ("eps", ctypes.c_double)]


class GsStatus(ctypes.Structure):
    _fields_ = [("n_instances", ctypes.c_int64), ("n_buckets", ctypes.c_int64),
                ("inst_capacity", ctypes.c_int64), ("overflow", ctypes.c_int32),
                ("error", ctypes.c_int32)]


class GsAdamGroup(ctypes.Structure):
    _fields_ = [("p", ctypes.c_void_p), ("g", ctypes.c_void_p), ("m", ctypes.c_void_p),
                ("v", ctypes.c_void_p), ("n", ctypes.c_int64), ("lr", ctypes.c_float),
                ("period", ctypes.c_int64), ("head", ctypes.c_int64), ("lr_head", ctypes.c_float)]


class GsNgParams(ctypes.Structure):
    _fields_ = [("n_anchors", ctypes.c_int64), ("anchor_xyz", ctypes.c_void_p), ("feat", ctypes.c_void_p),
                ("anchor_ls", ctypes.c_void_p), ("w1", ctypes.c_void_p), ("b1", ctypes.c_void_p),
                ("w2", ctypes.c_void_p), ("b2", ctypes.c_void_p)]


class GsError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = _lib.gs_error_string(code).decode() if _lib is not None else str(code)
        super().__init__(f"{where}: {msg} ({code})")


_lib = None
_lock = threading.Lock()

P = ctypes.c_void_p
_SIGS = {
    "gs_plan_create": (P, [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, P, P, ctypes.c_int64]),
    "gs_plan_create_tuned": (P, [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, P, P, ctypes.c_int64,
                                 ctypes.POINTER(GsTuning)]),
    "gs_plan_destroy": (None, [P]),
    "gs_plan_workspace_bytes": (ctypes.c_size_t, [P]),
    "gs_plan_pixels": (ctypes.c_int64, [P]),
    "gs_workspace_view": (ctypes.c_int, [P, P, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p),
                                         ctypes.POINTER(ctypes.c_size_t)]),
    "gs_read_status": (ctypes.c_int, [P, P, ctypes.POINTER(GsStatus), P]),
    "gs_error_string": (ctypes.c_char_p, [ctypes.c_int]),
    "gs_preprocess": (ctypes.c_int, [P, P, ctypes.POINTER(GsParams), P, P]),
    "gs_bin_sort": (ctypes.c_int, [P, P, ctypes.c_int, P]),
    "gs_render_fwd": (ctypes.c_int, [P, P, P, P, P, P, P]),
    "gs_render_bwd": (ctypes.c_int, [P, P, ctypes.POINTER(GsParams), P, P, P, P, P, P,
                                     ctypes.POINTER(GsParams), P]),
    "gs_render_bwd_blend": (ctypes.c_int, [P, P, P, P, P, P, P]),
    "gs_preprocess_bwd": (ctypes.c_int, [P, P, ctypes.POINTER(GsParams), P, ctypes.POINTER(GsParams), P]),
    "gs_loss_scratch_floats": (ctypes.c_int64, [P]),
    "gs_loss": (ctypes.c_int, [P, P, P, ctypes.c_float, P, P, ctypes.c_float, P, P, P, P, P]),
    "gs_adam_step": (ctypes.c_int, [P, P, P, P, ctypes.c_int64, ctypes.c_float, ctypes.c_float,
                                    ctypes.c_float, ctypes.c_float, ctypes.c_int32, P]),
    "gs_adam_step_multi": (ctypes.c_int, [ctypes.POINTER(GsAdamGroup), ctypes.c_int32, ctypes.c_float,
                                          ctypes.c_float, ctypes.c_float, ctypes.c_int32, P]),
    "gs_adam_step_multi_dev": (ctypes.c_int, [ctypes.POINTER(GsAdamGroup), ctypes.c_int32, ctypes.c_float,
                                              ctypes.c_float, ctypes.c_float, P, P]),
    "gs_preprocess_bwd_adam": (ctypes.c_int, [P, P, ctypes.POINTER(GsParams), P, ctypes.POINTER(GsParams),
                                              ctypes.POINTER(GsParams), ctypes.POINTER(GsAdamHparams), P, P]),
    "gs_densify_scratch_bytes": (ctypes.c_size_t, [ctypes.c_int64]),
    "gs_densify_score": (ctypes.c_int, [P, P, P, P, ctypes.c_float, P, P, P, P, P]),
    "gs_densify_plan": (ctypes.c_int, [ctypes.c_int64, ctypes.POINTER(GsParams), P, P,
                                       ctypes.POINTER(GsDensifyRules), P, P, P, ctypes.POINTER(ctypes.c_int64), P]),
    "gs_densify_apply": (ctypes.c_int, [ctypes.c_int64, ctypes.POINTER(GsParams), ctypes.POINTER(GsParams),
                                        ctypes.POINTER(GsParams), P, P, P, ctypes.POINTER(GsParams),
                                        ctypes.POINTER(GsParams), ctypes.POINTER(GsParams), P]),
    "gs_sort_scratch_bytes": (ctypes.c_size_t, [ctypes.c_int64]),
    "gs_sort_pairs_u32": (ctypes.c_int, [P, P, P, P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                         P, P]),
    "gs_sort_pairs_u32_noalloc": (ctypes.c_int, [P, P, P, P, ctypes.c_int64, ctypes.c_int32,
                                                 ctypes.c_int32, P]),
    "gs_ng_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int64]),
    "gs_ng_decode_fwd": (ctypes.c_int, [ctypes.POINTER(GsNgParams), P, ctypes.POINTER(GsParams), P, P]),
    "gs_ng_decode_preprocess": (ctypes.c_int, [ctypes.POINTER(GsNgParams), P, ctypes.POINTER(GsParams), P, P, P,
                                               P]),
    "gs_ng_decode_bwd": (ctypes.c_int, [ctypes.POINTER(GsNgParams), P, ctypes.POINTER(GsParams), ctypes.c_int32,
                                         ctypes.POINTER(GsNgParams), P, P]),
    "gs_ng_read_status": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int32), P]),
    "gs_ng_wait_probe": (ctypes.c_int, [P, ctypes.c_int64, ctypes.c_int32, P]),
    "gs_pose_init": (ctypes.c_int, [P, P]),
    "gs_plan_set_pose": (ctypes.c_int, [P, P]),
    "gs_pose_step": (ctypes.c_int, [P, ctypes.POINTER(GsPoseHparams), P]),
}


def load(build_if_missing: bool = True):
    """Load libgs.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing:
                from . import build as _build

                try:
                    _build.build()
                except RuntimeError:
                    if not os.path.exists(LIB_PATH):
                        raise
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"libgs.so not found at {LIB_PATH}; run paper_2601_19489_gb300.build")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def lib():
    return _lib if _lib is not None else load()


def check(rc: int, where: str) -> None:
    if rc != GS_OK:
        raise GsError(rc, where)
