"""ctypes wrapper of the float64 per-pixel render oracle (render.c).

TEST INFRASTRUCTURE: only the test suite, the smoke check and the benchmark's
CPU-baseline leg may import this module.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "render.c")
_LIB = os.path.join(_HERE, "_build", "liboracle_render.so")
_lock = threading.Lock()
_lib = None

STRIDE = 12
G2D = 10


class Amb(ctypes.Structure):
    """Relative bands inside which a float32 evaluation may branch differently."""
    _fields_ = [("alpha_rel", ctypes.c_double), ("clamp_rel", ctypes.c_double),
                ("tstop_rel", ctypes.c_double), ("depth_rel", ctypes.c_double),
                ("pos_abs", ctypes.c_double), ("cond_eps", ctypes.c_double)]


# relative bands for alpha, clamp and stop; depth band (one float32 ulp, two
# sided); no position uncertainty and no conditioning flag (set both with
# float32_bands for an image)
DEFAULT_AMB = (2e-5, 2e-5, 2e-5, 2.4e-7, 0.0, 0.0)


def float32_bands(width: int, height: int, rel: float = 2e-5, ulps: float = 1.0,
                  cond_eps: float = 3e-6):
    """Bands for comparing with a float32 evaluation on a width x height image:
    the projected mean is uncertain by `ulps` float32 ulps of the largest
    pixel coordinate, and every alpha by a relative cond_eps."""
    import math

    top = max(int(width), int(height), 1)
    ulp = 2.0 ** (math.floor(math.log2(top)) - 23)
    return (rel, rel, rel, 2.4e-7, ulps * ulp, cond_eps)


def build(force: bool = False) -> str:
    """Compile render.c with gcc (-O2, OpenMP) into oracle/_build/."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.orc_render_fwd.restype = ctypes.c_int64
            lib.orc_render_fwd.argtypes = [ctypes.c_int64, P, P, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_int, P, P, P, P, P, P,
                                           ctypes.c_int]
            lib.orc_render_bwd.restype = None
            lib.orc_render_bwd.argtypes = [ctypes.c_int64, P, P, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_int, P, P, P, ctypes.c_int]
            lib.orc_contrib_score.restype = None
            lib.orc_contrib_score.argtypes = [ctypes.c_int64, P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int, P, P]
            assert lib.orc_stride() == STRIDE and lib.orc_g2d() == G2D
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def render_fwd(proj: np.ndarray, bg, window, amb=DEFAULT_AMB, n_threads: int = 0) -> dict:
    """Blend the window (x0, y0, x1, y1) of the image.

    proj: (N, 12) float64 records from ``preprocess.pack_for_render``.
    Returns rgb (3, h, w), disp (h, w), T (h, w), count (h, w) int32,
    amb (h, w) bool and the total number of candidate pairs."""
    lib = _load()
    proj = np.ascontiguousarray(proj, dtype=np.float64)
    x0, y0, x1, y1 = (int(v) for v in window)
    h, w = y1 - y0, x1 - x0
    bg = np.ascontiguousarray(np.asarray(bg, dtype=np.float64).reshape(3))
    rgb = np.zeros((3, h, w))
    disp = np.zeros((h, w))
    T = np.zeros((h, w))
    count = np.zeros((h, w), dtype=np.int32)
    flags = np.zeros((h, w), dtype=np.uint8)
    if amb is not None and len(amb) < 6:
        amb = tuple(amb) + (0.0,) * (6 - len(amb))
    a = Amb(*amb) if amb is not None else None
    total = lib.orc_render_fwd(proj.shape[0], _ptr(proj), _ptr(bg), x0, y0, x1, y1,
                               ctypes.cast(ctypes.pointer(a), ctypes.c_void_p) if a else None,
                               _ptr(rgb), _ptr(disp), _ptr(T), _ptr(count), _ptr(flags),
                               int(n_threads))
    return {"rgb": rgb, "disp": disp, "T": T, "count": count, "amb": flags.astype(bool),
            "pairs": int(total)}


def render_bwd(proj: np.ndarray, bg, window, g_rgb: np.ndarray, g_disp: np.ndarray,
               n_threads: int = 0) -> np.ndarray:
    """Per-Gaussian 2D gradients (N, 10) of sum(g_rgb * rgb) + sum(g_disp * disp)
    over the window; see render.c for the column order."""
    lib = _load()
    proj = np.ascontiguousarray(proj, dtype=np.float64)
    x0, y0, x1, y1 = (int(v) for v in window)
    bg = np.ascontiguousarray(np.asarray(bg, dtype=np.float64).reshape(3))
    g_rgb = np.ascontiguousarray(g_rgb, dtype=np.float64)
    g_disp = np.ascontiguousarray(g_disp, dtype=np.float64)
    assert g_rgb.shape == (3, y1 - y0, x1 - x0) and g_disp.shape == (y1 - y0, x1 - x0)
    out = np.zeros((proj.shape[0], G2D))
    lib.orc_render_bwd(proj.shape[0], _ptr(proj), _ptr(bg), x0, y0, x1, y1, _ptr(g_rgb),
                       _ptr(g_disp), _ptr(out), int(n_threads))
    return out


def contrib_score(proj: np.ndarray, window, weight: np.ndarray, out: np.ndarray | None = None) -> np.ndarray:
    """Add, for every pixel of the window and every Gaussian blended there,
    the pixel's weight (h, w) to that Gaussian's entry of the (N,) score."""
    lib = _load()
    proj = np.ascontiguousarray(proj, dtype=np.float64)
    x0, y0, x1, y1 = (int(v) for v in window)
    weight = np.ascontiguousarray(weight, dtype=np.float64)
    assert weight.shape == (y1 - y0, x1 - x0)
    if out is None:
        out = np.zeros(proj.shape[0])
    assert out.dtype == np.float64 and out.flags.c_contiguous and out.shape == (proj.shape[0],)
    lib.orc_contrib_score(proj.shape[0], _ptr(proj), x0, y0, x1, y1, _ptr(weight), _ptr(out))
    return out
