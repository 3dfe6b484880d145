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
    """Bands inside which a float32 evaluation may branch differently (see
    render.c: a fixed part plus a per-pair model of the float32 rounding)."""
    _fields_ = [("ln_abs", ctypes.c_double), ("tstop_abs", ctypes.c_double),
                ("depth_rel", ctypes.c_double), ("q_rel", ctypes.c_double),
                ("conic_rel", ctypes.c_double), ("kappa_rel", ctypes.c_double), ("pos_rel", ctypes.c_double),
                ("t_rel", ctypes.c_double), ("z_rel", ctypes.c_double)]


# flag bits of render_fwd's "flags" (render.c ORC_F_*)
F_CUT, F_CLAMP, F_STOP, F_DEPTH, F_COND, F_UNRESOLVED = 1, 2, 4, 8, 16, 32
F_BRANCH = F_CUT | F_CLAMP | F_STOP | F_DEPTH | F_UNRESOLVED
FLAG_NAMES = {F_CUT: "cut", F_CLAMP: "clamp", F_STOP: "stop", F_DEPTH: "depth", F_COND: "cond",
              F_UNRESOLVED: "unresolved"}

U32 = 2.0 ** -24  # unit roundoff of float32


def fixed_bands(ln: float, tstop: float, depth: float) -> tuple:
    """Fixed bands: |ln alpha - ln threshold| < ln, |ln T - ln 1e-4| < tstop,
    blended depths closer than depth (relative).  Used where a finite
    difference step, not float32 rounding, moves values across thresholds."""
    return (ln, tstop, depth, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0)


def float32_bands(ln_abs: float = 1.0e-6, q_rel: float = 5 * U32, conic_rel: float = 32 * U32,
                  kappa_rel: float = 24 * U32, pos_rel: float = 2 * U32, t_rel: float = 2 * U32,
                  z_rel: float = 1e-12) -> tuple:
    """The error model of a float32 evaluation of the blend (render.c
    orc_pair_eps), in units of the float32 unit roundoff u = 2^-24:
      ln_abs    the ex2 approximation (relative error about 2^-22), the
                float32 opacity and its log2 (measured within 4.3 u), and the
                rounding of their sum (|ln alpha| <= 6 at the cut);
      q_rel     5 u: the pair's quadratic form evaluated from float32 conic
                entries and tile-local offsets (about four roundings), per
                unit of |a| dx^2 + 2 |b dx dy| + |c| dy^2;
      conic_rel, kappa_rel
                32 u + 24 u kappa: the relative error of the preprocess's
                float32 conic in its worst direction, kappa the conic's
                condition number.  Over 77k Gaussians of five parity scenes
                the error measured against the float64 projection of the
                same float32 inputs stays below half of this (largest 59 u
                at kappa < 5, 401 u at kappa = 265);
      pos_rel   a tile-local projected mean rounded once (the compensated
                projection agrees with the float64 one to 1e-12 px);
      t_rel     the rounding of 1 - alpha and of T (1 - alpha) per splat;
      z_rel     the band around a float32 rounding midpoint of a compensated
                depth (its float-float value is within a few u^2 of exact)."""
    return (ln_abs, 0.0, 0.0, q_rel, conic_rel, kappa_rel, pos_rel, t_rel, z_rel)


def _amb(amb):
    if amb is None:
        return None
    amb = tuple(amb)
    if len(amb) == 4:  # (alpha band, clamp band, stop band, depth band)
        amb = fixed_bands(max(amb[0], amb[1]), amb[2], amb[3])
    return Amb(*amb)


DEFAULT_AMB = fixed_bands(2e-5, 2e-5, 2.4e-7)


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
            lib.orc_render_fwd2.restype = ctypes.c_int64
            lib.orc_render_fwd2.argtypes = [ctypes.c_int64, P, P, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_int, P, P, P, P, P, P, P, P,
                                            ctypes.c_int64, P, P, P, P, ctypes.c_int]
            lib.orc_render_bwd2.restype = None
            lib.orc_render_bwd2.argtypes = [ctypes.c_int64, P, P, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_int, P, P, P, P, P, P, ctypes.c_int]
            lib.orc_contrib_score.restype = None
            lib.orc_contrib_score.argtypes = [ctypes.c_int64, P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int, P, P]
            assert lib.orc_stride() == STRIDE and lib.orc_g2d() == G2D
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _ref(a):
    return ctypes.cast(ctypes.pointer(a), ctypes.c_void_p) if a is not None else None


def render_fwd(proj: np.ndarray, bg, window, amb=DEFAULT_AMB, n_threads: int = 0,
               alternatives: bool = True) -> dict:
    """Blend the window (x0, y0, x1, y1) of the image.

    proj: (N, 12) float64 records from ``preprocess.pack_for_render``.
    Returns rgb (3, h, w), disp (h, w), T (h, w), count (h, w) int32 (splats
    blended), last (h, w) int64 (id of the last blended Gaussian, -1: none),
    flags (h, w) uint8 (F_* bits), amb (h, w) bool (a branch flag: cut,
    clamp, stop, depth or unresolved), cond (h, w) bool, bound (5, h, w) (the
    first-order float32 error bounds of r, g, b, disp, T), alts (the
    alternatives of the flagged pixels: pix (k,) pixel index in the window,
    val (k, 5), last (k,)) and the total number of candidate pairs."""
    lib = _load()
    proj = np.ascontiguousarray(proj, dtype=np.float64)
    x0, y0, x1, y1 = (int(v) for v in window)
    h, w = y1 - y0, x1 - x0
    bg = np.ascontiguousarray(np.asarray(bg, dtype=np.float64).reshape(3))
    rgb = np.zeros((3, h, w))
    disp = np.zeros((h, w))
    T = np.zeros((h, w))
    count = np.zeros((h, w), dtype=np.int32)
    last = np.zeros((h, w), dtype=np.int64)
    flags = np.zeros((h, w), dtype=np.uint8)
    bound = np.zeros((5, h, w))
    a = _amb(amb)
    cap = max(64, h * w // 4) if (a is not None and alternatives) else 0
    while True:
        alt_pix = np.zeros(max(cap, 1), dtype=np.int64)
        alt_val = np.zeros((max(cap, 1), 5))
        alt_last = np.zeros(max(cap, 1), dtype=np.int64)
        n_alt = ctypes.c_int64(0)
        total = lib.orc_render_fwd2(proj.shape[0], _ptr(proj), _ptr(bg), x0, y0, x1, y1, _ref(a),
                                    _ptr(rgb), _ptr(disp), _ptr(T), _ptr(count), _ptr(last), _ptr(flags),
                                    _ptr(bound), cap if alternatives else -1, _ptr(alt_pix), _ptr(alt_val),
                                    _ptr(alt_last), ctypes.cast(ctypes.pointer(n_alt), ctypes.c_void_p),
                                    int(n_threads))
        if not alternatives or n_alt.value <= cap:
            break
        cap = int(n_alt.value)
    k = int(n_alt.value) if alternatives else 0
    order = np.argsort(alt_pix[:k], kind="stable")
    alts = {"pix": alt_pix[:k][order], "val": alt_val[:k][order], "last": alt_last[:k][order]}
    return {"rgb": rgb, "disp": disp, "T": T, "count": count, "last": last, "flags": flags,
            "amb": (flags & F_BRANCH) != 0, "cond": (flags & F_COND) != 0, "bound": bound,
            "alts": alts, "pairs": int(total)}


def flag_fractions(flags: np.ndarray) -> dict:
    """Fraction of pixels carrying each flag, the branch flags together, and
    the unresolved ones."""
    f = np.asarray(flags)
    n = max(f.size, 1)
    out = {name: float(((f & bit) != 0).sum()) / n for bit, name in FLAG_NAMES.items()}
    out["branch"] = float(((f & F_BRANCH) != 0).sum()) / n
    return out


def render_bwd(proj: np.ndarray, bg, window, g_rgb: np.ndarray, g_disp: np.ndarray,
               n_threads: int = 0, amb=None, with_slack: bool = False, with_mag: bool = False):
    """Per-Gaussian 2D gradients (N, 10) of sum(g_rgb * rgb) + sum(g_disp * disp)
    over the window; see render.c for the column order.  Every pixel takes the
    canonical branch.  With amb and with_slack, also returns the slack
    (N, 10): for every Gaussian, the sum over the flagged pixels of the
    largest change of its values over the pixel's alternatives (+inf for a
    candidate of an unresolved pixel); returns (grad, slack) then.  With
    with_mag, also returns the magnitudes (N, 10) of the summed terms (each
    factor of each pixel's term by its absolute value, the colour behind a
    splat by the pixel's absolute composited colour): the scale of the
    float32 error of an order-free sum of those terms; returns
    (grad, slack, mag) then (slack None without with_slack)."""
    lib = _load()
    proj = np.ascontiguousarray(proj, dtype=np.float64)
    x0, y0, x1, y1 = (int(v) for v in window)
    bg = np.ascontiguousarray(np.asarray(bg, dtype=np.float64).reshape(3))
    g_rgb = np.ascontiguousarray(g_rgb, dtype=np.float64)
    g_disp = np.ascontiguousarray(g_disp, dtype=np.float64)
    assert g_rgb.shape == (3, y1 - y0, x1 - x0) and g_disp.shape == (y1 - y0, x1 - x0)
    out = np.zeros((proj.shape[0], G2D))
    slack = np.zeros((proj.shape[0], G2D)) if with_slack else None
    mag = np.zeros((proj.shape[0], G2D)) if with_mag else None
    a = _amb(amb) if with_slack else None
    lib.orc_render_bwd2(proj.shape[0], _ptr(proj), _ptr(bg), x0, y0, x1, y1, _ptr(g_rgb),
                        _ptr(g_disp), _ref(a), _ptr(out), _ptr(slack), _ptr(mag), int(n_threads))
    if with_mag:
        return out, slack, mag
    return (out, slack) if with_slack else out


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
