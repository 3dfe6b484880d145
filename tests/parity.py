"""Helpers shared by the GPU parity tests: the comparison rules of the CUDA
path against the float64 oracle.

Tolerances (stated by the method's float32 precision target):
  per pixel     |gpu - ref| <= 1e-4 |ref| + 1e-7 + bound, where bound is the
                oracle's first-order float32 error bound of that value (at most
                half of the first two terms except on the pixels the oracle
                flags as ill-conditioned); the id of the last blended
                Gaussian bit-exact.  At a pixel the oracle flags as
                branch-ambiguous, the GPU's values and last id must match
                the canonical branch or one of the oracle's alternatives.
  per gradient  |gpu - ref| <= 1e-3 max(|ref| + slack, 1e-3 max|ref|) + slack,
                elementwise over each gradient array, where slack is the
                oracle's bound of how far the alternatives at flagged pixels
                move that value (zero for a Gaussian that reaches no flagged
                pixel)
  block_mismatch  the normwise variant per Gaussian block (max over a
                Gaussian's entries of one parameter), used where the same sums
                are compared in two association orders
"""
from __future__ import annotations

import numpy as np
import torch

PIX_RTOL = 1e-4
PIX_ATOL = 1e-7
GRAD_RTOL = 1e-3


def pixel_mismatch(gpu: np.ndarray, ref: np.ndarray, mask: np.ndarray | None = None):
    """Boolean array of pixels outside the per-pixel tolerance (optionally
    restricted to `mask`)."""
    bad = np.abs(gpu - ref) > PIX_RTOL * np.abs(ref) + PIX_ATOL
    if mask is not None:
        bad &= mask
    return bad


def _within(gpu5: np.ndarray, ref5: np.ndarray, bound5: np.ndarray) -> np.ndarray:
    """(k,) rows of 5 values within the per-pixel tolerance."""
    return np.all(np.abs(gpu5 - ref5) <= PIX_RTOL * np.abs(ref5) + PIX_ATOL + bound5, axis=-1)


def check_forward(gpu_rgb, gpu_disp, gpu_T, gpu_last, ref: dict, last_map=None) -> dict:
    """Compare one window of the CUDA forward with the oracle's render_fwd
    result (computed with float32_bands).  No pixel is left out.

    gpu_rgb (3, h, w), gpu_disp, gpu_T (h, w) float; gpu_last (h, w): the id
    of the last blended Gaussian from the GPU's list (-1: none); last_map
    maps GPU ids to oracle ids (a view offset) if given.
    Returns counts: pixels, bad_value (outside tolerance at unflagged or
    conditioning-flagged pixels), bad_last (last id differs at an unflagged
    pixel), bad_branch (a flagged pixel matching neither the canonical branch
    nor an alternative), unresolved, matched_alt (flagged pixels that took an
    alternative), widened (pixels within the tolerance only once the
    oracle's float32 bound is added to it), and the fractions of the flag
    reasons."""
    from oracle import render as oren

    h, w = ref["T"].shape
    gv = np.stack([gpu_rgb[0], gpu_rgb[1], gpu_rgb[2], gpu_disp, gpu_T], -1).reshape(-1, 5).astype(np.float64)
    rv = np.stack([ref["rgb"][0], ref["rgb"][1], ref["rgb"][2], ref["disp"], ref["T"]], -1).reshape(-1, 5)
    bd = np.moveaxis(ref["bound"], 0, -1).reshape(-1, 5)
    gl = np.asarray(gpu_last).reshape(-1).astype(np.int64)
    if last_map is not None:
        gl = np.where(gl >= 0, last_map(gl), gl)
    rl = ref["last"].reshape(-1)
    fl = ref["flags"].reshape(-1)
    ok_val = _within(gv, rv, bd)
    plain = _within(gv, rv, np.zeros_like(bd))
    ok_last = gl == rl
    branch = (fl & oren.F_BRANCH) != 0
    unres = (fl & oren.F_UNRESOLVED) != 0
    strict = ~branch
    out = {"pixels": int(gv.shape[0]), "bad_value": int((strict & ~ok_val).sum()),
           "bad_last": int((strict & ~ok_last).sum()), "unresolved": int(unres.sum()),
           "widened": int((ok_val & ~plain).sum())}
    # flagged pixels: the canonical branch or one alternative
    alts = ref["alts"]
    bad_branch = 0
    matched_alt = 0
    for p in np.nonzero(branch & ~unres)[0]:
        if ok_val[p] and ok_last[p]:
            continue
        rows = np.nonzero(alts["pix"] == p)[0]
        good = _within(gv[p][None], alts["val"][rows], bd[p][None]) & (alts["last"][rows] == gl[p])
        if good.any():
            matched_alt += 1
        else:
            bad_branch += 1
    out["bad_branch"] = bad_branch
    out["matched_alt"] = matched_alt
    out["fractions"] = oren.flag_fractions(ref["flags"])
    out["first_bad"] = [int(p) for p in np.nonzero(strict & ~(ok_val & ok_last))[0][:5]]
    return out


def assert_forward(stats: dict, max_branch_frac: float = 1e-3, max_unresolved: int = 0):
    """The forward comparison passed: every pixel matched; the branch flags
    and unresolved pixels stay within the stated bounds."""
    assert stats["bad_value"] == 0 and stats["bad_last"] == 0 and stats["bad_branch"] == 0, stats
    assert stats["unresolved"] <= max_unresolved, stats
    assert stats["fractions"]["branch"] <= max_branch_frac, stats


def gpu_last_ids(plan, sizes, n: int) -> list:
    """Per view, the (H, W) ids (Gaussian index, -1: none) of the last splat
    the CUDA forward blended at each pixel: the tile list entry at
    n_contrib - 1 (n_contrib is the list position of the last blended splat
    + 1)."""
    from paper_2601_19489_gb300 import _lib as L

    nc = plan.view(L.GS_WS_N_CONTRIB, torch.int32)
    item = plan.view(L.GS_WS_INST_GID, torch.int32)
    ranges = plan.view(L.GS_WS_TILE_RANGES, torch.int32).reshape(-1, 2)
    out = []
    tile_off, pix_off = 0, 0
    for (w, h) in sizes:
        tx = (w + 15) // 16
        pix = torch.arange(w * h, device=nc.device)
        tile = tile_off + (pix // w // 16) * tx + (pix % w) // 16
        c = nc[pix_off: pix_off + w * h].long()
        pos = ranges[tile, 0].long() + c - 1
        last = torch.where(c > 0, item[pos.clamp(min=0)].long() % n, torch.full_like(c, -1))
        out.append(last.cpu().numpy().reshape(h, w))
        tile_off += tx * ((h + 15) // 16)
        pix_off += w * h
    return out


def format_stats(stats: dict) -> str:
    fr = stats["fractions"]
    return ("pixels %d: branch-flagged %.2e (cut %.1e, clamp %.1e, stop %.1e, depth %.1e), conditioning %.2e, "
            "unresolved %d, took an alternative %d, widened %d" % (
                stats["pixels"], fr["branch"], fr["cut"], fr["clamp"], fr["stop"], fr["depth"], fr["cond"],
                stats["unresolved"], stats["matched_alt"], stats["widened"]))


def grad_mismatch(gpu: np.ndarray, ref: np.ndarray, rtol: float = GRAD_RTOL, slack: np.ndarray | None = None):
    """Elements outside the per-gradient tolerance; slack (same shape) widens
    it where the oracle's alternatives at flagged pixels move the value."""
    scale = max(np.abs(ref).max(), 1e-30)
    if slack is None:
        tol = rtol * np.maximum(np.abs(ref), 1e-3 * scale)
    else:
        tol = rtol * np.maximum(np.abs(ref) + slack, 1e-3 * scale) + slack
    return np.abs(gpu - ref) > tol


def block_mismatch(gpu: np.ndarray, ref: np.ndarray, rtol: float = GRAD_RTOL, slack: np.ndarray | None = None):
    """Rows (one per Gaussian) whose normwise error exceeds the tolerance
    (widened by the row's largest slack where given)."""
    g = np.asarray(gpu, dtype=np.float64).reshape(gpu.shape[0], -1)
    r = np.asarray(ref, dtype=np.float64).reshape(ref.shape[0], -1)
    top = max(np.abs(r).max(), 1e-30)
    s = np.zeros(r.shape[0]) if slack is None else np.asarray(slack, dtype=np.float64).reshape(r.shape[0], -1).max(axis=1)
    scale = np.maximum(np.abs(r).max(axis=1) + s, 1e-3 * top)
    return np.abs(g - r).max(axis=1) > rtol * scale + s


def to_np(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy()


def view_image(flat: torch.Tensor, width: int, height: int, offset: int = 0, channels: int = 3):
    """(C, H, W) numpy image of view at pixel `offset` from a flat planar buffer."""
    n = width * height
    a = to_np(flat)[channels * offset: channels * offset + channels * n]
    return a.reshape(channels, height, width)


def cuda_available() -> bool:
    return torch.cuda.is_available()
