"""Oracle for tile binning and sorting, float64 numpy.

TEST INFRASTRUCTURE: only the test suite, the smoke check and the benchmark's
CPU-baseline leg may import this module.

Paper passages: Sec. 2.1, Eq. 1 (the ellipse a x^2 + 2 b x y + c y^2 = t with
t = 2 ln(255 o)) and the per-column tile test that follows Eq. 2.  A tile is
touched when the ellipse's closed interior meets the tile.  The tile is taken
as the rectangle spanned by its pixel centres (pixel (i, j) has its centre at
(i + 0.5, j + 0.5)), clipped to the image; a pixel whose centre lies outside
every touched tile has alpha < 1/255 and is skipped by the blend anyway, so the
rendered result does not depend on the choice of rectangle beyond containing
the pixel centres.

The definition used here is brute force: the minimum of the convex quadratic
form over the rectangle (zero if the mean is inside, else the smallest of the
four edge minima, each a clamped 1-D vertex) compared with t.
"""
from __future__ import annotations

import numpy as np


def _edge_min(a, b, c, ux0, ux1, uy):
    """min over u in [ux0, ux1] of a u^2 + 2 b u v + c v^2 at v = uy."""
    with np.errstate(divide="ignore", invalid="ignore"):
        u_star = np.where(a > 0, -b * uy / a, ux0)
    u = np.clip(u_star, ux0, ux1)
    return a * u * u + 2.0 * b * u * uy + c * uy * uy


def min_q_rect(mx, my, a, b, c, x0, x1, y0, y1):
    """Minimum of q(x, y) = a dx^2 + 2 b dx dy + c dy^2, d = (x - mx, y - my),
    over the rectangle [x0, x1] x [y0, y1] (arrays broadcast)."""
    dx0, dx1 = x0 - mx, x1 - mx
    dy0, dy1 = y0 - my, y1 - my
    inside = (dx0 <= 0) & (dx1 >= 0) & (dy0 <= 0) & (dy1 >= 0)
    m = np.minimum.reduce([
        _edge_min(a, b, c, dx0, dx1, dy0),
        _edge_min(a, b, c, dx0, dx1, dy1),
        _edge_min(c, b, a, dy0, dy1, dx0),
        _edge_min(c, b, a, dy0, dy1, dx1),
    ])
    return np.where(inside, 0.0, m)


def tile_rects(width: int, height: int, tile: int = 16):
    """Pixel-centre rectangles of all tiles, row-major tile order."""
    tw = (width + tile - 1) // tile
    th = (height + tile - 1) // tile
    tx, ty = np.meshgrid(np.arange(tw), np.arange(th))
    tx = tx.ravel()
    ty = ty.ravel()
    x0 = tx * tile + 0.5
    x1 = np.minimum(tx * tile + tile - 1, width - 1) + 0.5
    y0 = ty * tile + 0.5
    y1 = np.minimum(ty * tile + tile - 1, height - 1) + 0.5
    return tw, th, x0, x1, y0, y1


def tile_min_q(proj: np.ndarray, width: int, height: int, tile: int = 16, reach: float = 2.0):
    """For every valid Gaussian with t > 0, the min of q over each tile whose
    rectangle lies within ``reach`` x its level-set box.

    proj: (N, 12) render records.  Returns a dict gid -> (tile ids, min_q,
    level t)."""
    tw, th, x0, x1, y0, y1 = tile_rects(width, height, tile)
    out = {}
    for gid in range(proj.shape[0]):
        mx, my, a, b, c, o = proj[gid, 0:6]
        t = proj[gid, 10]
        if proj[gid, 11] == 0 or not t > 0:
            continue
        det = a * c - b * b
        rx = reach * np.sqrt(t * c / det) + tile
        ry = reach * np.sqrt(t * a / det) + tile
        sel = (x1 >= mx - rx) & (x0 <= mx + rx) & (y1 >= my - ry) & (y0 <= my + ry)
        ids = np.nonzero(sel)[0]
        if ids.size == 0:
            continue
        mq = min_q_rect(mx, my, a, b, c, x0[ids], x1[ids], y0[ids], y1[ids])
        out[gid] = (ids, mq, t)
    return out


def stable_sort_pairs(keys: np.ndarray, values: np.ndarray):
    """Keys ascending, equal keys in input order; values follow."""
    order = np.argsort(keys, kind="stable")
    return keys[order], values[order]
