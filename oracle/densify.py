"""Oracle for the multi-view score-guided densification and pruning of
Sec. 3.2, float64 numpy on the CPU.

TEST INFRASTRUCTURE: only the test suite, the smoke check and the benchmark's
CPU-baseline leg may import this module.

Readings of the passage (the paper gives the scores, not every rule):
  e^j(u, v)  = E^j(u, v) / max_{u,v} E^j with E^j = sum_c |R^j_c - G^j_c|
               (Eq. 3: "normalize" read as division by the view's maximum);
  M^j(u, v)  = [e^j(u, v) > tau];
  s_i^+      = (1 / K) sum_j (number of pixels of view j with M^j = 1 that
               Gaussian i is blended into)  (Eq. 4: its sum carries no i; read
               as the sum over the pixels Gaussian i contributes to);
  E^j_photo  = the view's own (1 - lambda) L1 + lambda (1 - SSIM) (Eq. 5);
  s_i^-      = r_i / max_k r_k with r_i = sum_j (masked pixels of view j that
               Gaussian i is blended into) E^j_photo (Eq. 6);
  actions    = prune if s_i^- > tau_minus or its opacity < min_opacity
               (the 3DGS opacity cull); otherwise, if s_i^+ > tau_plus, clone
               when its largest scale is at most percent_dense * extent and
               split when larger (the 3DGS rules the method builds on);
               otherwise keep.  Pruning wins over densifying.
  clone      = the Gaussian and an exact copy.
  split      = two Gaussians at mean + R diag(s) z_k (z_k ~ N(0, I), k = 1, 2,
               passed in), scales s / 1.6, the parent's rotation, opacity and
               SH; the parent is removed.
Output order: the sources in index order, each replaced by its 0, 1 or 2
results; new Gaussians start with zero Adam moments, kept ones keep theirs.
"""
from __future__ import annotations

import numpy as np

from . import preprocess, render

KEEP, PRUNE, CLONE, SPLIT = 1, 0, 2, 3
SPLIT_SCALE = 1.6


def error_mask(rgb: np.ndarray, target: np.ndarray, tau: float) -> np.ndarray:
    """M^j for one view: rgb, target (3, h, w)."""
    E = np.abs(np.asarray(rgb, np.float64) - np.asarray(target, np.float64)).sum(axis=0)
    m = E.max()
    if m <= 0.0:
        return np.zeros(E.shape, dtype=bool)
    return E / m > tau


def view_scores(scene, cam, mask: np.ndarray, photo: float, s_plus: np.ndarray, r_minus: np.ndarray) -> None:
    """Add view j's terms of s^+ (unnormalised by K) and r^- to the arrays."""
    rec = preprocess.pack_for_render(preprocess.project(preprocess.params_from_scene(scene), cam,
                                                        scene.sh_degree))
    win = (0, 0, cam.width, cam.height)
    render.contrib_score(rec, win, mask.astype(np.float64), s_plus)
    render.contrib_score(rec, win, mask.astype(np.float64) * float(photo), r_minus)


def actions(scene, s_plus_sum: np.ndarray, r_minus: np.ndarray, K: int, tau_plus: float, tau_minus: float,
            min_opacity: float, percent_dense: float, extent: float) -> np.ndarray:
    s_plus = s_plus_sum / float(K)
    top = r_minus.max()
    s_minus = r_minus / top if top > 0.0 else np.zeros_like(r_minus)
    opacity = 1.0 / (1.0 + np.exp(-np.asarray(scene.opacity_logits, np.float64)))
    big = np.exp(np.asarray(scene.log_scales, np.float64)).max(axis=1) > percent_dense * extent
    act = np.full(s_plus.shape, KEEP, dtype=np.int32)
    grow = s_plus > tau_plus
    act[grow & ~big] = CLONE
    act[grow & big] = SPLIT
    act[(s_minus > tau_minus) | (opacity < min_opacity)] = PRUNE
    return act


def quat_rotation(q: np.ndarray) -> np.ndarray:
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    return np.stack([np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
                     np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
                     np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], -2)


def apply(arrays: dict, m: dict, v: dict, act: np.ndarray, normals: np.ndarray):
    """arrays / m / v: dicts of means, log_scales, quats, opacity_logits, sh
    (N rows each); normals (N, 2, 3), used by split rows only.  Returns the
    new (arrays, m, v)."""
    out = {k: [] for k in arrays}
    om = {k: [] for k in arrays}
    ov = {k: [] for k in arrays}
    R = quat_rotation(arrays["quats"])
    s = np.exp(np.asarray(arrays["log_scales"], np.float64))
    for i, a in enumerate(act):
        if a == PRUNE:
            continue
        if a in (KEEP, CLONE):
            for k in arrays:
                out[k].append(np.asarray(arrays[k][i], np.float64))
                om[k].append(np.asarray(m[k][i], np.float64))
                ov[k].append(np.asarray(v[k][i], np.float64))
            if a == CLONE:
                for k in arrays:
                    out[k].append(np.asarray(arrays[k][i], np.float64))
                    om[k].append(np.zeros_like(np.asarray(m[k][i], np.float64)))
                    ov[k].append(np.zeros_like(np.asarray(v[k][i], np.float64)))
            continue
        for c in range(2):  # split
            for k in arrays:
                if k == "means":
                    val = np.asarray(arrays[k][i], np.float64) + R[i] @ (s[i] * normals[i, c])
                elif k == "log_scales":
                    val = np.asarray(arrays[k][i], np.float64) - np.log(SPLIT_SCALE)
                else:
                    val = np.asarray(arrays[k][i], np.float64)
                out[k].append(val)
                om[k].append(np.zeros_like(val))
                ov[k].append(np.zeros_like(val))
    stack = lambda d, like: {k: (np.stack(d[k]) if d[k] else np.zeros((0,) + np.shape(like[k])[1:])) for k in d}
    return stack(out, arrays), stack(om, arrays), stack(ov, arrays)
