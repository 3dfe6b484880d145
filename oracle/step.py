"""One whole training step of the oracle: preprocess -> blend -> loss ->
per-pixel backward -> preprocess backward -> Adam, all float64 on the CPU.

TEST INFRASTRUCTURE: only the test suite, the smoke check and the benchmark's
CPU-baseline leg may import this module.

Learning rates follow the 3DGS defaults the paper trains with (Sec. 4 builds
on 3DGS; the paper itself names no optimiser settings): means 1.6e-4 x scene
extent, SH DC 2.5e-3, higher SH 2.5e-3 / 20, opacity 0.05, log-scales 5e-3,
quaternions 1e-3, Adam betas (0.9, 0.999), eps 1e-15.
"""
from __future__ import annotations

import time

import numpy as np

from . import adam, loss, preprocess, render

GROUPS = ("means", "log_scales", "quats", "opacity_logits", "sh_dc", "sh_rest")


def default_lrs(extent: float = 1.0) -> dict:
    return {"means": 1.6e-4 * extent, "log_scales": 5e-3, "quats": 1e-3,
            "opacity_logits": 0.05, "sh_dc": 2.5e-3, "sh_rest": 2.5e-3 / 20.0}


def _split(grads: dict) -> dict:
    out = {k: grads[k] for k in ("means", "log_scales", "quats", "opacity_logits")}
    out["sh_dc"] = grads["sh"][:, :1]
    out["sh_rest"] = grads["sh"][:, 1:]
    return out


def new_state(scene) -> dict:
    p = {"means": scene.means, "log_scales": scene.log_scales, "quats": scene.quats,
         "opacity_logits": scene.opacity_logits, "sh_dc": scene.sh[:, :1], "sh_rest": scene.sh[:, 1:]}
    return {"step": 0,
            "params": {k: np.asarray(v, dtype=np.float64).copy() for k, v in p.items()},
            "m": {k: np.zeros(np.shape(v)) for k, v in p.items()},
            "v": {k: np.zeros(np.shape(v)) for k, v in p.items()}}


def scene_from_state(state, template):
    from synth import Scene

    p = state["params"]
    sh = np.concatenate([p["sh_dc"], p["sh_rest"]], axis=1)
    # Kept in float64: the oracle carries its state at full precision.
    return Scene(p["means"], p["log_scales"], p["quats"], p["opacity_logits"], sh,
                 template.sh_degree)


def forward_backward(scene, cam, target, bg=(0.0, 0.0, 0.0), lam: float = 0.2,
                     window=None, n_threads: int = 0, disp_target=None, disp_weight: float = 0.0,
                     timings: dict | None = None):
    """Loss and parameter gradients (float64) of one view."""
    t0 = time.perf_counter()
    params = preprocess.params_from_scene(scene)
    pr = preprocess.project(params, cam, scene.sh_degree)
    rec = preprocess.pack_for_render(pr)
    t1 = time.perf_counter()
    win = window if window is not None else (0, 0, cam.width, cam.height)
    x0, y0, x1, y1 = win
    f = render.render_fwd(rec, bg, win, amb=None, n_threads=n_threads)
    tgt = np.asarray(target, dtype=np.float64)[:, y0:y1, x0:x1]
    L, g_rgb = loss.photometric(f["rgb"], tgt, lam)
    g_disp = np.zeros_like(f["disp"])
    if disp_target is not None and disp_weight != 0.0:
        Ld, g_disp = loss.disparity_l1(f["disp"], np.asarray(disp_target)[y0:y1, x0:x1], disp_weight)
        L += Ld
    t2 = time.perf_counter()
    g2d = render.render_bwd(rec, bg, win, g_rgb, g_disp, n_threads=n_threads)
    t3 = time.perf_counter()
    grads = preprocess.preprocess_backward(scene, cam, g2d)
    f["grad2d"] = g2d
    t4 = time.perf_counter()
    if timings is not None:
        timings.update(preprocess=t1 - t0, render_fwd_loss=t2 - t1, render_bwd=t3 - t2,
                       preprocess_bwd=t4 - t3)
    return L, grads, f


def forward_backward_batch(scene, cams, targets, bg=(0.0, 0.0, 0.0), lam: float = 0.2,
                           disp_targets=None, disp_weight: float = 0.0, n_threads: int = 0):
    """Loss and parameter gradients of a batch of views (the paper says
    nothing about batching views, so it gives no weighting).  Reading: the
    batch loss is the mean over all the batch's pixels, i.e. each view's own
    loss weighted by its share of the pixels,
        L = sum_v (P_v / P) L_v,   P = sum_v P_v,
    so that views of equal size enter equally and the gradients of the views
    add up before one optimiser update."""
    P = float(sum(c.width * c.height for c in cams))
    total, acc = 0.0, None
    for i, cam in enumerate(cams):
        w = cam.width * cam.height / P
        dt = disp_targets[i] if disp_targets is not None else None
        L, g, _ = forward_backward(scene, cam, targets[i], bg=bg, lam=lam, n_threads=n_threads,
                                   disp_target=dt, disp_weight=disp_weight)
        total += w * L
        acc = {k: w * v for k, v in g.items()} if acc is None else {k: acc[k] + w * g[k] for k in acc}
    return total, acc


def adam_update(state: dict, grads: dict, lrs: dict) -> None:
    state["step"] += 1
    g = _split(grads)
    for k in GROUPS:
        p, m, v = adam.adam_step(state["params"][k], g[k], state["m"][k], state["v"][k],
                                 state["step"], lrs[k])
        state["params"][k], state["m"][k], state["v"][k] = p, m, v


def train_step(state: dict, template, cam, target, lrs: dict, **kw):
    scene = scene_from_state(state, template)
    L, grads, f = forward_backward(scene, cam, target, **kw)
    t0 = time.perf_counter()
    adam_update(state, grads, lrs)
    if kw.get("timings") is not None:
        kw["timings"]["adam"] = time.perf_counter() - t0
    return L, grads, f
