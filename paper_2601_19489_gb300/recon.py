"""Timed reconstruction: train from a sparse start against a set of posed
views for a wall-clock budget and follow the held-out PSNR (the 1-minute
reconstruction setting of the paper's Sec. 4).

Ways to spend the budget, all on one schedule:
  plain          one view per step, eager launches;
  densify        plain, plus a multi-view score-guided densify-and-prune
                 stage (Sec. 3.2) after each of the first half of the
                 evaluation segments (K = 10 random training views; its time
                 counts as training time);
  batched_graph  8 views per step through the batched plan, launch shapes from
                 the autotuner, every step replayed from a CUDA graph; every
                 learning rate scaled by batch_lr_scale (default sqrt(8)):
                 a batch of 8 takes 8x fewer Adam steps, each of which moves
                 a parameter by about its rate whatever the gradient's scale,
                 while the batch's averaged gradient is less noisy, so the
                 rate grows with the square root of the batch (the usual
                 rule for Adam); with batch_betas "scaled" (the default)
                 Adam's betas become beta^8, so the moments forget at the
                 same rate per view as with one view per step (the rule of
                 Grendel, Zhao et al. 2024, for batched 3DGS); "fixed" keeps
                 (0.9, 0.999); the decay schedule is unchanged;
  ng             one view per step of the neural-Gaussian model (Sec. 2.3):
                 anchors at the starting points, 10 decoded children each;
  ng_frozen      the same anchors and children with the decoder's MLP kept at
                 its initialisation (features and anchor scales still
                 train): what the trained network adds;
  pose           plain, plus the global pose refinement of Sec. 2.5 (one
                 camera-side correction for all views, updated every 300
                 steps, applied to the held-out views too).
The schedule is piecewise constant over the evaluation segments: the mean
positions' learning rate decays exponentially from lr0 to lr0 / 100 (the
3DGS schedule), the pose rates the same way, and the disparity weight
linearly to zero (Sec. 3.1).
Evaluation time is not counted in the budget.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from .api import Gaussians, NgParams
from .autotune import TUNED, autotune
from .trainer import NgTrainer, Trainer, default_lrs, default_pose


def psnr(img: torch.Tensor, ref: torch.Tensor) -> float:
    """PSNR of a rendered image (clamped to [0, 1]) against a reference."""
    mse = torch.mean((img.clamp(0.0, 1.0) - ref) ** 2).item()
    return float("inf") if mse == 0.0 else 10.0 * math.log10(1.0 / mse)


def render_views(trainer: Trainer, cams) -> list:
    """(colour, disparity) of each view through trainer.forward, as copies."""
    out = []
    for c in cams:
        sl = trainer.forward([c])
        out.append((sl.rgb.clone(), sl.disp.clone()))
    return out


def eval_psnr(trainer: Trainer, cams, refs) -> float:
    vals = []
    for c, ref in zip(cams, refs):
        sl = trainer.forward([c])
        vals.append(psnr(sl.rgb, ref))
    return float(np.mean(vals))


def _ng_start(init, seed: int) -> dict:
    """Anchors at the starting points, anchor scales from their spacing."""
    from scipy.spatial import cKDTree

    import synth

    d = synth.ng_anchors(np.asarray(init.means), init.n, seed=seed)
    dist, _ = cKDTree(d["anchor_xyz"].astype(np.float64)).query(d["anchor_xyz"].astype(np.float64), k=4)
    s = np.log(np.maximum(dist[:, 1:].mean(axis=1), 1e-4)).astype(np.float32)
    d["anchor_ls"][:, 0:3] = s[:, None]
    d["anchor_ls"][:, 3:6] = s[:, None]
    return d


def reconstruct(method: str, init, train_cams, train_rgb, train_disp, eval_cams, eval_rgb, *,
                budget_s: float = 60.0, eval_every_s: float = 5.0, lam: float = 0.2, disp_weight: float = 0.1,
                extent: float = 4.4, batch: int = 8, seed: int = 0, densify_rules: dict | None = None,
                densify_tau: float = 0.3, densify_k: int = 10, max_gaussians: int | None = None,
                pose: dict | None = None, batch_lr_scale: float | None = None, batch_betas: str = "scaled",
                ng_lrs: dict | None = None, device="cuda") -> dict:
    """Run one method for budget_s seconds of training; returns its held-out
    PSNR curve [(seconds trained, PSNR)], steps and views trained.
    pose: settings of the `pose` method (default_pose(extent) by default).
    ng_lrs: decoder learning rates of the ng methods (default_ng_lrs()
    overridden by name)."""
    W, H = train_cams[0].width, train_cams[0].height
    lrs = default_lrs(extent)
    if method == "batched_graph":
        scale = math.sqrt(batch) if batch_lr_scale is None else float(batch_lr_scale)
        lrs = {k: v * scale for k, v in lrs.items()}
    lr0 = lrs["means"]
    rng = np.random.default_rng(seed)
    nv = len(train_cams)
    if method in ("ng", "ng_frozen"):
        tr = NgTrainer(NgParams.from_dict(_ng_start(init, seed), device=device), W, H, lam=lam,
                       disp_weight=disp_weight, lrs=lrs,
                       ng_lrs={**(ng_lrs or {}), "mlp": 0.0} if method == "ng_frozen" else ng_lrs, device=device)
    else:
        params = Gaussians.from_scene(init, device=device)
        tuning, lb = None, True
        if method == "batched_graph":
            batches = [[(batch * b + i) % nv for i in range(batch)] for b in range(-(-nv // batch))]
            b_rgb = [torch.cat([train_rgb[i] for i in ix]) for ix in batches]
            b_disp = [torch.cat([train_disp[i] for i in ix]) for ix in batches]
            b_cams = [[train_cams[i] for i in ix] for ix in batches]
            best, _ = autotune(params, b_cams[:2], b_rgb[:2], lam=lam, device=device)
            tuning = {k: best[k] for k in TUNED}
            lb = best["load_balanced"]
        elif method not in ("plain", "densify", "pose"):
            raise ValueError(method)
        pose_cfg = {**default_pose(extent), **(pose or {})} if method == "pose" else None
        betas = (0.9, 0.999)
        if method == "batched_graph" and batch_betas == "scaled":
            betas = (0.9 ** batch, 0.999 ** batch)
        elif batch_betas not in ("scaled", "fixed"):
            raise ValueError(batch_betas)
        tr = Trainer(params, W, H, lam=lam, disp_weight=disp_weight, lrs=lrs, load_balanced=lb, tuning=tuning,
                     pose=pose_cfg, betas=betas, device=device)
    views = b_cams if method == "batched_graph" else [[c] for c in train_cams]
    tr.ensure_capacity(views, slack=2.0)
    n_seg = max(1, int(round(budget_s / eval_every_s)))
    seg_s = budget_s / n_seg
    curve = [(0.0, eval_psnr(tr, eval_cams, eval_rgb))]
    steps = 0
    trained = 0.0
    order = []
    densify_log = []
    for seg in range(n_seg):
        frac = seg / n_seg
        tr.disp_weight = disp_weight * (1.0 - frac)
        if method not in ("ng", "ng_frozen"):
            tr.set_lr("means", lr0 * 0.01 ** frac)
        if method == "pose":
            tr.set_pose_lr(pose_cfg["lr_rot"] * 0.01 ** frac, pose_cfg["lr_trans"] * 0.01 ** frac)
        graphs = None
        if method == "batched_graph":
            graphs = [tr.capture(b_cams[b], b_rgb[b], b_disp[b]) for b in range(len(b_cams))]
        chunk = 4 if method == "batched_graph" else 16
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < seg_s:
            for _ in range(chunk):
                if not order:
                    order = list(rng.permutation(len(views)))
                i = order.pop()
                if graphs is not None:
                    graphs[i].replay()
                else:
                    tr.step(views[i], train_rgb[i], train_disp[i])
                steps += 1
            torch.cuda.synchronize()
        if method == "densify" and seg < n_seg // 2:
            pick = rng.choice(nv, size=min(densify_k, nv), replace=False)
            rules = dict({"extent": extent}, **(densify_rules or {}))
            info = tr.densify([train_cams[i] for i in pick], [train_rgb[i] for i in pick], tau=densify_tau,
                              rules=rules, seed=seed + seg, max_gaussians=max_gaussians)
            tr.ensure_capacity(views, slack=2.0)
            densify_log.append(info)
            torch.cuda.synchronize()
        trained += time.perf_counter() - t0
        st = tr.slot_for(views[0]).plan.status()
        if st["error"]:
            raise RuntimeError(f"device status during {method}: {st}")
        if st["overflow"]:  # grown scene: more instances than planned
            tr.ensure_capacity(views, slack=2.0)
        del graphs
        curve.append((trained, eval_psnr(tr, eval_cams, eval_rgb)))
    per_step = batch if method == "batched_graph" else 1
    extra = {}
    if method == "pose":
        R, t = tr.pose.correction()
        extra["pose_correction"] = {"R": R.tolist(), "t": t.tolist(), "updates": int(tr.pose.buf[24].item())}
    if method == "batched_graph":
        extra["lr_scale"] = lrs["log_scales"] / default_lrs(extent)["log_scales"]
        extra["betas"] = list(tr.betas)
    return {**extra, "method": method, "curve": curve, "psnr_final": curve[-1][1], "psnr_start": curve[0][1],
            "steps": steps, "views": steps * per_step, "seconds": trained,
            "views_per_s": steps * per_step / trained, "gaussians_final": tr.params.n,
            "densify": densify_log}


def time_to_psnr(curve, target: float) -> float | None:
    """Training seconds at which a held-out PSNR curve [(seconds, PSNR)]
    first reaches `target`, interpolated linearly between evaluations; None
    if it never does."""
    for (t0, p0), (t1, p1) in zip(curve[:-1], curve[1:]):
        if p0 >= target:
            return float(t0)
        if p1 >= target:
            return float(t0 + (t1 - t0) * (target - p0) / (p1 - p0))
    return float(curve[0][0]) if curve and curve[0][1] >= target else None
