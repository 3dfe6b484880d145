"""Launch-shape autotuner for the training step.

The choices change speed, not results (beyond float32 summation order):
  load_balanced  warp-cooperative (LB) or one-thread-per-Gaussian (Sq) tile-key
                 write of the binning (Sec. 2.1 compares the two);
  bucket         splats per checkpoint bucket and per backward work unit
                 (Sec. 2.2 uses 32; 64 halves the checkpoint traffic and runs
                 the backward with two splats per lane in packed pairs);
  bwd_warps      warps per CTA of the per-Gaussian backward;
  bwd_chains     pixel chains per lane of the 32-splat backward pipeline (1,
                 2, or 0: chosen per bucket by its live pixel count);
  fwd_pixels     pixels per thread of the forward blend (1, or 2 in packed
                 float32 pairs).
Tile size stays at the paper's 16 x 16 (Sec. 2.2).

``autotune`` times a few real training steps of candidates on the caller's
own views and targets, using a scratch copy of the parameters so that
tuning does not train the model, and returns the fastest.  The binning
mode is settled first (at the default backward shape); the backward shapes
are then searched with the faster binning, and last the forward's pixels per
thread with the best of them.
"""
from __future__ import annotations

import itertools
import statistics

import torch

from .api import Gaussians
from .trainer import Trainer

BINNING = ({"load_balanced": True, "bucket": 64, "bwd_warps": 1, "bwd_chains": 0},
           {"load_balanced": False, "bucket": 64, "bwd_warps": 1, "bwd_chains": 0})
# 32-splat buckets: one splat per lane, CTA width and pixel chains searched;
# 64-splat buckets: two splats per lane in packed pairs (one chain), CTA
# width searched
SHAPES = (tuple({"bucket": 32, "bwd_warps": w, "bwd_chains": c}
                for w, c in itertools.product((2, 4, 8), (0, 1, 2)))
          + tuple({"bucket": 64, "bwd_warps": w, "bwd_chains": 0} for w in (1, 2, 4)))


TUNED = ("bucket", "bwd_warps", "bwd_chains", "fwd_pixels")


def tuning_key(load_balanced: bool, t: dict) -> str:
    """'LB/b64/w1/c0', with '/f2' appended for the two-pixel forward."""
    return (f"{'LB' if load_balanced else 'Sq'}/b{t['bucket']}/w{t['bwd_warps']}/c{t['bwd_chains']}"
            + ("/f2" if t.get("fwd_pixels", 1) == 2 else ""))


def parse_tuning_key(key: str) -> tuple[bool, dict]:
    """Inverse of tuning_key: (load_balanced, tuning dict)."""
    parts = key.split("/")
    t = {"bucket": int(parts[1][1:]), "bwd_warps": int(parts[2][1:]), "bwd_chains": 0, "fwd_pixels": 1}
    for p in parts[3:]:
        if p.startswith("c"):
            t["bwd_chains"] = int(p[1:])
        elif p.startswith("f"):
            t["fwd_pixels"] = int(p[1:])
    return parts[0] == "LB", t


def _key(c: dict) -> str:
    return tuning_key(c["load_balanced"], c)


def _clone(params: Gaussians) -> Gaussians:
    return Gaussians(*(t.clone() for t in params.tensors()), params.sh_degree)


def _time(scratch, cand, batches, targets, lam, trials, inst_capacity, device) -> float:
    tr = Trainer(scratch, lam=lam, load_balanced=cand["load_balanced"], inst_capacity=inst_capacity,
                 tuning={k: cand.get(k, 1 if k == "fwd_pixels" else 0) for k in TUNED}, device=device)
    tr.ensure_capacity(batches)
    for b, t in zip(batches, targets):  # warm-up: every launch shape once
        tr.step(b, t)
    times = []
    for _ in range(trials):
        for b, t in zip(batches, targets):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            tr.step(b, t)
            e1.record()
            times.append((e0, e1))
    torch.cuda.synchronize()
    return statistics.median(a.elapsed_time(z) for a, z in times)


def autotune(params: Gaussians, batches, targets, *, lam: float = 0.2, trials: int = 3,
             inst_capacity: int | None = None, device="cuda"):
    """batches: list of camera lists (one training step each); targets: the
    matching flat colour targets on the device.  Returns (best candidate,
    {candidate key: median ms per step})."""
    table = {}
    scratch = _clone(params)
    for cand in BINNING:
        table[_key(cand)] = _time(scratch, cand, batches, targets, lam, trials, inst_capacity, device)
    lb = min(BINNING, key=lambda c: table[_key(c)])["load_balanced"]
    best, best_ms = None, float("inf")
    for shape in SHAPES:
        cand = {"load_balanced": lb, **shape}
        k = _key(cand)
        if k not in table:
            table[k] = _time(scratch, cand, batches, targets, lam, trials, inst_capacity, device)
        if table[k] < best_ms:
            best, best_ms = dict(cand), table[k]
    best["fwd_pixels"] = 1
    cand = {**best, "fwd_pixels": 2}
    table[_key(cand)] = _time(scratch, cand, batches, targets, lam, trials, inst_capacity, device)
    if table[_key(cand)] < best_ms:
        best = cand
    del scratch
    torch.cuda.empty_cache()
    return best, table
