"""Launch-shape autotuner for the training step.

The choices change speed, not results (beyond float32 summation order):
  load_balanced  warp-cooperative (LB) or one-thread-per-Gaussian (Sq) tile-key
                 write of the binning (Sec. 2.1 compares the two);
  bucket         splats per checkpoint bucket and per backward work unit
                 (Sec. 2.2 uses 32; 64 halves the checkpoint traffic and runs
                 the backward with two splats per lane in packed pairs);
  bwd_warps      warps per CTA of the per-Gaussian backward;
  bwd_chains     pixel chains per lane of the 32-splat backward pipeline (1,
                 2, or 0: chosen per bucket by its live pixel count).
Tile size stays at the paper's 16 x 16 (Sec. 2.2).

``autotune`` times a few real training steps of candidates on the caller's
own views and targets, using a scratch copy of the parameters so that
tuning does not train the model, and returns the fastest.  The binning
mode is settled first (at the default backward shape); the backward shapes
are then searched with the faster binning.
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


def _key(c: dict) -> str:
    return (f"{'LB' if c['load_balanced'] else 'Sq'}/b{c['bucket']}/w{c['bwd_warps']}/"
            f"c{c['bwd_chains']}")


def _clone(params: Gaussians) -> Gaussians:
    return Gaussians(*(t.clone() for t in params.tensors()), params.sh_degree)


def _time(scratch, cand, batches, targets, lam, trials, inst_capacity, device) -> float:
    tr = Trainer(scratch, lam=lam, load_balanced=cand["load_balanced"], inst_capacity=inst_capacity,
                 tuning={k: cand[k] for k in ("bucket", "bwd_warps", "bwd_chains")}, device=device)
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
    del scratch
    torch.cuda.empty_cache()
    return best, table
