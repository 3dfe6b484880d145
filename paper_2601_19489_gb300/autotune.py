"""Launch-shape autotuner for the training step.

The choices change speed, not results (beyond float32 summation order):
  load_balanced  warp-cooperative (LB) or one-thread-per-Gaussian (Sq) tile-key
                 write of the binning (Sec. 2.1 compares the two);
  bucket         splats per checkpoint bucket and per backward work unit
                 (Sec. 2.2 uses 32; 64 halves the checkpoint traffic);
  bwd_warps      warps per CTA of the per-Gaussian backward.
Tile size stays at the paper's 16 x 16 (Sec. 2.2).

``autotune`` times a few real training steps of every candidate on the
caller's own views and targets, using a scratch copy of the parameters so
that tuning does not train the model, and returns the fastest.
"""
from __future__ import annotations

import itertools
import statistics

import torch

from .api import Gaussians
from .trainer import Trainer

CANDIDATES = tuple({"load_balanced": lb, "bucket": b, "bwd_warps": w}
                   for lb, b, w in itertools.product((True, False), (32, 64), (2, 4, 8)))


def _clone(params: Gaussians) -> Gaussians:
    return Gaussians(*(t.clone() for t in params.tensors()), params.sh_degree)


def autotune(params: Gaussians, batches, targets, *, lam: float = 0.2, trials: int = 3,
             candidates=CANDIDATES, inst_capacity: int | None = None, device="cuda"):
    """batches: list of camera lists (one training step each); targets: the
    matching flat colour targets on the device.  Returns (best candidate,
    {candidate key: median ms per step})."""
    table = {}
    best, best_ms = None, float("inf")
    scratch = _clone(params)
    for cand in candidates:
        tr = Trainer(scratch, lam=lam, load_balanced=cand["load_balanced"], inst_capacity=inst_capacity,
                     tuning={"bucket": cand["bucket"], "bwd_warps": cand["bwd_warps"]}, device=device)
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
        ms = statistics.median(a.elapsed_time(z) for a, z in times)
        key = f"{'LB' if cand['load_balanced'] else 'Sq'}/b{cand['bucket']}/w{cand['bwd_warps']}"
        table[key] = ms
        if ms < best_ms:
            best, best_ms = dict(cand), ms
        del tr
    del scratch
    torch.cuda.empty_cache()
    return best, table
