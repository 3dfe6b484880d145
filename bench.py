#!/usr/bin/env python
"""Throughput of the GB300 3DGS training step.

Metric: train steps/s (forward + backward + Adam) at 1M Gaussians, 1080p.
Workload: 2^20 Gaussians in 64 anisotropic clusters (SH degree 3), 16 ring
cameras at 1920x1080, 16x16 tiles, loss 0.8 L1 + 0.2 (1 - SSIM); one view
per step, round robin.  Synthetic, seeded inputs stand in for the paper's
Tanks-and-Temples / challenge scenes (not available).

One step = preprocess, bin + sort, forward blend, loss, per-Gaussian
backward, preprocess backward, Adam, all on the GPU through libgs.so.  The
timed steps replay one captured CUDA graph per view (Trainer.capture; the
same 27 launches as an eager step, without the per-launch host overhead);
an eager pass over the same steps from the same state, with CUDA events
between the stages, gives the stage split (--eager times eager steps).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank trains its own replica on its own GPU (the
step has no cross-GPU exchange); the value is the sum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "train steps/s (fwd+bwd+Adam) @1M Gaussians 1080p"
UNIT = "steps/s"
# Peak numbers: measured by the pool's driver (MEASURED_PEAKS.json) where it
# exists; FP32 ALU peak = 152 SMs x 128 FP32 lanes x 2 FLOP x 2070 MHz.
FALLBACK_HBM_GBS = 6800.0
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# Algorithmic floating-point work per evaluated pixel-splat pair, counted
# from the kernels' arithmetic (FMA = 2): forward blend 25, backward 62.
FLOP_PER_PAIR = {"render_fwd": 25.0, "render_bwd_blend": 62.0}
# CPU oracle samples: WINDOW x WINDOW pixel windows, one per cell of an
# 8 x 5 grid over the image in the cpu_baseline leg, one per step (cells in
# rotation) in the reference arm; preprocess and Adam on a random subset
WINDOW = 16
REF_PRE_SAMPLE = 1 << 12
BASELINE_PRE_SAMPLE = 1 << 18
# DRAM bytes per launch from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum, 1 pass, on this workload at full size: 1M Gaussians,
# one 1920x1080 view), valid only for the kernel source they were taken on
# (sha256 of the .cu file, first 16 hex digits) and the same launch shape.
NCU_TRAFFIC: dict = {
    "k_render_bwd_pk": {"bytes_per_launch": 1.84628e8, "src_sha": "e9218455b5419109", "tuning": "LB/b64/w1/c0/f2",
                        "read": 1.79498e8, "write": 5.130e6},
}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--n", "--gaussians", dest="n", type=int, default=1 << 20)
    ap.add_argument("--width", type=int, default=1920)
    ap.add_argument("--height", type=int, default=1080)
    ap.add_argument("--views", type=int, default=16)
    ap.add_argument("--lam", type=float, default=0.2)
    ap.add_argument("--sq", action="store_true", help="sequential tile-key write instead of load-balanced")
    ap.add_argument("--tuning", type=str, default="",
                    help="fixed launch shapes instead of the autotuner, e.g. LB/b32/w2/c0")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched CUDA-graph measurement")
    ap.add_argument("--batched-steps", type=int, default=60)
    ap.add_argument("--no-ng", action="store_true", help="skip the neural-Gaussian step measurement")
    ap.add_argument("--workload", choices=("explicit", "batched", "recon60", "ablation"), default="explicit",
                    help="batched: only the 8-view CUDA-graph step, one line per --batched-n; "
                         "recon60: held-out PSNR after a timed reconstruction")
    ap.add_argument("--recon-budget", type=float, default=60.0, help="seconds of training per method")
    ap.add_argument("--recon-methods", type=str, default="plain,densify,batched_graph,ng,ng_frozen")
    ap.add_argument("--recon-batch-lr-scale", type=float, default=None,
                    help="learning-rate scale of the batched method (default sqrt(8))")
    ap.add_argument("--densify-tau-plus", type=float, default=5.0)
    ap.add_argument("--batched-n", type=str, default="",
                    help="comma-separated Gaussian counts for --workload batched (default: --n)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--eager", action="store_true",
                    help="time the headline steps as eager launches instead of per-view CUDA graph replays")
    ap.add_argument("--no-pose", action="store_true", help="skip the pose-refinement overhead measurement")
    ap.add_argument("--no-visible-adam", action="store_true", help="skip the visible-only Adam measurement")
    ap.add_argument("--recon-pose-error", type=str, default="",
                    help="'rot_rad,trans': give every recon view one seeded camera-side pose error "
                         "(methods suffixed @true keep the true poses)")
    return ap.parse_args()


def workload(args):
    import synth

    scene = synth.scene_clustered(args.n, seed=0, sh_degree=3)
    cams = synth.ring_cameras(args.views, args.width, args.height)
    return scene, cams


def render_targets(n: int, cams, dev, seed: int = 1, bg=(0.0, 0.0, 0.0)):
    """Training targets: a second seeded clustered scene of the same kind (n
    Gaussians, SH degree 3) rendered through the same cameras by the CUDA
    forward, one flat planar colour image per camera (device tensors).  A
    workload to fit, not a parity reference: the oracle would take hours per
    1080p view of a 1M-Gaussian scene."""
    import torch

    import synth
    from paper_2601_19489_gb300 import api
    from paper_2601_19489_gb300.trainer import Trainer

    tgt_scene = synth.scene_clustered(n, seed=seed, sh_degree=3)
    tr = Trainer(api.Gaussians.from_scene(tgt_scene, device=dev), lam=0.2, bg=bg, device=dev)
    tr.ensure_capacity([[c] for c in cams])
    out = []
    for c in cams:
        sl = tr.forward([c])
        out.append(sl.rgb[: 3 * c.width * c.height].clone())
    torch.cuda.synchronize()
    del tr
    torch.cuda.empty_cache()
    return out


def config_of(args):
    return {"workload": f"clustered {args.n} Gaussians SH3, {args.views} ring views {args.width}x{args.height}, "
                        f"16x16 tiles, loss {1 - args.lam:.1f} L1 + {args.lam:.1f} D-SSIM, one view per step",
            "gaussians": args.n, "views": args.views, "width": args.width, "height": args.height,
            "targets": "a second seeded clustered scene (seed 1, same size) rendered through the same cameras",
            "tile": 16, "bucket": 64, "sh_degree": 3, "binning": "radix, sequential key write" if args.sq else "counting",
            "l2": "working set > L2 (params + Adam state ~1 GB, instances, checkpoints); no flush"}


# ------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = [r.split(",") for r in (self.out or "").strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def src_sha(name: str) -> str:
    p = os.path.join(ROOT, "paper_2601_19489_gb300", "csrc", name)
    with open(p, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


# ------------------------------------------------------------ CPU oracle

def window_cells(W: int, H: int):
    """The grid of cells the CPU samples stratify over: 240 x 216 pixels at
    1920 x 1080 (8 x 5 = 40 cells)."""
    nx, ny = max(1, W // 240), max(1, H // 216)
    return nx, ny, W // nx, H // ny


def sample_windows(W: int, H: int, cells, seed: int, size: int = WINDOW):
    """One size x size window per listed cell of window_cells's grid, at a
    seeded position anywhere inside the cell.  Listing every cell gives a
    stratified sample of the whole image; the positions differ per seed."""
    rng = np.random.default_rng(seed)
    nx, ny, cw, ch = window_cells(W, H)
    out = []
    for c in cells:
        x0 = (c % nx) * cw + int(rng.integers(0, max(1, cw - size)))
        y0 = (c // nx) * ch + int(rng.integers(0, max(1, ch - size)))
        out.append((int(x0), int(y0), int(x0) + size, int(y0) + size))
    return out


def near_windows(rec: np.ndarray, wins) -> np.ndarray:
    """The render records of the Gaussians whose level-set box (Eq. 1 level
    set, widened by one pixel) reaches one of the windows (in input order).  The oracle builds its per-pixel candidate lists from
    every Gaussian on each call, so without this each small window would also
    pay a pass over all N Gaussians, a cost that does not scale with the
    window's area; outside its box a Gaussian reaches no pixel, so the
    windows' results are unchanged."""
    a, b, c, t = rec[:, 2], rec[:, 3], rec[:, 4], rec[:, 10]
    det = a * c - b * b
    ok = (rec[:, 11] > 0) & (t > 0) & (det > 0)
    with np.errstate(divide="ignore", invalid="ignore"):
        rx = np.sqrt(np.where(ok, t * c / det, 0.0)) + 1.0
        ry = np.sqrt(np.where(ok, t * a / det, 0.0)) + 1.0
    hit = np.zeros(rec.shape[0], bool)
    for (x0, y0, x1, y1) in wins:
        hit |= (rec[:, 0] + rx >= x0) & (rec[:, 0] - rx <= x1) & (rec[:, 1] + ry >= y0) & (rec[:, 1] - ry <= y1)
    return rec[ok & hit]


def oracle_records(scene, cam):
    """The oracle's render records of every Gaussian for one view (setup of
    the CPU samples, untimed)."""
    import torch

    from oracle import preprocess as opre

    with torch.no_grad():
        return opre.pack_for_render(opre.project(opre.params_from_scene(scene), cam, scene.sh_degree))


def sample_plan(W: int, H: int, n_views: int, steps):
    """The (view, window) of each CPU sample step s: view s mod n_views, one
    seeded window (seed s) in cell 7 s mod 40 of the 8 x 5 grid, so 40
    consecutive steps visit every cell once."""
    nx, ny, _, _ = window_cells(W, H)
    n_cells = nx * ny
    stride = next(k for k in (7, 3, 1) if n_cells % k or k == 1)
    return [(s % n_views, sample_windows(W, H, [(stride * s) % n_cells], seed=s)[0]) for s in steps]


def oracle_sample(scene, groups, pre_cam, pre_sample: int, n_threads: int, seed: int = 0):
    """Time the float64 oracle on a bounded sample of one training step and
    extrapolate to the whole step.  Returns (seconds per full step, detail).

    preprocess fwd+bwd and Adam: a random subset of `pre_sample` Gaussians on
    view pre_cam, scaled by N / pre_sample; blend fwd + loss + per-pixel bwd:
    the windows of `groups`, a list of (cam, rec_full, trec_full, windows)
    (rec_full / trec_full: that view's records of the trained and of the
    target scene, oracle_records), scaled by one view's H * W over the
    windows' pixels.  The target inside each window is the oracle's own
    render of the target scene there (setup, untimed)."""
    import torch

    from oracle import preprocess as opre
    from oracle import render as oren
    from oracle import loss as oloss
    from oracle import adam as oadam
    import synth

    torch.set_num_threads(n_threads)
    rng = np.random.default_rng(seed)
    N = scene.n
    sub = np.sort(rng.choice(N, size=min(pre_sample, N), replace=False))
    sub_scene = synth.Scene(*(a[sub] for a in scene.arrays()), sh_degree=scene.sh_degree)
    W, H = pre_cam.width, pre_cam.height
    work = []
    for cam, rec_full, trec_full, wins in groups:
        rec = near_windows(rec_full, wins)
        trec = near_windows(trec_full, wins)
        for w in wins:
            work.append((rec, w, oren.render_fwd(trec, (0.0, 0.0, 0.0), w, amb=None, n_threads=n_threads)["rgb"]))
    t0 = time.perf_counter()
    with torch.no_grad():
        opre.project(opre.params_from_scene(sub_scene), pre_cam, scene.sh_degree)
    g2d = rng.standard_normal((sub.size, 10))
    grads = opre.preprocess_backward(sub_scene, pre_cam, g2d)
    t1 = time.perf_counter()
    pairs = 0
    for rec, w, tgt in work:
        f = oren.render_fwd(rec, (0.0, 0.0, 0.0), w, amb=None, n_threads=n_threads)
        _, g_rgb = oloss.photometric(f["rgb"], tgt, 0.2)
        oren.render_bwd(rec, (0.0, 0.0, 0.0), w, g_rgb, np.zeros_like(f["disp"]), n_threads=n_threads)
        pairs += f["pairs"]
    t2 = time.perf_counter()
    for k, v in grads.items():
        oadam.adam_step(getattr(sub_scene, k), v, np.zeros_like(v), np.zeros_like(v), 1, 1e-3)
    t3 = time.perf_counter()
    scale_g = N / sub.size
    px = float(sum((w[2] - w[0]) * (w[3] - w[1]) for _, w, _ in work))
    scale_p = (W * H) / px
    est = (t1 - t0) * scale_g + (t2 - t1) * scale_p + (t3 - t2) * scale_g
    detail = {"preprocess_s": (t1 - t0) * scale_g, "render_s": (t2 - t1) * scale_p,
              "adam_s": (t3 - t2) * scale_g, "measured_s": t3 - t0, "pairs": pairs,
              "pairs_per_px": pairs / px, "windows": len(work)}
    return est, detail


def run_reference(args, rank, world):
    """The reference arm: the float64 oracle as it stands, on the host cores.
    Step s renders one window in cell (7 s mod 40) of view s mod 16, so every
    40 steps cover all cells of the image once; the per-view records are
    computed once beforehand (untimed)."""
    if rank != 0:
        return
    scene, cams = workload(args)
    import synth

    target_scene = synth.scene_clustered(args.n, seed=1, sh_degree=3)
    n_threads = os.cpu_count() or 1
    nx, ny, _, _ = window_cells(args.width, args.height)
    records = {}
    times = []
    for s, (v, win) in zip(range(args.warmup + args.steps),
                           sample_plan(args.width, args.height, len(cams), range(args.warmup + args.steps))):
        cam = cams[v]
        if v not in records:
            records[v] = (oracle_records(scene, cam), oracle_records(target_scene, cam))
        est, _ = oracle_sample(scene, [(cam, *records[v], [win])], cam, pre_sample=REF_PRE_SAMPLE,
                               n_threads=n_threads, seed=s)
        if s >= args.warmup:
            times.append(est)
    value = 1.0 / float(np.mean(times))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(args), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": n_threads, "kind": "oracle",
                             "sample": f"per step s (view s mod {len(cams)}): preprocess fwd+bwd and Adam on "
                                       f"{REF_PRE_SAMPLE} random Gaussians (x N/{REF_PRE_SAMPLE}), blend "
                                       f"fwd+loss+bwd on one seeded {WINDOW}x{WINDOW} window in cell "
                                       f"(7 s mod {nx * ny}) of a {nx}x{ny} grid over the image "
                                       f"(x H*W/{WINDOW * WINDOW}); the mean over steps covers every cell"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ GPU arm

def bin_bytes(n: int, instances: float, entries: float = 0.0, chunks: float = 0.0, tiles: int = 0,
              counting: bool = True) -> float:
    """Algorithmic bytes of the binning stage.
      both paths    depth sort 4 passes x 20 B per Gaussian (keys and
                    values read, written; the upsweep's key read)
      counting      per Gaussian: entry count and entry write read its
                    order, count and rectangle twice (2 x 16 B); per
                    (Gaussian, block) entry: 8 B written, one sort pass
                    20 B, two column walks reading the entry and its
                    record, level set and rectangle (2 x 40 B); per
                    instance the 4 B id written once; per chunk its 64
                    tile counts written, rescanned and read (3 x 256 B);
                    per tile its range (8 B)
      radix         counts 72 B per Gaussian; per instance the 8 B key
                    write, two tile-sort passes 2 x 20 B and the range
                    search 8 B"""
    if counting:
        return 80 * n + 32 * n + 108 * entries + 4 * instances + 768 * chunks + 8 * tiles
    return 152 * n + 56 * instances


def stage_roofline(stage_ms: dict, n: int, sh_degree: int, pixels: int, bin_b: float, pairs: float,
                   hbm_gbs: float, ssim: bool = True) -> dict:
    """Each stage's achieved rate against its bound, from the algorithmic
    work per unit (parameters of P = 4 (11 + 3 K) bytes per Gaussian):
      preprocess    P read + 76 B of records written per Gaussian      (HBM)
      bin_sort      bin_bytes                                          (HBM)
      render_fwd    25 FLOP per pixel-splat pair                       (FP32)
      loss          with SSIM: 1215 FLOP per pixel (per channel: x^2,
                    y^2, x y 3; five 11-tap separable window sums 220;
                    SSIM and its three partials 40; L1 2; three 11-tap
                    separable sums of the maps 132; the gradient 8)    (FP32)
                    plain L1: 36 B per pixel                           (HBM)
      render_bwd    62 FLOP per pixel-splat pair                       (FP32)
      fused bwd     2 P parameters + 4 P moments per Gaussian          (HBM)
    Pairs are counted up to each pixel's last contributor."""
    P = 4 * (11 + 3 * (sh_degree + 1) ** 2)
    work = {"preprocess": ("hbm", (P + 76) * n), "bin_sort": ("hbm", bin_b),
            "render_fwd": ("alu", 25 * pairs), "loss": ("alu", 1215 * pixels) if ssim else ("hbm", 36 * pixels),
            "render_bwd_blend": ("alu", 62 * pairs), "preprocess_bwd_adam": ("hbm", 6 * P * n)}
    out = {}
    for name, (bound, w) in work.items():
        if name not in stage_ms or stage_ms[name] <= 0:
            continue
        sec = stage_ms[name] / 1e3
        if bound == "hbm":
            ach = w / sec / 1e9
            out[name] = {"bound": "hbm", "achieved": ach, "unit": "GB/s", "frac": ach / hbm_gbs}
        else:
            ach = w / sec / 1e12
            out[name] = {"bound": "alu", "achieved": ach, "unit": "TFLOP/s", "frac": ach / FP32_PEAK_TFLOPS}
    return out


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest of every rank's x (each rank's timed region; the job
    takes as long as its slowest rank)."""
    if world <= 1:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, steps: int, seconds: float) -> float:
    """Whole-job throughput: every rank runs `steps` steps of its own views
    (replicas, weak scaling) in at most `seconds`."""
    return world * steps / seconds


def block_bits(sizes) -> int:
    """Bits of the block ids of the counting binning (8 x 8-tile blocks)."""
    blocks = sum(-(-(-(-w // 16)) // 8) * -(-(-(-h // 16)) // 8) for (w, h) in sizes)
    return max(1, int(np.ceil(np.log2(blocks))) if blocks > 1 else 1)


def kernels_per_step(trainer, sizes) -> int:
    # loss: the fused SSIM pass (or L1 + final reduction), and the disparity
    # L1 when it is weighted
    loss_k = (1 if trainer.lam > 0 else 2) + (1 if trainer.disp_weight > 0 else 0)
    # preprocess 1; depth sort 4 passes x 3; then the binning: counting
    # (entry count 1, entry write 1, entry sort 3/pass, block bounds 1 when
    # the sort takes more than one pass, chunk scan 1, mask / offsets /
    # scatter 3) or radix (count 1, keys 1, tile sort 3/pass, ranges 1);
    # forward 1; loss; blend bwd 1; then either the fused preprocess backward
    # + Adam (step-count tick + 1) or preprocess bwd 1 + adam 2 (tick +
    # update)
    tail = 2 if trainer.fused_adam else 3
    if trainer.load_balanced and not trainer.tuning.get("bin_radix", 0):
        passes = -(-block_bits(sizes) // 8)
        binning = 2 + 3 * passes + (1 if passes > 1 else 0) + 1 + 3
    else:
        binning = 2 + 3 * -(-trainer.plan_tile_bits // 8) + 1
    return 1 + 12 + binning + 1 + loss_k + 1 + tail


def run_ours(args, rank, world):
    import torch

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2601_19489_gb300 import api
    from paper_2601_19489_gb300 import _lib as L
    from paper_2601_19489_gb300.trainer import Trainer
    from paper_2601_19489_gb300.autotune import TUNED, parse_tuning_key, tuning_key
    import synth

    L.load()
    scene, cams = workload(args)
    params = api.Gaussians.from_scene(scene, device=dev)
    targets_d = render_targets(args.n, cams, dev)
    tuning, lb, table = {}, not args.sq, None
    if args.tuning:
        lb, tuning = parse_tuning_key(args.tuning)
    elif not args.sq:  # launch shapes from the autotuner, on this workload's own views
        from paper_2601_19489_gb300.autotune import TUNED, autotune

        best, table = autotune(params, [[cams[0]], [cams[1]]], targets_d[:2], lam=args.lam, device=dev)
        tuning = {k: best[k] for k in TUNED}
        lb = best["load_balanced"]
    trainer = Trainer(params, args.width, args.height, lam=args.lam, load_balanced=lb, tuning=tuning, device=dev)
    trainer.autotune_table = table
    tu = trainer.slot_for([cams[0]]).plan.tuning
    trainer_tuning_key = tuning_key(lb, tu)
    ntiles = ((args.width + 15) // 16) * ((args.height + 15) // 16)
    trainer.plan_tile_bits = max(1, int(np.ceil(np.log2(ntiles))))
    targets_h = [t.cpu().pin_memory() for t in targets_d]
    torch.cuda.synchronize()
    worst = trainer.ensure_capacity(cams)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # (at least one eager step: every kernel is loaded before a graph is captured)
    for s in range(max(1, args.warmup)):
        trainer.step(cams[s % len(cams)], targets_d[s % len(cams)])
    barrier()
    st0 = trainer.plan.status()
    assert st0["rc"] == 0, st0
    # the training state after the warm-up: every timed pass below restarts
    # from it, so that all of them time the same stretch of the same run (the
    # scene changes as it trains, and with it the work per step)
    snapshot = [t.clone() for t in trainer._state_tensors().values()] + [trainer.d_step.clone()]
    step_count0 = trainer.step_count

    def restore():
        for dst, src in zip(list(trainer._state_tensors().values()) + [trainer.d_step], snapshot):
            dst.copy_(src)
        trainer.step_count = step_count0
        barrier()

    # the headline steps: each view's whole step (27 launches) captured once
    # in a CUDA graph (Trainer.capture) and replayed, the views round robin
    graphs = None if args.eager else [trainer.capture([c], t) for c, t in zip(cams, targets_d)]
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        start.record(stream)
        for s in range(args.steps):
            v = (args.warmup + s) % len(cams)
            if graphs is None:
                trainer.step(cams[v], targets_d[v])
            else:
                graphs[v].replay()
        end.record(stream)
        barrier()
    clocks = clk.summary()
    elapsed = start.elapsed_time(end) / 1e3
    st1 = trainer.plan.status()
    if st1["rc"] != 0:
        raise RuntimeError(f"device status after the timed region: {st1}")
    elapsed = max_over_ranks(elapsed, world, dev)

    # the same steps again from the same state, eager, with CUDA events
    # between the stages on the launching stream: the stage split and the
    # dominant kernel's launch duration
    restore()
    n_st = len(trainer.STAGES)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(n_st + 1)] for _ in range(args.steps)]
    e_start = torch.cuda.Event(enable_timing=True)
    e_end = torch.cuda.Event(enable_timing=True)
    e_start.record(stream)
    for s in range(args.steps):
        v = (args.warmup + s) % len(cams)
        trainer.step(cams[v], targets_d[v], events=evs[s])
    e_end.record(stream)
    barrier()
    eager_ms = e_start.elapsed_time(e_end) / args.steps
    st1e = trainer.plan.status()
    if st1e["rc"] != 0:
        raise RuntimeError(f"device status after the eager pass: {st1e}")
    stage_ms = {name: float(np.mean([evs[s][i].elapsed_time(evs[s][i + 1]) for s in range(args.steps)]))
                for i, name in enumerate(trainer.STAGES)}
    # per step from its first stage event to its last: the protocol the
    # neural-Gaussian leg is timed with
    eager_step_ms = float(np.mean([evs[s][0].elapsed_time(evs[s][n_st]) for s in range(args.steps)]))

    # algorithmic work of the blend kernels: evaluated pairs up to each
    # pixel's last contributor, summed over the views of the timed steps
    pairs = []
    for s in range(args.steps):
        v = (args.warmup + s) % len(cams)
        if len(pairs) >= len(cams):
            break
        trainer.forward(cams[v])
        nc = trainer.plan.view(L.GS_WS_N_CONTRIB, torch.int32)[: args.width * args.height]
        pairs.append(float(nc.double().sum().item()))
    mean_pairs = float(np.mean(pairs))
    st2 = trainer.plan.status()
    words = trainer.plan.view(L.GS_WS_STATUS, torch.int32)
    counting = trainer.load_balanced and not trainer.tuning.get("bin_radix", 0)
    tiles = -(-args.width // 16) * -(-args.height // 16)
    bin_b = bin_bytes(args.n, st2["n_instances"], float(words[5].item()), float(words[6].item()), tiles,
                      counting=counting)

    # e2e: through the public API with host buffers, the target copied in from
    # pinned host memory and the loss read back every step.  Eager: the next
    # step's target goes to a second buffer on a side stream while the current
    # step runs (HostFeeder).  Graphs: a view's graph reads that view's target
    # buffer, which the side stream refills from the host before the replay
    # (events order the copy after the buffer's last replay and before the next).
    e2e = None
    if not args.no_e2e:
        from paper_2601_19489_gb300.trainer import HostFeeder

        restore()
        loss_h = torch.empty(1, pin_memory=True)
        barrier()
        t0 = time.perf_counter()
        if graphs is None:
            feeder = HostFeeder(targets_d[0])
            for s in range(args.steps):
                v = (args.warmup + s) % len(cams)
                nxt = targets_h[(args.warmup + s + 1) % len(cams)] if s + 1 < args.steps else None
                tgt = feeder.get(targets_h[v], nxt)
                trainer.step(cams[v], tgt)
                feeder.done()
                loss_h.copy_(trainer.loss, non_blocking=True)
        else:
            side = torch.cuda.Stream(dev)
            ready = [torch.cuda.Event() for _ in cams]
            free = [torch.cuda.Event() for _ in cams]

            def refill(v):
                side.wait_event(free[v])  # the view's previous replay is done with its buffer
                with torch.cuda.stream(side):
                    targets_d[v].copy_(targets_h[v], non_blocking=True)
                    ready[v].record(side)

            refill(args.warmup % len(cams))
            for s in range(args.steps):
                v = (args.warmup + s) % len(cams)
                if s + 1 < args.steps:
                    refill((args.warmup + s + 1) % len(cams))
                stream.wait_event(ready[v])
                graphs[v].replay()
                free[v].record(stream)
                loss_h.copy_(trainer.loss, non_blocking=True)
        barrier()
        t_e2e = max_over_ranks(time.perf_counter() - t0, world, dev)
        e2e = {"value": job_rate(world, args.steps, t_e2e), "unit": UNIT,
               "h2d_bytes_per_step": int(targets_h[0].numel() * 4), "d2h_bytes_per_step": 4}

    if rank != 0:
        return
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    dominant = max(stage_ms, key=stage_ms.get)
    stages_roof = stage_roofline(stage_ms, args.n, 3, args.width * args.height, bin_b, mean_pairs,
                                 hbm or FALLBACK_HBM_GBS, ssim=args.lam > 0)
    bucket = trainer.slot_for([cams[0]]).plan.tuning["bucket"]
    kname = {"render_bwd_blend": "k_render_bwd_pk" if bucket == 64 else "k_render_bwd",
             "render_fwd": "k_render_fwd_pk" if tu["fwd_pixels"] == 2 else "k_render_fwd",
             "preprocess": "k_preprocess",
             "preprocess_bwd_adam": "k_preprocess_bwd (Adam fused)", "loss": "k_ssim_fused",
             "bin_sort": ("bin_sort (depth sort, counting binning)" if counting else
                          "bin_sort (depth sort, key write, tile sort)")}.get(dominant, dominant)
    sr = stages_roof[dominant]
    tr = NCU_TRAFFIC.get(kname)
    src = {"k_render_bwd": "render_bwd.cu", "k_render_bwd_pk": "render_bwd.cu",
           "k_render_fwd": "render_fwd.cu", "k_render_fwd_pk": "render_fwd.cu"}.get(kname)
    traffic = (tr["bytes_per_launch"] if tr and src and tr.get("src_sha") == src_sha(src)
               and tr.get("tuning") == trainer_tuning_key else None)
    if sr["bound"] == "alu":
        roof = {"bound": "alu", "achieved": sr["achieved"], "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": sr["frac"], "traffic": traffic, "kernel": kname,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz",
                "work": (f"{FLOP_PER_PAIR[dominant]:.0f} FLOP x {mean_pairs:.4g} pixel-splat pairs per launch"
                         if dominant in FLOP_PER_PAIR else "algorithmic FLOP of the stage")}
    else:
        roof = {"bound": "hbm", "achieved": sr["achieved"], "peak": hbm or FALLBACK_HBM_GBS, "unit": "GB/s",
                "frac": sr["frac"], "traffic": traffic, "kernel": kname,
                "peak_source": "measured" if hbm else "fallback", "work": "algorithmic bytes of the stage"}
    value = job_rate(world, args.steps, elapsed)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
            "launch": ("eager" if graphs is None else
                       f"one CUDA graph per view ({len(cams)}, Trainer.capture), replayed round robin"),
            "eager_ms_per_step": eager_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {**config_of(args), "binning": ("counting, load-balanced column walk" if counting else
                                                      "radix, load-balanced key write" if trainer.load_balanced
                                                      else "radix, sequential key write"),
                       "bucket": trainer.slot_for([cams[0]]).plan.tuning["bucket"],
                       "bwd_warps": trainer.slot_for([cams[0]]).plan.tuning["bwd_warps"],
                       "bwd_chains": trainer.slot_for([cams[0]]).plan.tuning["bwd_chains"],
                       "fwd_pixels": trainer.slot_for([cams[0]]).plan.tuning["fwd_pixels"],
                       "autotune_ms_per_step": trainer.autotune_table},
            "clocks": clocks, "e2e": e2e,
            "gpu_launches": kernels_per_step(trainer, [(args.width, args.height)]) * args.steps,
            "roofline": roof,
            "stages_ms": stage_ms,
            "stages_roofline": stages_roof,
            "work": {"instances_max": worst, "instances_last": st2["n_instances"],
                     "buckets_last": st2["n_buckets"], "pairs_per_view": mean_pairs},
            "peaks": {"hbm_gbs": hbm or FALLBACK_HBM_GBS, "hbm_source": "measured" if hbm else "fallback",
                      "fp32_tflops": FP32_PEAK_TFLOPS}}
    if world == 1 and not (args.no_batched and args.no_ng):
        del trainer
        torch.cuda.empty_cache()
    if world == 1 and not args.no_batched:
        line["batched_graph"] = run_batched(args, dev, args.n, args.batched_steps)
        torch.cuda.empty_cache()
    if world == 1 and not args.no_ng:
        ng = run_ng(args, dev, max(1, args.n // 10), cams, targets_d, args.warmup, args.steps, lb, tuning)
        ng["vs_explicit_same_protocol"] = {
            "explicit_steps_per_s": 1e3 / eager_step_ms, "neural_steps_per_s": ng["steps_per_s"],
            "timing": "both eager, CUDA events from each step's first stage to its last, averaged over the "
                      "timed steps (the headline value replays graphs instead)",
            "explicit_instances_per_view": st2["n_instances"], "explicit_pairs_per_view": mean_pairs,
            "note": "both from their own initial state, the same warm-up and timed steps on the same views and "
                    "targets; per-step work differs (children whose decoded opacity is <= 0 reach no tile)"}
        torch.cuda.empty_cache()
        fz = run_ng(args, dev, max(1, args.n // 10), cams, targets_d, args.warmup, args.steps, lb, tuning,
                    fused_decode=True)
        ng["fused_decode_preprocess"] = {
            "steps_per_s": fz["steps_per_s"], "ms_per_step": fz["ms_per_step"], "stages_ms": fz["stages_ms"],
            "note": "decode and the children's preprocess in one launch (gs_ng_decode_preprocess), the same "
                    "protocol; its 'decode' stage holds both, 'preprocess' is empty"}
        line["neural_gaussians"] = ng
        torch.cuda.empty_cache()
    if world == 1 and not args.no_pose:
        line["pose_refinement"] = run_pose_overhead(args, dev, scene, cams, targets_d, lb, tuning,
                                                      max(60, args.steps // 3))
        torch.cuda.empty_cache()
    if world == 1 and not args.no_visible_adam:
        line["visible_adam"] = run_visible_adam(args, dev, scene, lb, tuning, max(60, args.steps // 3))
    if world == 1 and not args.no_cpu_baseline:
        n_threads = os.cpu_count() or 1
        nx, ny, _, _ = window_cells(args.width, args.height)
        # the reference arm's first 40 steps: every cell once, views s mod 16
        plan = sample_plan(args.width, args.height, len(cams), range(nx * ny))
        tscene = synth.scene_clustered(args.n, seed=1, sh_degree=3)
        groups = []
        for v in sorted({v for v, _ in plan}):
            groups.append((cams[v], oracle_records(scene, cams[v]), oracle_records(tscene, cams[v]),
                           [w for vv, w in plan if vv == v]))
        est, detail = oracle_sample(scene, groups, cams[0], pre_sample=BASELINE_PRE_SAMPLE, n_threads=n_threads)
        line["cpu_baseline"] = {"value": 1.0 / est, "unit": UNIT, "cores": n_threads, "kind": "oracle",
                                "sample": f"preprocess fwd+bwd and Adam on {BASELINE_PRE_SAMPLE} random Gaussians "
                                          f"(x N/{BASELINE_PRE_SAMPLE}, view 0); blend fwd + loss + per-pixel bwd "
                                          f"on {nx * ny} seeded {WINDOW}x{WINDOW} windows, window s in cell "
                                          f"7 s mod {nx * ny} of a {nx}x{ny} grid over view s mod {len(cams)} "
                                          f"(every cell once; the reference arm's first {nx * ny} steps), "
                                          f"x H*W/({nx * ny}*{WINDOW * WINDOW}); float64",
                                "detail": detail}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ batched graph step

def run_batched(args, dev, n: int, steps: int, warmup: int = 3) -> dict:
    """8 views of uneven resolution per step (3 x 960x540, 3 x 1280x720,
    2 x 1920x1080 from the ring), launch shapes from the autotuner, the whole
    step captured in one CUDA graph per batch; two batches alternate.
    Compared with the same batch run eagerly and with the same 8 views as 8
    sequential single-view steps."""
    import torch

    import synth
    from paper_2601_19489_gb300 import api
    from paper_2601_19489_gb300.autotune import TUNED, autotune
    from paper_2601_19489_gb300.trainer import Trainer

    scene = synth.scene_clustered(n, seed=0, sh_degree=3)
    batches = [synth.mixed_ring_cameras(8, seed=s) for s in (0, 1)]
    targets = [torch.cat(render_targets(n, cams, dev)) for cams in batches]
    params = api.Gaussians.from_scene(scene, device=dev)
    best, table = autotune(params, batches, targets, lam=args.lam, device=dev)
    tr = Trainer(params, lam=args.lam, load_balanced=best["load_balanced"],
                 tuning={k: best[k] for k in TUNED}, device=dev)
    tr.ensure_capacity(batches)
    # eager batched steps (also the warm-up before capture)
    stream = torch.cuda.current_stream()

    def timed(fn, k):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(k):
            fn(i)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    for i in range(warmup):
        tr.step(batches[i % 2], targets[i % 2])
    t_eager = timed(lambda i: tr.step(batches[i % 2], targets[i % 2]), steps)
    graphs = [tr.capture(batches[b], targets[b]) for b in (0, 1)]
    for i in range(warmup):
        graphs[i % 2].replay()
    with ClockSampler(dev.index or 0) as clk:
        t_graph = timed(lambda i: graphs[i % 2].replay(), steps)
    st = tr.slot_for(batches[0]).plan.status()
    if st["rc"] != 0:
        raise RuntimeError(f"device status after the batched steps: {st}")
    # the same views one at a time (single-view plans, eager)
    singles = [[c] for cams in batches for c in cams]
    seq = Trainer(params, lam=args.lam, load_balanced=best["load_balanced"],
                  tuning={k: best[k] for k in TUNED}, device=dev)
    seq.ensure_capacity(singles)
    offs = []
    for b, cams in enumerate(batches):
        o = 0
        for c in cams:
            offs.append((b, o, 3 * c.width * c.height))
            o += 3 * c.width * c.height
    single_t = [targets[b][o:o + k] for (b, o, k) in offs]
    for i in range(len(singles)):
        seq.step(singles[i], single_t[i])
    t_seq = timed(lambda i: seq.step(singles[i % 16], single_t[i % 16]), 8 * steps)
    views = 8 * steps
    small = graph_vs_eager_small(args, dev, steps)
    return {"gaussians": n, "views_per_step": 8,
            "views": "3 x 960x540, 3 x 1280x720, 2 x 1920x1080 ring views; two batches alternate",
            "graph_steps_per_s": steps / t_graph, "graph_views_per_s": views / t_graph,
            "eager_batched_views_per_s": views / t_eager, "sequential_views_per_s": views / t_seq,
            "graph_ms_per_step": 1e3 * t_graph / steps, "sequential_ms_per_8_views": 1e3 * t_seq / steps,
            "tuning": best, "autotune_ms_per_step": table, "clocks": clk.summary(),
            "instances_last": st["n_instances"], "launch_bound_case": small}


def graph_vs_eager_small(args, dev, steps: int) -> dict:
    """Where a CUDA graph pays: a launch-bound step (8 views of 320x180, 20k
    Gaussians; about 40 launches of a few microseconds each), the same batch
    eager and replayed from a graph."""
    import torch

    import synth
    from paper_2601_19489_gb300 import api
    from paper_2601_19489_gb300.trainer import Trainer

    n = 20000
    cams = synth.ring_cameras(8, 320, 180)
    tgt = torch.cat(render_targets(n, cams, dev))
    tr = Trainer(api.Gaussians.from_scene(synth.scene_clustered(n, seed=0, sh_degree=3), device=dev),
                 lam=args.lam, device=dev)
    tr.ensure_capacity([cams])
    for _ in range(3):
        tr.step(cams, tgt)
    stream = torch.cuda.current_stream()

    def timed(fn, k):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    k = max(50, 4 * steps)
    t_eager = timed(lambda: tr.step(cams, tgt), k)
    g = tr.capture(cams, tgt)
    for _ in range(3):
        g.replay()
    t_graph = timed(g.replay, k)
    return {"gaussians": n, "views": "8 ring views 320x180", "eager_ms_per_step": 1e3 * t_eager / k,
            "graph_ms_per_step": 1e3 * t_graph / k, "graph_speedup": t_eager / t_graph}


def run_ng(args, dev, n_anchors: int, cams, targets, warmup: int, steps: int, lb: bool = True,
           tuning: dict | None = None, fused_decode: bool = False) -> dict:
    """Neural-Gaussian step: n_anchors anchors subsampled from the clustered
    scene's points, 10 children each, the same ring views and targets as the
    headline, one view per step (decode, splat, loss, backward, decoder
    backward, Adam on features, anchor scales and MLP).  Timed over the
    headline's own protocol (the same warm-up and timed step counts from the
    method's initial state, the same view order), with the work per step
    (tile instances, pixel-splat pairs up to each pixel's last contributor)
    reported beside the time, since a decoder in training changes how many of
    its children reach the blend.  Binning and launch shapes are the
    headline's (lb, tuning).  fused_decode: the decode and the children's
    preprocess in one launch (its time is the decode stage's)."""
    import torch

    import synth
    from paper_2601_19489_gb300 import _lib as L
    from paper_2601_19489_gb300 import api
    from paper_2601_19489_gb300.trainer import NgTrainer

    pts = synth.scene_clustered(args.n, seed=0, sh_degree=0).means
    d = synth.ng_anchors(pts, n_anchors, seed=0)
    tr = NgTrainer(api.NgParams.from_dict(d, device=dev), args.width, args.height, lam=args.lam,
                   load_balanced=lb, tuning=tuning, fused_decode=fused_decode, device=dev)
    tr.ensure_capacity(cams)
    for s in range(warmup):
        tr.step(cams[s % len(cams)], targets[s % len(cams)])
    n_st = len(tr.STAGES)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(n_st + 1)] for _ in range(steps)]
    torch.cuda.synchronize()
    inst = []
    for s in range(steps):
        v = (warmup + s) % len(cams)
        tr.step(cams[v], targets[v], events=evs[s])
    torch.cuda.synchronize()
    if tr.status() != 0 or tr.plan.status()["rc"] != 0:
        raise RuntimeError("device status after the neural-Gaussian steps")
    total = sum(evs[s][0].elapsed_time(evs[s][n_st]) for s in range(steps)) / steps
    stage_ms = {name: float(np.mean([evs[s][i].elapsed_time(evs[s][i + 1]) for s in range(steps)]))
                for i, name in enumerate(tr.STAGES)}
    # the work of the trained state, on the views of the timed steps
    pairs = []
    for s in range(min(steps, len(cams))):
        v = (warmup + s) % len(cams)
        tr.forward(cams[v])
        inst.append(tr.plan.status()["n_instances"])
        nc = tr.plan.view(L.GS_WS_N_CONTRIB, torch.int32)[: args.width * args.height]
        pairs.append(float(nc.double().sum().item()))
    return {"anchors": n_anchors, "children": 10 * n_anchors, "steps_per_s": 1e3 / total, "ms_per_step": total,
            "warmup": warmup, "steps": steps, "stages_ms": stage_ms, "loss_last": tr.loss.item(),
            "instances_per_view": float(np.mean(inst)), "pairs_per_view": float(np.mean(pairs)),
            "decoder": "x = [feature 32, view dir 3] -> 32 ReLU -> 140 = 10 children x 14; bf16 tcgen05 MMAs"}


def run_pose_overhead(args, dev, scene, cams, targets, lb, tuning, steps: int, warmup: int = 5) -> dict:
    """The headline step with and without the global pose refinement of
    Sec. 2.5 (gradient accumulated by every step's preprocess backward, the
    correction updated every 300 steps), same launch shapes, eager."""
    import torch

    import synth
    from paper_2601_19489_gb300 import api
    from paper_2601_19489_gb300.trainer import Trainer

    out = {}
    for name, pose in (("off", None), ("on", {"every": 300})):
        tr = Trainer(api.Gaussians.from_scene(scene, device=dev), args.width, args.height, lam=args.lam,
                     load_balanced=lb, tuning=tuning, pose=pose, device=dev)
        tr.ensure_capacity(cams)
        for s in range(warmup):
            tr.step(cams[s % len(cams)], targets[s % len(cams)])
        n_st = len(tr.STAGES)
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(n_st + 1)] for _ in range(steps)]
        torch.cuda.synchronize()
        for s in range(steps):
            v = (warmup + s) % len(cams)
            tr.step(cams[v], targets[v], events=evs[s])
        torch.cuda.synchronize()
        if tr.plan.status()["rc"] != 0:
            raise RuntimeError(f"device status after the pose-{name} steps")
        ms = float(np.mean([evs[s][0].elapsed_time(evs[s][n_st]) for s in range(steps)]))
        out[name] = {"steps_per_s": 1e3 / ms, "ms_per_step": ms,
                     "preprocess_ms": float(np.mean([evs[s][0].elapsed_time(evs[s][1]) for s in range(steps)])),
                     "preprocess_bwd_adam_ms": float(np.mean([evs[s][n_st - 1].elapsed_time(evs[s][n_st])
                                                              for s in range(steps)]))}
        del tr
        torch.cuda.empty_cache()
    out["overhead_pct"] = 100.0 * (out["on"]["ms_per_step"] / out["off"]["ms_per_step"] - 1.0)
    out["note"] = ("pose on: camera composition kernel + pose-gradient terms and warp sums in the fused "
                   "preprocess backward + Adam; the 1-block pose update every 300 steps")
    return out


def run_visible_adam(args, dev, scene, lb, tuning, steps: int, warmup: int = 5, radius: float = 2.2) -> dict:
    """Dense against visible-only (sparse) Adam in the fused preprocess
    backward, on the headline scene seen from a closer ring (radius 2.2
    instead of 4), where part of the scene is outside each view."""
    import torch

    import synth
    from paper_2601_19489_gb300 import _lib as L
    from paper_2601_19489_gb300 import api
    from paper_2601_19489_gb300.trainer import Trainer

    cams = synth.ring_cameras(args.views, args.width, args.height, radius=radius)
    targets = render_targets(scene.n, cams, dev)
    out = {"ring_radius": radius}
    for name, vis in (("dense", False), ("visible_only", True)):
        tr = Trainer(api.Gaussians.from_scene(scene, device=dev), args.width, args.height, lam=args.lam,
                     load_balanced=lb, tuning=tuning, visible_adam=vis, device=dev)
        tr.ensure_capacity(cams)
        if not vis:
            frac = []
            for c in cams:
                tr.forward([c])
                frac.append(float((tr.plan.view(L.GS_WS_TILES_TOUCHED, torch.int32) > 0).float().mean().item()))
            out["visible_fraction"] = float(np.mean(frac))
        for s in range(warmup):
            tr.step(cams[s % len(cams)], targets[s % len(cams)])
        n_st = len(tr.STAGES)
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(n_st + 1)] for _ in range(steps)]
        torch.cuda.synchronize()
        for s in range(steps):
            v = (warmup + s) % len(cams)
            tr.step(cams[v], targets[v], events=evs[s])
        torch.cuda.synchronize()
        if tr.plan.status()["rc"] != 0:
            raise RuntimeError(f"device status after the {name} steps")
        ms = float(np.mean([evs[s][0].elapsed_time(evs[s][n_st]) for s in range(steps)]))
        out[name] = {"steps_per_s": 1e3 / ms, "ms_per_step": ms,
                     "preprocess_bwd_adam_ms": float(np.mean([evs[s][n_st - 1].elapsed_time(evs[s][n_st])
                                                              for s in range(steps)]))}
        del tr
        torch.cuda.empty_cache()
    out["adam_stage_speedup"] = out["dense"]["preprocess_bwd_adam_ms"] / out["visible_only"]["preprocess_bwd_adam_ms"]
    return out


def run_batched_only(args):
    import torch

    from paper_2601_19489_gb300 import _lib as L

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    L.load()
    ns = [int(float(x)) for x in args.batched_n.split(",") if x] or [args.n]
    for n in ns:
        r = run_batched(args, dev, n, args.batched_steps)
        line = {"metric": "train views/s (8-view batched step, CUDA graph)", "value": r["graph_views_per_s"],
                "unit": "views/s", "n_gpus": 1, "steps": args.batched_steps, "warmup": 3,
                "ms_per_step": r["graph_ms_per_step"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"clustered {n} Gaussians SH3, 8 mixed-resolution ring views per step"},
                "batched_graph": r}
        print(json.dumps(line), flush=True)


# ------------------------------------------------------------ timed reconstruction

def run_recon(args):
    """300k-Gaussian clustered ground truth (SH 3) seen by 200 orbit views at
    1600x1060; every 10th view held out; training starts from 50k jittered
    ground-truth points with noisy colour and runs for the budget per
    method.  The views' colour and disparity are rendered by the CUDA
    forward of the ground truth (a workload, not a parity reference)."""
    import torch

    import synth
    from paper_2601_19489_gb300 import _lib as L
    from paper_2601_19489_gb300 import api
    from paper_2601_19489_gb300.recon import reconstruct, render_views
    from paper_2601_19489_gb300.trainer import Trainer

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    L.load()
    W, H = 1600, 1060
    gt = synth.scene_clustered(300000, seed=100, sh_degree=3)
    cams = synth.orbit_cameras(200, W, H)
    gt_tr = Trainer(api.Gaussians.from_scene(gt, device=dev), W, H, device=dev)
    gt_tr.ensure_capacity([[c] for c in cams])
    views = render_views(gt_tr, cams)
    del gt_tr
    torch.cuda.empty_cache()
    ev = [i for i in range(len(cams)) if i % 10 == 0]
    tr_ix = [i for i in range(len(cams)) if i % 10 != 0]
    init = synth.recon_init(gt, 50000, seed=1)
    err = None
    given = cams
    if args.recon_pose_error:
        rot, trans = (float(x) for x in args.recon_pose_error.split(","))
        err = synth.camera_pose_error(rot, trans, seed=7)
        given = synth.with_pose_error(cams, *err)
    results = {}
    with ClockSampler(0) as clk:
        for m in [x for x in args.recon_methods.split(",") if x]:
            # "<method>@true": on the true poses; "batched_graph~fixed": Adam's
            # betas unscaled by the batch
            method, true_poses = m.split("@")[0].split("~")[0], m.endswith("@true")
            cs = cams if true_poses else given
            results[m] = reconstruct(method, init, [cs[i] for i in tr_ix], [views[i][0] for i in tr_ix],
                                     [views[i][1] for i in tr_ix], [cs[i] for i in ev], [views[i][0] for i in ev],
                                     budget_s=args.recon_budget, lam=args.lam,
                                     densify_rules={"tau_plus": args.densify_tau_plus}, max_gaussians=600000,
                                     batch_lr_scale=args.recon_batch_lr_scale,
                                     batch_betas="fixed" if "~fixed" in m else "scaled", device=dev)
            if err is not None and not true_poses:
                results[m]["pose_error"] = pose_error_report(gt.means, cams, given, results[m].get("pose_correction"))
            torch.cuda.empty_cache()
    from paper_2601_19489_gb300.recon import time_to_psnr

    head = results.get("plain") or next(iter(results.values()))
    line = {"metric": f"held-out PSNR after {args.recon_budget:g} s of training", "value": head["psnr_final"],
            "unit": "dB", "n_gpus": 1, "higher_is_better": True, "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "method": head["method"],
            "vs_plain_db": {m: r["psnr_final"] - head["psnr_final"] for m, r in results.items()},
            # wall time (training seconds) each method takes to reach the
            # head method's final held-out PSNR (None: not within the budget)
            "time_to_plain_psnr_s": {m: time_to_psnr(r["curve"], head["psnr_final"]) for m, r in results.items()},
            "config": {"workload": "300k clustered Gaussians SH3 ground truth, 200 orbit views 1600x1060 "
                                   "(20 held out), start from 50k noisy points",
                       "camera_pose_error": args.recon_pose_error or None},
            "clocks": clk.summary(), "results": results}
    print(json.dumps(line), flush=True)


def pose_error_report(means, true_cams, given_cams, corr) -> dict:
    """How far the views a method trained on are from the true cameras: the
    residual camera-side transform (correction o error) as an angle and a
    translation length, and the mean image distance of the ground-truth
    Gaussian centres seen through the true and the (corrected) given cameras."""
    R = np.eye(3) if corr is None else np.asarray(corr["R"])
    t = np.zeros(3) if corr is None else np.asarray(corr["t"])
    p = np.asarray(means, dtype=np.float64)[::50]
    px, ang, dist = [], [], []
    for c0, c1 in zip(true_cams, given_cams):
        Rg, tg = R @ c1.R, R @ c1.t + t
        Rd = Rg @ c0.R.T  # residual: world->camera of the used view after the true one's inverse
        td = tg - Rd @ c0.t
        ang.append(float(np.arccos(np.clip((np.trace(Rd) - 1.0) / 2.0, -1.0, 1.0))))
        dist.append(float(np.linalg.norm(td)))
        pcs = [p @ Rc.T + tc for Rc, tc in ((c0.R, c0.t), (Rg, tg))]
        keep = (pcs[0][:, 2] > 0.5) & (pcs[1][:, 2] > 0.5)
        uv = [np.stack([c0.fx * q[keep, 0] / q[keep, 2], c0.fy * q[keep, 1] / q[keep, 2]], 1) for q in pcs]
        px.append(float(np.linalg.norm(uv[0] - uv[1], axis=1).mean()))
    return {"residual_rot_rad": float(np.mean(ang)), "residual_trans": float(np.mean(dist)),
            "reprojection_px": float(np.mean(px))}


# ------------------------------------------------------------ Tab. 1 ablation

def run_ablation(args, steps: int = 200, warmup: int = 10):
    """The paper's speed ablation (Tab. 1) on the headline workload: per-pixel
    backward + 3-sigma tile box + sequential key write (the classic step),
    then the per-Gaussian backward (B), then the SnugBox (F) with the
    sequential (Sq) and the load-balanced (LB) key write.  Train steps/s and
    the time 30,000 iterations would take."""
    import torch

    import synth
    from paper_2601_19489_gb300 import _lib as L
    from paper_2601_19489_gb300 import api
    from paper_2601_19489_gb300.trainer import Trainer

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    L.load()
    scene, cams = workload(args)
    targets = render_targets(args.n, cams, dev)
    shape = {"bucket": 64, "bwd_warps": 1, "bwd_chains": 0}
    configs = [("3DGS (per-pixel backward, 3-sigma box, Sq)", False, {"bwd_per_pixel": 1, "bbox_3sigma": 1}),
               ("w/ B", False, {**shape, "bbox_3sigma": 1}),
               ("w/ B & F & Sq", False, dict(shape)),
               ("w/ B & F & LB (counting binning)", True, dict(shape)),
               ("w/ B & F & LB (key write + tile sort; not in Tab. 1)", True, {**shape, "bin_radix": 1}),
               ("w/ F & LB, per-pixel backward (not in Tab. 1)", True, {"bwd_per_pixel": 1})]
    rows = []
    with ClockSampler(0) as clk:
        for name, lb, tuning in configs:
            tr = Trainer(api.Gaussians.from_scene(scene, device=dev), args.width, args.height, lam=args.lam,
                         load_balanced=lb, tuning=tuning, device=dev)
            tr.ensure_capacity(cams)
            for s in range(warmup):
                tr.step(cams[s % len(cams)], targets[s % len(cams)])
            n_st = len(tr.STAGES)
            evs = [[torch.cuda.Event(enable_timing=True) for _ in range(n_st + 1)] for _ in range(steps)]
            torch.cuda.synchronize()
            for s in range(steps):
                v = (warmup + s) % len(cams)
                tr.step(cams[v], targets[v], events=evs[s])
            torch.cuda.synchronize()
            st = tr.plan.status()
            if st["rc"] != 0:
                raise RuntimeError(f"device status in {name}: {st}")
            ms = float(np.mean([evs[s][0].elapsed_time(evs[s][n_st]) for s in range(steps)]))
            stage = {k: float(np.mean([evs[s][i].elapsed_time(evs[s][i + 1]) for s in range(steps)]))
                     for i, k in enumerate(tr.STAGES)}
            rows.append({"config": name, "steps_per_s": 1e3 / ms, "ms_per_step": ms,
                         "seconds_per_30k_iterations": 30.0 * ms, "instances": st["n_instances"],
                         "stages_ms": stage})
            del tr
            torch.cuda.empty_cache()
    base = rows[0]["ms_per_step"]
    for r in rows:
        r["speedup_vs_3dgs"] = base / r["ms_per_step"]
    line = {"metric": "train steps/s, Tab. 1 ablation", "value": rows[3]["steps_per_s"], "unit": "steps/s",
            "n_gpus": 1, "steps": steps, "warmup": warmup, "higher_is_better": True, "vs_baseline": None,
            "dtype": "f32", "data": "synthetic", "config": config_of(args), "clocks": clk.summary(),
            "ablation": rows}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.workload == "ablation":
        run_ablation(args)
        return
    if args.workload == "batched":
        run_batched_only(args)
        return
    if args.workload == "recon60":
        run_recon(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch

        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        torch.distributed.init_process_group("nccl")
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)
    if world > 1 and args.impl == "ours":
        import torch

        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
