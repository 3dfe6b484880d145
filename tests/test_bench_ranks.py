"""The benchmark's multi-rank host logic on CPU with the gloo backend
(world size 2): the timed region is the slowest rank's, the job's throughput
counts every rank's steps, and under torchrun the reference arm prints one
line from rank 0 while the other ranks exit without work."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sys.path.insert(0, ROOT)
        import bench

        elapsed = 1.0 + 2.5 * rank  # this rank's timed region, seconds
        worst = bench.max_over_ranks(elapsed, world, "cpu")
        rate = bench.job_rate(world, 300, worst)
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump({"worst": worst, "rate": rate}, f)
    finally:
        dist.destroy_process_group()


def test_slowest_rank_sets_the_time_and_all_steps_count(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        got = json.load(open(tmp_path / f"r{r}.json"))
        assert got["worst"] == 3.5
        assert got["rate"] == pytest.approx(world * 300 / 3.5)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(2.25, 1, "cpu") == 2.25
    assert bench.job_rate(1, 100, 0.5) == 200.0


@pytest.mark.slow
def test_reference_arm_prints_once_under_torchrun():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--gaussians", "16384", "--views", "2",
           "--width", "128", "--height", "96"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["value"] == line["value"] and line["cpu_baseline"]["kind"] == "oracle"
    # the rest of the one-line contract
    for key in ("metric", "unit", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config"):
        assert key in line, key
    assert line["steps"] == 1 and line["higher_is_better"] is True and line["vs_baseline"] is None
    assert "workload" in line["config"] and line["data"] == "synthetic"
    assert line["e2e"]["unit"] == line["unit"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    cb = line["cpu_baseline"]
    assert cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
