"""CPU, two processes over gloo: bench.py's bookkeeping for N > 1 replicas.

With N GPUs the benchmark runs N independent replicas, one process each,
with no collective on the data path.  The job's time is the slowest rank's,
taken by one max all-reduce, and its throughput counts the units of every
rank.  Only rank 0 prints.  The reference arm (the CPU oracle) runs on rank 0
alone; other ranks exit 0 without work.  These tests run the same helpers
with the gloo backend on the CPU.
"""
import multiprocessing as mp
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, loc = bench.dist_env()
    # rank r took 100 (r + 1) ms for 1000 units
    t, v = bench.job_time_and_value(100.0 * (rank + 1), 1000, w)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, w, r, loc, t, v))


def test_job_time_is_the_slowest_rank_and_value_counts_every_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=180) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert [p.exitcode for p in procs] == [0, 0]
    for rank, w, r, loc, t, v in res:
        assert (w, r, loc) == (2, rank, rank)
        assert t == 200.0                      # max over ranks, seen by both
        assert v == pytest.approx(2 * 1000 / 0.2)  # both ranks' units over the slowest time


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    t, v = bench.job_time_and_value(50.0, 1000, 1)
    assert (t, v) == (50.0, pytest.approx(1000 / 0.05))


def test_reference_arm_runs_on_rank_0_only():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert out.returncode == 0
    assert out.stdout.strip() == ""  # rank 1 prints nothing and does no work


def test_reference_arm_prints_one_contract_line():
    """Alone (rank 0), the reference arm times the FP64 oracle on a bounded
    sample of the same workload and prints one JSON line carrying the
    benchmark's keys, with no host-device traffic in its e2e record."""
    import json

    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "voxel-iters/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
