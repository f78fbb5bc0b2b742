"""The multi-rank host logic of the benchmark on CPU: two gloo ranks in spawned processes.

The path runs as independent replicas (every rank its own volume, no collective on the data
path); what crosses ranks is the timing: the step time is the slowest rank's (an all-reduce
MAX) and the job's throughput counts every rank's units over that time.  The reference arm
runs on rank 0 alone; the other ranks exit at once.
"""
import json
import multiprocessing as mp
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, local_ms, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = bench.max_over_ranks(local_ms[rank], dist, torch.device("cpu"))
        q.put((rank, ms, bench.job_rate(world, 1_000_000, ms)))
    finally:
        dist.destroy_process_group()


def test_step_time_is_the_slowest_rank_and_rate_counts_every_rank():
    world, local_ms = 2, [12.5, 20.0]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, local_ms, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, ms, rate in got:
        assert ms == max(local_ms)
        assert rate == pytest.approx(world * 1_000_000 / (max(local_ms) / 1e3))


def _reference_arm(rank: int, world: int) -> subprocess.CompletedProcess:
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
               MASTER_ADDR="127.0.0.1")
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", str(world),
                           "--workload", "cube64", "--steps", "1", "--warmup", "0"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_runs_on_rank_zero_only():
    other = _reference_arm(1, 2)
    assert other.returncode == 0 and other.stdout.strip() == ""
    first = _reference_arm(0, 2)
    assert first.returncode == 0, first.stderr[-2000:]
    lines = [l for l in first.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
