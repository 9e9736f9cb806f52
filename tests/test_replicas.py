"""Runs on several GPUs shard as independent solves (replicas): the ranks
share only the measurement. These tests run that host logic as two gloo
ranks on the CPU: the rank environment, the maximum of the per-rank times,
the whole-job rate, and the reference arm under torch.distributed.run (rank 0
alone runs and prints one line, the other rank exits 0 without work).
"""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1712_08740_gb300.replicas import (max_over_ranks, rank_env,  # noqa: E402
                                             whole_job_rate)


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_rank_env_defaults_and_checks():
    e = rank_env({})
    assert (e.world, e.rank, e.local) == (1, 0, 0)
    e = rank_env({"WORLD_SIZE": "4", "RANK": "3", "LOCAL_RANK": "3"})
    assert (e.world, e.rank, e.local) == (4, 3, 3)
    with pytest.raises(ValueError):
        rank_env({"WORLD_SIZE": "2", "RANK": "2"})
    with pytest.raises(ValueError):
        rank_env({"WORLD_SIZE": "0"})


def test_whole_job_rate():
    # two ranks, 30 solves each, the slower took 360 ms: 60 solves in 0.36 s
    assert whole_job_rate(30, 2, 360.0) == pytest.approx(60 / 0.36)
    assert whole_job_rate(30, 1, 360.0) == pytest.approx(30 / 0.36)
    with pytest.raises(ValueError):
        whole_job_rate(30, 2, 0.0)
    # without a process group the maximum is the value itself
    assert max_over_ranks(12.5) == 12.5


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # per-rank timed regions; the job's time is the slowest rank's
        local_ms = [240.0, 360.0][rank]
        dist.barrier()
        slowest = max_over_ranks(local_ms, dist, "cpu")
        dist.barrier()
        q.put((rank, slowest, whole_job_rate(30, world, slowest)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_rank():
    world, port = 2, free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    out = sorted(q.get(timeout=5) for _ in range(world))
    assert [r for r, _, _ in out] == [0, 1]
    for _, slowest, rate in out:
        assert slowest == 360.0
        assert rate == pytest.approx(60 / 0.36)


def test_reference_arm_under_torchrun_prints_once():
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0
