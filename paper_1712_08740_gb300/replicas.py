"""Replica bookkeeping for runs on several GPUs of one node.

The solver shards as independent solves (every rank runs its own solves on
its own GPU; there is no data exchange between ranks). What the ranks share
is only the measurement: a barrier before and after the timed region, the
maximum of the per-rank times, and the whole-job rate = the units all ranks
processed divided by that maximum. These helpers hold that logic so that it
runs the same under NCCL (one rank per GPU) and under gloo on CPU.
"""
from __future__ import annotations

import os
from dataclasses import dataclass


@dataclass(frozen=True)
class RankEnv:
    world: int
    rank: int
    local: int


def rank_env(environ=None) -> RankEnv:
    """WORLD_SIZE / RANK / LOCAL_RANK as set by torch.distributed.run (defaults: one rank)."""
    e = os.environ if environ is None else environ
    world = int(e.get("WORLD_SIZE", "1"))
    rank = int(e.get("RANK", "0"))
    local = int(e.get("LOCAL_RANK", str(rank)))
    if world < 1 or not (0 <= rank < world) or local < 0:
        raise ValueError(f"bad rank environment: world={world} rank={rank} local={local}")
    return RankEnv(world, rank, local)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The maximum of `value` over all ranks of the default process group
    (the value itself when there is no group)."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, slowest_ms: float) -> float:
    """Units per second of the whole job: every rank processed `units_per_rank`
    units, the job took as long as its slowest rank."""
    if slowest_ms <= 0.0:
        raise ValueError("timed region must be positive")
    return world * units_per_rank / (slowest_ms / 1e3)
