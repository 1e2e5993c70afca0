"""Host-side bookkeeping of independent replicas across ranks.

The fluctuating LB path shards into independent boxes (ensemble members)
that never exchange data, so running on N GPUs means N replica boxes, one per
rank, each with its own Philox replica id (counter word 2).  The only
collective is on the timing: a barrier around the timed region and the
maximum of the per-rank times, so the reported throughput is the work of all
ranks divided by the slowest rank's time (weak scaling).
"""
from __future__ import annotations

import os
from dataclasses import dataclass


@dataclass(frozen=True)
class RankInfo:
    rank: int
    world: int
    local: int


def rank_info(env=None) -> RankInfo:
    """RANK / WORLD_SIZE / LOCAL_RANK as torchrun sets them (defaults: one rank)."""
    env = os.environ if env is None else env
    return RankInfo(int(env.get("RANK", "0")), int(env.get("WORLD_SIZE", "1")), int(env.get("LOCAL_RANK", "0")))


def replica_id(rank: int, base: int = 0) -> int:
    """Philox replica id of the box a rank advances: distinct per rank."""
    if rank < 0:
        raise ValueError("rank must be >= 0")
    return base + rank


def max_over_ranks(value: float, dist=None, device: str = "cpu") -> float:
    """The maximum of `value` over all ranks of the default process group (or
    `value` itself without one)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_mlups(sites_per_rank: int, steps: int, world: int, max_seconds: float) -> float:
    """Whole-job site updates per second (in millions): every rank advanced
    sites_per_rank sites for `steps` steps; the job took the slowest rank's time."""
    if max_seconds <= 0:
        raise ValueError("time must be positive")
    return world * sites_per_rank * steps / max_seconds / 1e6
