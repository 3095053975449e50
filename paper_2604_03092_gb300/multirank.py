"""Host-side logic of the multi-GPU (weak-scaling) run.

The refinement step shards by submap: every rank owns an independent submap
(its own surfels, keyframes and poses) and renders it forward and backward
on its own GPU.  Nothing on the data path is exchanged between ranks; the
only collectives are the timing reductions below (a barrier around the
timed region, the maximum of the per-rank times, and the sum of the views
the ranks rendered), which run after the timed region ends.

The functions take the process group's backend as it is (NCCL on GPUs, gloo
in the CPU tests), so the same code is exercised in both.
"""
from __future__ import annotations

import os
from dataclasses import dataclass
from typing import Optional


@dataclass(frozen=True)
class RankInfo:
    rank: int
    world: int
    local: int


def rank_info(env: Optional[dict] = None) -> RankInfo:
    """Rank, world size and local rank from the torchrun environment (1 rank without it)."""
    e = os.environ if env is None else env
    world = int(e.get("WORLD_SIZE", "1"))
    rank = int(e.get("RANK", "0"))
    local = int(e.get("LOCAL_RANK", str(rank)))
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"bad rank {rank} of world size {world}")
    return RankInfo(rank, world, local)


def submap_seed_offset(rank: int) -> int:
    """Seed offset of the submap a rank owns: each rank renders a different submap."""
    return rank


def _reduce(x: float, op, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x: float, device=None) -> float:
    """Largest value of x over all ranks (the job's time is its slowest rank's)."""
    import torch.distributed as dist
    return _reduce(x, dist.ReduceOp.MAX, device)


def sum_over_ranks(x: float, device=None) -> float:
    """Sum of x over all ranks (units of work the whole job processed)."""
    import torch.distributed as dist
    return _reduce(x, dist.ReduceOp.SUM, device)


def barrier() -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def whole_job_rate(units_all_ranks: float, max_elapsed_ms: float) -> float:
    """Throughput of the whole job: all ranks' units over the slowest rank's time."""
    if max_elapsed_ms <= 0.0:
        raise ValueError("elapsed time must be positive")
    return units_all_ranks / (max_elapsed_ms / 1e3)
