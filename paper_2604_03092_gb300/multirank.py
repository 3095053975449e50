"""Host-side logic of the multi-GPU (weak-scaling) run.

The refinement step shards by submap: every rank owns an independent submap
(its own surfels, keyframes and poses) and renders it forward and backward
on its own GPU.  Nothing on the data path is exchanged between ranks; the
only collectives are the timing reductions below (a barrier around the
timed region, the maximum of the per-rank times, and the sum of the views
the ranks rendered), which run after the timed region ends.

A second partition splits the views of ONE submap across ranks: every rank
holds all of the submap's surfels, renders its own contiguous share of the
views forward and backward, and the ranks then sum their surfel-parameter
gradients (one all-reduce of d_params [N, 13]: means 3, scales 2, quats 4,
opacity 1, rgb 3); the per-view pose gradients stay with the rank that owns
the view.  `view_shard` and `allreduce_surfel_grads` are that exchange.

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


def view_shard(n_views: int, rank: int, world: int) -> range:
    """The views of one submap that `rank` renders when its views are split
    across `world` ranks: contiguous, sizes differing by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"bad rank {rank} of world size {world}")
    q, r = divmod(int(n_views), world)
    lo = rank * q + min(rank, r)
    return range(lo, lo + q + (1 if rank < r else 0))


SURFEL_GRAD_FIELDS = (("means", 3), ("scales", 2), ("quats", 4), ("opacity", 1), ("rgb", 3))


def allreduce_surfel_grads(grads) -> None:
    """Sum, in place and over all ranks, the surfel-parameter gradients of
    ranks that rendered disjoint views of the same surfels: the five arrays
    (any object with tensor attributes means [N,3], scales [N,2], quats
    [N,4], opacity [N], rgb [N,3] of one dtype and device) are packed into
    one [N, 13] buffer, all-reduced with a sum, and unpacked.  The pose
    gradients are per view and are not exchanged.  A no-op on one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return
    parts = [getattr(grads, name).reshape(-1, k) for name, k in SURFEL_GRAD_FIELDS]
    n = parts[0].shape[0]
    if any(p.shape[0] != n for p in parts):
        raise ValueError("surfel gradient arrays disagree on the surfel count")
    flat = torch.cat(parts, 1).contiguous()
    dist.all_reduce(flat, op=dist.ReduceOp.SUM)
    col = 0
    for (name, k), p in zip(SURFEL_GRAD_FIELDS, parts):
        p.copy_(flat[:, col:col + k])
        col += k
