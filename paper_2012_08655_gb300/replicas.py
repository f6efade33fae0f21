"""Replica parallelism (one process per GPU, no data-path collective).

Frames are independent given their input, so N GPUs run N independent
replicas of the path. The host assigns frames to ranks by estimated cost
(longest-processing-time greedy, deterministic on every rank), and the only
communication is the max-over-ranks of the measured time.
"""
from __future__ import annotations

from typing import Sequence


def frame_cost(width: int, height: int, channels: int, rmax: int, block: int = 32) -> float:
    """Rough FMA count of one frame at its largest radius (for assignment only)."""
    nb = ((width + block - 1) // block) * ((height + block - 1) // block)
    return float(nb * channels * (2 * rmax + 1) * block * (2 * block + 2 * rmax))


def shard_frames(costs: Sequence[float], world: int, rank: int) -> list[int]:
    """Indices of the frames rank `rank` renders: greedy LPT over `world` ranks
    (largest cost first, ties by index), identical on every rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    load = [0.0] * world
    mine = []
    for i in sorted(range(len(costs)), key=lambda j: (-costs[j], j)):
        r = min(range(world), key=lambda q: (load[q], q))
        load[r] += costs[i]
        if r == rank:
            mine.append(i)
    return sorted(mine)


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of `value` over the default process group (identity when
    torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
