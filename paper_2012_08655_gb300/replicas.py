"""Replica parallelism (one process per GPU, no data-path collective).

Frames are independent given their input, so N GPUs run N independent
replicas of the path. The host assigns frames to ranks by estimated cost
(longest-processing-time greedy, deterministic on every rank) or, for a
request stream, whole streams to ranks (a stream's fixation walk stays on
one GPU). The only communication is on the measurement path: the
max-over-ranks of the measured time and the gathering of per-request
latencies to rank 0.
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


def frame_rmax(width: int, height: int, fix_x: float, fix_y: float, sigma0: float, k: float,
               block: int = 32) -> int:
    """Radius bound of a frame under the linear law: ceil(3 sigma) at the
    block centre farthest from the fixation (for cost estimates only)."""
    import math
    cx = [0.5 * block, (math.ceil(width / block) - 0.5) * block]
    cy = [0.5 * block, (math.ceil(height / block) - 0.5) * block]
    e = max(math.hypot(x - fix_x, y - fix_y) for x in cx for y in cy)
    return int(math.ceil(3.0 * (sigma0 + k * e)))


def shard_streams(n_streams: int, world: int, rank: int) -> list[int]:
    """Stream ids rank `rank` serves: stream s goes to rank s mod world."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    return [s for s in range(n_streams) if s % world == rank]


def gather_to_rank0(obj):
    """Every rank's `obj` as a list on rank 0 (None on the other ranks); [obj]
    when torch.distributed is not initialised."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [obj]
    got = [None] * dist.get_world_size()
    dist.all_gather_object(got, obj)
    return got if dist.get_rank() == 0 else None


def merged_percentiles(parts, qs=(50, 99)):
    """Percentiles of the union of several ranks' latency lists."""
    import numpy as np
    allv = np.concatenate([np.asarray(p, dtype=np.float64) for p in parts if len(p)])
    return [float(np.percentile(allv, q)) for q in qs]
