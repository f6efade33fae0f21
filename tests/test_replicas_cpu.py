"""World-size-2 CPU (gloo) test of the replica host logic: every frame is
assigned to exactly one rank, the assignment is balanced, and the timing
reduction takes the maximum over ranks."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2012_08655_gb300.replicas import frame_cost, max_over_ranks, shard_frames


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, costs, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard_frames(costs, world, rank)
    got = [None] * world
    dist.all_gather_object(got, mine)
    m = max_over_ranks(10.0 * (rank + 1))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got, m))


def test_two_rank_sharding_and_max():
    from paper_2012_08655_gb300 import workloads as wl
    sizes = wl.MIXED_SIZES
    costs = [frame_cost(w, h, 3, 60) for (w, h) in sizes]
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, costs, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, m in res:
        assert m == 20.0
        flat = sorted(i for part in got for i in part)
        assert flat == list(range(len(sizes)))
        loads = [sum(costs[i] for i in part) for part in got]
        assert max(loads) - min(loads) <= max(costs)


def test_single_process_identity():
    assert max_over_ranks(3.5) == 3.5
    assert shard_frames([1.0, 2.0, 3.0], 1, 0) == [0, 1, 2]
