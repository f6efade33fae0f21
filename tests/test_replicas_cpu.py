"""World-size-2 CPU (gloo) test of the replica host logic: every frame is
assigned to exactly one rank, the assignment is balanced, and the timing
reduction takes the maximum over ranks."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2012_08655_gb300.replicas import (frame_cost, frame_rmax, gather_to_rank0, max_over_ranks,
                                             merged_percentiles, shard_frames, shard_streams)


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


def _stream_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard_streams(32, world, rank)
    lat = [float(s) + 0.5 for s in mine]          # a stand-in latency per served stream
    got = gather_to_rank0({"streams": mine, "lat": lat, "span": 1.0 + rank})
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got))


def test_two_rank_stream_sharding_and_latency_gather():
    """The served stream split by stream id over two gloo ranks: every stream
    served by one rank, latencies gathered on rank 0 only, and the merged
    percentiles those of the union."""
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_stream_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[1] is None
    parts = res[0]
    assert sorted(s for part in parts for s in part["streams"]) == list(range(32))
    p50, p99 = merged_percentiles([part["lat"] for part in parts])
    import numpy as np
    allv = np.arange(32) + 0.5
    assert (p50, p99) == (float(np.percentile(allv, 50)), float(np.percentile(allv, 99)))
    assert max(part["span"] for part in parts) == 2.0


def test_frame_rmax_matches_the_oracle_bound():
    """The cost estimate's radius is the largest block radius of the frame."""
    import oracle
    for (w, h, fx, fy, k) in [(1920, 1080, 960.0, 540.0, 0.02), (640, 480, 600.5, 3.25, 0.04), (33, 65, -5.0, 70.0, 0.1)]:
        _, rad = oracle.sigma_table(w, h, 32, fx, fy, 0.5, k)
        assert frame_rmax(w, h, fx, fy, 0.5, k) == int(rad.max())
