"""Multi-rank bench logic on CPU (gloo, world size 2): ranks render disjoint
runs of poses (replicas, no data-path collective) and the step time is the max
over ranks."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = bench.shard_poses(rank, world, 5, 64)
        t = bench.max_over_ranks(10.0 + rank)
        s = bench.sum_over_ranks(len(mine))
        q.put((rank, mine, t, s))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(world):
        rank, mine, t, s = q.get(timeout=120)
        out[rank] = (mine, t, s)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert set(out[0][0]).isdisjoint(out[1][0])
    assert out[0][1] == out[1][1] == 11.0
    assert out[0][2] == out[1][2] == 10.0


def test_single_process_identity():
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.shard_poses(0, 1, 3, 64) == [0, 1, 2]
    assert bench.shard_poses(1, 2, 3, 4) == [3, 0, 1]
