"""The N>1 benchmark path on CPU: two gloo ranks, replica sharding by stream.

Replicas are independent (Section 3), so ranks shard them with no data-path
collective: each rank draws its own replicas from Philox stream = rank and the
job reduces only the slowest rank's time and the total spin-updates.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle as O
    # each rank: its own replicas of one small instance (stream = rank)
    m0, t0 = O.draw_replicas(0, 4, 50, 0.0, 4.0, stream=rank)
    tot_ms, upd = 10.0 + 5.0 * rank, 1000 * (rank + 1)
    t, u = bench.aggregate(tot_ms, upd, "cpu")
    out[rank] = (t, u, float(m0[0, 0]), float(t0[0]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_reduce_time_and_updates_and_draw_disjoint_replicas():
    world = 2
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    r0, r1 = out[0], out[1]
    assert r0[0] == r1[0] == 15.0          # max over ranks
    assert r0[1] == r1[1] == 3000.0        # sum over ranks
    assert (r0[2], r0[3]) != (r1[2], r1[3])  # different replica draws per rank
