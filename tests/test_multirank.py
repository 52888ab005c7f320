"""The benchmark's multi-rank path on CPU: two gloo ranks, each an independent
replica, combine their counts into whole-job figures (units summed, times
max-reduced) with no collective on the data path."""
from __future__ import annotations

import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    assert (r, w, local) == (rank, world, rank)
    units = [1000.0 * (rank + 1), 7.0 * (rank + 1)]
    times = [0.5 + rank, 0.25 * (rank + 1)]
    s, m = bench.reduce_over_ranks(units, times, world, "gloo")
    out[rank] = (s, m)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    for rank in range(world):
        s, m = out[rank]
        assert s == pytest.approx([3000.0, 21.0])
        assert m == pytest.approx([1.5, 0.5])


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_over_ranks([5.0], [2.0], 1, None) == ([5.0], [2.0])
