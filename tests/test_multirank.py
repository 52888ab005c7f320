"""Multi-rank paths on CPU (gloo ranks): the benchmark's replicas combine their
counts into whole-job figures (units summed, times max-reduced) with no
collective on the data path; a sharded batch's exchange step gathers every
replica's records (counts first, then a padded all-gather)."""
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


def _shard_rank_main(rank, world, port, sizes, out):
    """One replica of the sharded batch's exchange: its records (length
    sizes[rank]) go out, every replica's come back in rank order."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import numpy as np

    from paper_2505_02741_b300.dygrass import SHARD_DTYPE
    from paper_2505_02741_b300.shard import allgather_records
    dist.init_process_group("gloo", rank=rank, world_size=world)
    recs = np.zeros(sizes[rank], SHARD_DTYPE)
    base = sum(sizes[:rank])
    recs["j"] = base + np.arange(sizes[rank])
    recs["best"] = rank
    recs["result"]["r_est"] = np.linspace(0.5, 2.5, sizes[rank]) * (rank + 1)
    got = allgather_records(recs, device="cpu")
    out[rank] = got.tobytes()
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("sizes", [(5, 3), (0, 4), (7, 0, 2)])
def test_shard_record_exchange_gloo(sizes):
    """The exchange step of a sharded batch over gloo ranks on CPU: counts
    first, padded all-gather, every rank gets all records in rank order."""
    import numpy as np

    from paper_2505_02741_b300.dygrass import SHARD_DTYPE
    world = len(sizes)
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_shard_rank_main, args=(world, port, list(sizes), out), nprocs=world, start_method="spawn",
                       join=True)
    expect = np.zeros(sum(sizes), SHARD_DTYPE)
    expect["j"] = np.arange(sum(sizes))
    lo = 0
    for r, n in enumerate(sizes):
        expect["best"][lo:lo + n] = r
        expect["result"]["r_est"][lo:lo + n] = np.linspace(0.5, 2.5, n) * (r + 1)
        lo += n
    for rank in range(world):
        assert out[rank] == expect.tobytes()
