"""The exchange step of a sharded batch over torch.distributed.

Each replica holds its shard's records (``Graph.shard_export``, a SHARD_DTYPE
array whose length differs between replicas).  ``allgather_records`` sends the
counts first, pads every replica's records to the largest count, all-gathers
the padded byte tensors (NCCL on device tensors, gloo on host tensors) and
returns every replica's records, concatenated in rank order, for
``Graph.shard_commit``.  Marshalling only: nothing of the method runs here.
"""
from __future__ import annotations

import numpy as np

from .dygrass import SHARD_DTYPE


def allgather_records(recs: np.ndarray, group=None, device=None) -> np.ndarray:
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    dev = torch.device(device) if device is not None else (
        torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else torch.device("cpu"))
    recs = np.ascontiguousarray(recs, SHARD_DTYPE)
    count = torch.tensor([recs.size], dtype=torch.int64, device=dev)
    counts = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(counts, count, group=group)
    counts = [int(c.item()) for c in counts]
    width = max(counts) * SHARD_DTYPE.itemsize
    if width == 0:
        return np.zeros(0, SHARD_DTYPE)
    buf = np.zeros(width, np.uint8)
    buf[: recs.nbytes] = recs.view(np.uint8)
    mine = torch.from_numpy(buf).to(dev)
    parts = [torch.empty(width, dtype=torch.uint8, device=dev) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    out = [p.cpu().numpy()[: c * SHARD_DTYPE.itemsize].view(SHARD_DTYPE) for p, c in zip(parts, counts)]
    return np.concatenate(out)
