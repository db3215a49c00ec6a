"""Replica sharding across processes (one process per GPU).

FEM's replicas never interact (Results, "Free-Energy Machine": every replica
minimises its own mean-field free energy), so the replica dimension shards with
no data-path communication: rank k runs replicas [off_k, off_k + R_k) of the
global replica set, from the matching columns of the initial fields, and the
only exchange is one gather of (best energy, rank, replica) at the end.
"""
from __future__ import annotations

import numpy as np

__all__ = ["shard_replicas", "shard_fields", "best_over_ranks"]


def shard_replicas(total: int, world: int, rank: int, multiple: int = 32):
    """(offset, count) of rank's replica block.  Blocks are multiples of `multiple`
    (the kernels' replica granularity); the last ranks may get one block less."""
    if total % multiple != 0:
        raise ValueError(f"total replicas {total} must be a multiple of {multiple}")
    blocks = total // multiple
    if blocks < world:
        raise ValueError(f"{blocks} replica blocks cannot feed {world} ranks")
    base, extra = divmod(blocks, world)
    start = rank * base + min(rank, extra)
    count = base + (1 if rank < extra else 0)
    return start * multiple, count * multiple


def shard_fields(h0: np.ndarray, world: int, rank: int, multiple: int = 32) -> np.ndarray:
    """The columns of h0 ([n][R] or [n][R][q]) that rank runs, contiguous."""
    off, cnt = shard_replicas(h0.shape[1], world, rank, multiple)
    return np.ascontiguousarray(h0[:, off:off + cnt])


def best_over_ranks(energy: float, replica: int, rank: int, world: int, group=None, device=None):
    """Global argmin of (energy, global replica index) over ranks with one all_gather.
    `replica` is the rank-local index; ties go to the lowest global replica index.
    Returns (energy, global_replica, owner_rank)."""
    import torch
    import torch.distributed as dist

    dev = device if device is not None else torch.device("cpu")
    mine = torch.tensor([float(energy), float(replica), float(rank)], dtype=torch.float64, device=dev)
    parts = [torch.zeros_like(mine) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    rows = [p.cpu().numpy() for p in parts]
    return min(((r[0], int(r[1]), int(r[2])) for r in rows), key=lambda x: (x[0], x[2], x[1]))
