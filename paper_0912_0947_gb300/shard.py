"""A batch of covers over several GPUs, one process per GPU.

Covers are independent, so the batch shards with no exchange on the data
path: ``stego_partition`` gives every cover a rank by byte volume, each rank
runs the batched calls on its own covers, and the per-cover results are
gathered on the host afterwards (``torch.distributed.all_gather_object``:
a few bytes per cover, no device data).  Marshalling only: the
steganography runs in the library's batched kernels on each rank.
"""
from __future__ import annotations

import numpy as np

from . import stego_partition


def my_covers(sizes, rank: int, world: int) -> np.ndarray:
    """Indices (ascending) of the covers rank `rank` of `world` processes."""
    rank_of, _ = stego_partition(sizes, world)
    return np.nonzero(rank_of == rank)[0]


def gather_results(mine: np.ndarray, results, n: int, group=None) -> list:
    """Per-cover results of every rank, in cover order.  `mine` are this
    rank's cover indices and `results` its results for them (same order);
    with one process no collective runs."""
    import torch.distributed as dist
    part = list(zip((int(i) for i in mine), results))
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        parts = [None] * dist.get_world_size(group)
        dist.all_gather_object(parts, part, group=group)
    else:
        parts = [part]
    out = [None] * n
    for p in parts:
        for i, r in p:
            out[i] = r
    return out


def run_sharded(sizes, rank: int, world: int, compute, group=None) -> list:
    """compute(indices) -> results for those covers, run on this rank's
    share; returns every cover's result in cover order."""
    mine = my_covers(sizes, rank, world)
    return gather_results(mine, compute(mine), len(sizes), group)
