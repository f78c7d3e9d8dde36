"""Particle-range partitioning across ranks and the one exchange step of a partitioned run.

Particles never interact (Sec. 4.2), so a release of N particles splits into contiguous
id ranges, one per rank; each rank's context holds its range (``lpm_release_range``),
draws the same keyed random numbers as a single run would, and bins with the scale of
the whole release. The only exchange is an integer sum of the fixed-point grids and
counters, which is associative, so the reduced result is bit-identical to the
single-context run whatever the rank count or reduction order.
"""
from __future__ import annotations

from typing import Tuple

import numpy as np


def partition(n_total: int, world: int, rank: int) -> Tuple[int, int]:
    """Contiguous range [first, first + count) of ``n_total`` ids held by ``rank``;
    range sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside world of {world}")
    if n_total < world:
        raise ValueError("fewer particles than ranks")
    base, extra = divmod(n_total, world)
    first = rank * base + min(rank, extra)
    count = base + (1 if rank < extra else 0)
    return first, count


def allreduce_fixed(values: np.ndarray, group=None, device=None) -> np.ndarray:
    """Integer sum over all ranks of a fixed-point array (uint64 or int64 values below
    2^63) through torch.distributed; returns an array of the input dtype."""
    import torch
    import torch.distributed as dist
    a = np.ascontiguousarray(values)
    t = torch.from_numpy(a.view(np.int64).copy())
    if device is not None:
        t = t.to(device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy().view(a.dtype).reshape(a.shape)
