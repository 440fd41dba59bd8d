"""Independent problems across ranks (one process per GPU).

The periodic sum of one unit cell is evaluated on one GPU; several GPUs
evaluate independent problems (different cells, or the problems of a batch)
with no data exchange.  Two host-side pieces: which problems a rank owns, and
the max over ranks of a time, which is the job's time.
"""

from __future__ import annotations

import numpy as np


def shard(nprob: int, rank: int, world: int) -> np.ndarray:
    """Problems of `rank`: a contiguous block, sizes differing by at most one."""
    if world < 1 or not 0 <= rank < world or nprob < 0:
        raise ValueError("bad rank / world / nprob")
    base, extra = divmod(nprob, world)
    lo = rank * base + min(rank, extra)
    return np.arange(lo, lo + base + (1 if rank < extra else 0), dtype=np.int64)


def shard_offsets(off: np.ndarray, rank: int, world: int):
    """Sub-batch of a CSR batch: (first, last + 1) rows and the rebased offsets."""
    off = np.asarray(off, dtype=np.int64)
    p = shard(len(off) - 1, rank, world)
    if len(p) == 0:
        return 0, 0, np.zeros(1, dtype=np.int64)
    a, b = int(off[p[0]]), int(off[p[-1] + 1])
    return a, b, off[p[0]:p[-1] + 2] - a


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Max of a per-rank float over the process group (the value itself alone)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, dist=None, device=None) -> float:
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
