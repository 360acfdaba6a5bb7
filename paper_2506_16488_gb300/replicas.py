"""Query-parallel replicas across GPUs (one process per GPU).

PPSP queries are independent (Sec. 4: a batch is a set of s-t pairs), so
several GPUs each hold a full copy of the graph and answer their own share of
the query stream; no search state crosses GPUs and there is no collective on
the data path.  The only communication is host-side bookkeeping: the timing
of a step is the maximum over ranks (``max_over_ranks``) and the throughput is
the queries of all ranks over that time (weak scaling: the per-GPU batch is
fixed as ranks are added).
"""

from __future__ import annotations

import numpy as np


def shard(pairs: np.ndarray, rank: int, world: int) -> np.ndarray:
    """Rank `rank`'s share of a query array (contiguous, sizes differ by <= 1)."""
    k = pairs.shape[0]
    lo = k * rank // world
    hi = k * (rank + 1) // world
    return pairs[lo:hi]


def rank_seed(base: int, rank: int) -> int:
    """Seed of rank `rank`'s own query batch in weak scaling (rank 0 = base)."""
    return base + 7919 * rank


def max_over_ranks(value: float, device: str = "cpu") -> float:
    """Maximum of a scalar over all ranks of the default process group
    (identity without one)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device: str = "cpu") -> float:
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
