"""One process per GPU: which series a rank evaluates, and the rank bookkeeping
around a timed region.

Series are independent units of the estimator (Sec. 2.3: every c_k of one
series or pair depends on that series or pair only), so a batch splits across
ranks with no exchange on the data path.  Two ways are offered:

* weak scaling -- every rank evaluates its own batch (``rank_seed``);
* strong scaling -- one batch is cut into contiguous series ranges of about
  equal cost (``partition_series``), each rank evaluates its range
  (``sub_batch``) and rank 0 gathers the rows (``gather_rows``).

The only collectives are host-side bookkeeping: barriers, the maximum of the
per-rank times and the gather of result rows (``torch.distributed``; NCCL on
GPUs, gloo in the CPU tests).
"""
from __future__ import annotations

import os

import numpy as np


def dist_env():
    """(rank, world_size, local_rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of rank `rank`'s own batch under weak scaling."""
    return int(base_seed) + int(rank)


def series_cost(offs, K: int, offs_y=None) -> np.ndarray:
    """Work of each series: (outer points) x K items plus a fixed per-series term
    (launch tiles, statistics)."""
    offs = np.asarray(offs, dtype=np.int64)
    n = np.diff(offs if offs_y is None else np.asarray(offs_y, dtype=np.int64)).astype(np.float64)
    return n * float(max(K, 1)) + 2048.0 * float(max(K, 1))


def partition_series(offs, K: int, world: int, offs_y=None):
    """Contiguous series ranges [(b0, b1)] per rank, cut where the cumulative cost
    crosses r / world of the total.  Every series lands on exactly one rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    cost = series_cost(offs, K, offs_y)
    B = cost.size
    cum = np.concatenate([[0.0], np.cumsum(cost)])
    total = cum[-1]
    cuts = [0]
    for r in range(1, world):
        cuts.append(int(np.searchsorted(cum, total * r / world, side="left")))
    cuts.append(B)
    cuts = np.maximum.accumulate(np.minimum(np.asarray(cuts), B))
    return [(int(cuts[r]), int(cuts[r + 1])) for r in range(world)]


def sub_batch(offs, b0: int, b1: int):
    """CSR offsets of series [b0, b1) rebased to 0, and the point slice they cover."""
    offs = np.asarray(offs, dtype=np.int64)
    lo, hi = int(offs[b0]), int(offs[b1])
    return offs[b0:b1 + 1] - lo, slice(lo, hi)


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank scalar (the timed region's length)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_rows(rows: np.ndarray, dst: int = 0):
    """Rank `dst` receives every rank's rows, concatenated in rank order (None elsewhere)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return rows
    out = [None] * dist.get_world_size() if dist.get_rank() == dst else None
    dist.gather_object(rows, out, dst=dst)
    if dist.get_rank() != dst:
        return None
    return np.concatenate([np.asarray(r).reshape(-1, *np.asarray(rows).shape[1:]) for r in out], axis=0)
