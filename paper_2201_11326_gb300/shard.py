"""Row-range sharding of one s-line graph across ranks (host logic).

Rows are the independent units of Algorithm 2's parallel loop (Section III-C):
rank r builds the rows [splits[r], splits[r+1]) of L_s(H) with
slg_build_window, and the canonical list is the ranks' slices in rank order.
The ranks exchange nothing but their pair counts (8 bytes each), which place
each slice in the global list. Splits balance the per-row work.
"""
from __future__ import annotations

import numpy as np


def balanced_splits(work: np.ndarray, nshards: int) -> np.ndarray:
    """Row boundaries 0 = b_0 <= ... <= b_n = m with about equal work per shard.

    ``work`` is a non-negative per-row cost (e.g. wedges plus pairs). Shard k
    ends at the first row where the running work reaches (k+1)/n of the total.
    """
    w = np.asarray(work, dtype=np.float64)
    m = w.size
    if nshards < 1:
        raise ValueError("nshards must be >= 1")
    csum = np.concatenate([[0.0], np.cumsum(w)])
    total = csum[-1]
    splits = np.zeros(nshards + 1, np.int64)
    splits[-1] = m
    if total <= 0:
        splits[1:-1] = (np.arange(1, nshards) * m) // nshards
        return splits
    for k in range(1, nshards):
        splits[k] = int(np.searchsorted(csum, total * k / nshards, side="left"))
    return np.maximum.accumulate(np.clip(splits, 0, m))


def global_offsets(counts_per_rank) -> np.ndarray:
    """Exclusive prefix of the ranks' pair counts: where each slice starts."""
    c = np.asarray(counts_per_rank, dtype=np.int64)
    return np.concatenate([[0], np.cumsum(c)])


def exchange_counts(local_count: int, group=None) -> np.ndarray:
    """All ranks' pair counts (one int64 per rank) via torch.distributed."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    t = torch.tensor([int(local_count)], dtype=torch.int64)
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    out = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(out, t, group=group)
    return np.array([int(x.item()) for x in out], np.int64)
