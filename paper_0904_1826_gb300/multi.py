"""Host-side pieces of the multi-GPU path: templates shard by sky point with
no data-path communication; the one exchange is the merge of the per-rank
toplists (each rank's K best, K x 12 bytes)."""
from __future__ import annotations

import numpy as np


def shard_range(n_total: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [lo, hi) share of n_total items for `rank` (sizes differ by at most 1)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank outside the world")
    base, extra = divmod(n_total, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def merge_toplists(lists, k: int):
    """Merge per-rank toplists [(idx int64[k_r], 2F float32[k_r]), ...] whose
    indices are already global into the global top k, ordered by (2F desc,
    index asc) -- the same order every rank's list has."""
    idx = np.concatenate([np.asarray(a, dtype=np.int64) for a, _ in lists])
    val = np.concatenate([np.asarray(b, dtype=np.float32) for _, b in lists])
    order = np.lexsort((idx, -val.astype(np.float64)))[:k]
    return idx[order], val[order]
