"""Host-side sharding of the hot path across ranks (one process per GPU).

Stage 2 has no exchange step: any index window can be seeded on its own, so
a window is cut into contiguous index ranges, one per rank, and each rank
reduces its range with hlf_enumerate_reduce. The three reduce quantities
combine by +, + (mod 2^64) and XOR, in any order. Batches of independent
matrices are dealt round-robin. Nothing here touches a GPU.
"""

from __future__ import annotations

import numpy as np


def shard_range(offset: int, count: int, rank: int, world: int) -> tuple[int, int]:
    """The rank's contiguous slice (offset, count) of [offset, offset + count)."""
    if not 0 <= rank < world:
        raise ValueError("rank outside [0, world)")
    base, extra = divmod(count, world)
    start = offset + rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def shard_items(n_items: int, rank: int, world: int) -> list[int]:
    """Round-robin deal of n_items independent work items."""
    return list(range(rank, n_items, world))


def combine_reduce(parts) -> tuple[int, int, np.ndarray]:
    """Combine (count, hsum, xor_fold[W]) partials from disjoint ranges."""
    count, hsum, fold = 0, 0, None
    for c, h, f in parts:
        f = np.asarray(f, dtype=np.uint64)
        count += int(c)
        hsum = (hsum + int(h)) % (1 << 64)
        fold = f.copy() if fold is None else fold ^ f
    return count, hsum, fold
