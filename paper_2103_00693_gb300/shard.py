"""Sharding of the hot path across ranks (one process per GPU).

Stage 2 has no exchange step: any index window can be seeded on its own, so
a window is cut into contiguous index ranges, one per rank, and each rank
reduces its range (hlf_enumerate_reduce on a GPU, or any function with the
same result). The three reduce quantities combine by +, + (mod 2^64) and
XOR, in any order, so the one exchange is a single all-gather of (2 + W)
64-bit words per rank over the default process group, followed by the
combine. Batches of independent matrices are dealt round-robin. The same
functions serve the benchmark's sharded mode (NCCL) and the CPU tests
(gloo).
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


def pack_partial(part, W: int) -> np.ndarray:
    """(count, hsum, xor_fold[W]) as int64 words [2 + W] (bit patterns)."""
    c, h, f = part
    row = np.zeros(2 + W, dtype=np.uint64)
    row[0], row[1] = np.uint64(int(c) % (1 << 64)), np.uint64(int(h) % (1 << 64))
    row[2:] = np.asarray(f, dtype=np.uint64)[:W]
    return row.view(np.int64)


def unpack_partial(row, W: int) -> tuple[int, int, np.ndarray]:
    r = np.asarray(row).astype(np.int64).view(np.uint64)
    return int(r[0]), int(r[1]), r[2:2 + W].copy()


def reduce_shard(reduce_fn, offset: int, count: int, rank: int, world: int):
    """This rank's partial: reduce_fn(o, c) over its slice of [offset, offset + count)."""
    o, c = shard_range(offset, count, rank, world)
    return reduce_fn(o, c)


def allgather_combine(part, W: int, world: int, device: str = "cpu") -> tuple[int, int, np.ndarray]:
    """Exchange every rank's partial with one all-gather over the default
    process group (tensors on `device`: "cuda" for NCCL, "cpu" for gloo) and
    combine them; every rank gets the whole window's reduce."""
    if world == 1:
        return combine_reduce([part])
    import torch
    import torch.distributed as dist

    mine = torch.from_numpy(pack_partial(part, W)).to(device)
    rows = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(rows, mine)
    return combine_reduce([unpack_partial(t.cpu().numpy(), W) for t in rows])
