"""Autotuner for the batched launch shape.

The knobs are the warps that work on each queue item (the CTA size: 2, 4
or 8 warps per factorisation and per chunk), the persistent grid's CTAs per
SM and the solutions per chunk item. Each candidate runs the real batch a few times, timed with CUDA
events on the launching stream; the fastest is kept. Results are cached per
(GPU name, batch signature) in a JSON file next to the built library, so a
later process with the same kind of batch skips the search.

The batch signature buckets the matrices by words per row (W = 1..4) and
rounds each bucket's share to 1/16, plus log2 of the per-matrix cap.
"""

from __future__ import annotations

import json
import os

import numpy as np

from . import build as _build

WARPS = (2, 4, 8)                   # warps per work item (CTA size / 32)
CTAS_PER_SM = (1, 2, 4, 0)          # 0 = as many as fit
CHUNKS = (1 << 14, 1 << 15, 1 << 16, 1 << 17, 1 << 18)
CACHE = os.path.join(_build.OUT_DIR, "autotune.json")


def signature(Ws: np.ndarray, cap: int) -> str:
    hist = np.bincount(np.asarray(Ws, dtype=np.int64), minlength=5)[1:5]
    share = np.round(16 * hist / max(1, hist.sum())).astype(int)
    return f"W{'-'.join(map(str, share))}|cap{int(cap).bit_length() - 1}"


def _gpu_name() -> str:
    import torch

    return torch.cuda.get_device_name()


def _load_cache() -> dict:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save_cache(d: dict):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def time_batch(batch, cap: int, reps: int = 3) -> float:
    """Median milliseconds of one batch launch (after one warm-up)."""
    import torch

    batch.run(cap)
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        batch.run(cap)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return float(np.median(times))


def autotune(batch, cap: int, reps: int = 3, use_cache: bool = True) -> dict:
    """Pick (warps_per_item, ctas_per_sm, chunk) for this batch; set it on
    the batch and return {"tiles": [warps, cps, chunk], "ms": best,
    "table": [...], "cached": bool}."""
    key = f"{_gpu_name()}|{signature(batch.Ws, cap)}"
    cache = _load_cache() if use_cache else {}
    if key in cache and len(cache[key].get("tiles", ())) == 3:
        batch.set_tiles(*cache[key]["tiles"])
        return dict(cache[key], cached=True)
    table = []
    for warps in WARPS:
        for cps in CTAS_PER_SM:
            for chunk in CHUNKS:
                batch.set_tiles(warps, cps, chunk)
                table.append((warps, cps, chunk, time_batch(batch, cap, reps)))
    warps, cps, chunk, ms = min(table, key=lambda t: t[3])
    batch.set_tiles(warps, cps, chunk)
    entry = {"tiles": [warps, cps, chunk], "ms": ms, "table": [list(t) for t in table]}
    if use_cache:
        cache = _load_cache()
        cache[key] = entry
        _save_cache(cache)
    return dict(entry, cached=False)
