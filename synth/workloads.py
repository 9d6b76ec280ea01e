"""The five named workloads (inputs only: sizes, seeds and draws).

1. grid3x3     3 x 3 grid, p = 1/2, Bernoulli(1/2) diagonal, seed 5 (r = 9):
               factor and materialise every solution (<= 512).
2. grid6x6     all-connected 6 x 6 grid, Bernoulli(1/2) diagonal, seed 3
               (r = 36, the largest rank this family reaches, 2^36 = 6.9e10
               solutions): reduce all 2^r, materialise the first 2^30.
3. grid8x8     8 x 8 grid, p = 1/2, Bernoulli(1/2) diagonal, seed 0 (r = 54):
               reduce a 2^40 window at a seeded offset, sample 2^20 indices.
4. batch4096   4096 grids, N uniform in 4..16, p = 1/2: factor all, reduce
               min(2^r, 2^20) solutions of each.
5. stream      Poisson arrivals, N uniform in 3..32, p = 1/2, windows
               log-uniform in 2^10..2^24 solutions, returned to the host.

The ranks quoted above are what the seeded matrices have; they are facts
about the inputs that the tests recompute, not inputs themselves. Both
headline single instances are full rank (r = n maximises 2^r), where the
RREF basis is the identity and z^a = 0. The parity tests therefore also run
each of these two workloads at full size on a seed of lower rank:

* grid3x3 seed 9: r = 6, z^a != 0, pivots {0, 3, 4, 5, 6, 8};
* grid6x6 seed 1: r = 34, z^a != 0, free columns 33 and 35.
"""

from __future__ import annotations

from . import grid

GRID3 = dict(N=3, p=0.5, seed=5)
GRID6 = dict(N=6, p=1.0, seed=3)
GRID3_LOWRANK = dict(N=3, p=0.5, seed=9)
GRID6_LOWRANK = dict(N=6, p=1.0, seed=1)
GRID6_STORE_LOG2 = 30
GRID8 = dict(N=8, p=0.5, seed=0)
GRID8_WINDOW_LOG2 = 40
GRID8_OFFSET_SEED = 17
GRID8_SAMPLE_LOG2 = 20
GRID8_SAMPLE_SEED = 23
BATCH = dict(count=4096, N_lo=4, N_hi=16, p=0.5, seed=4096)
BATCH_CAP_LOG2 = 20
STREAM = dict(N_lo=3, N_hi=32, p=0.5, win_log2_lo=10, win_log2_hi=24, seed=5150)


def grid3():
    return grid.grid_instance(GRID3["N"], GRID3["p"], GRID3["seed"])


def grid6():
    return grid.grid_instance(GRID6["N"], GRID6["p"], GRID6["seed"])


def grid3_lowrank():
    return grid.grid_instance(GRID3_LOWRANK["N"], GRID3_LOWRANK["p"], GRID3_LOWRANK["seed"])


def grid6_lowrank():
    return grid.grid_instance(GRID6_LOWRANK["N"], GRID6_LOWRANK["p"], GRID6_LOWRANK["seed"])


def grid8():
    return grid.grid_instance(GRID8["N"], GRID8["p"], GRID8["seed"])


def grid8_window(space_log2: int) -> tuple[int, int]:
    """(offset, count) of the 2^40 window inside [0, 2^space_log2)."""
    count = 1 << GRID8_WINDOW_LOG2
    return grid.window_offset(GRID8_OFFSET_SEED, space_log2, count), count


def grid8_samples(offset: int, count: int):
    """2^20 indices drawn uniformly from the window."""
    return grid.sample_indices(GRID8_SAMPLE_SEED, 1 << GRID8_SAMPLE_LOG2, offset, offset + count)


def batch():
    return grid.batch_instances(**BATCH)


def stream(count: int, rate_per_s: float, seed: int | None = None):
    kw = dict(STREAM)
    if seed is not None:
        kw["seed"] = seed
    return grid.poisson_stream(count, rate_per_s, kw["N_lo"], kw["N_hi"], kw["p"],
                               kw["win_log2_lo"], kw["win_log2_hi"], kw["seed"])
