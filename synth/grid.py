"""Grid-graph instances G(A) of the 2D HLF problem (§1, Fig. 1(a)) and the
random draws the workloads need.

Conventions (the same on both sides of every parity test):

* Vertices of the N x N grid are numbered row-major, vertex v = row * N + col
  (0-based here; the paper's z_1 ... z_n is vertex 0 ... n-1).
* A[i, j] = 1 iff (i, j) is a grid edge that is present (i != j), and
  A[i, i] = b_i, the diagonal bit (§1; Fig. 1(a) marks b_i = 1 vertices yellow).
* Random grids draw, in row-major vertex order, first the right edge and then
  the down edge of each vertex (each present with probability p), and then the
  whole diagonal b_i ~ Bernoulli(1/2); all draws come from one
  numpy.random.Generator(PCG64(seed)).

Nothing in this module knows how the problem is solved.
"""

from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def grid_edges(N: int) -> list[tuple[int, int]]:
    """All nearest-neighbour edges of the N x N grid, in draw order: for each
    vertex in row-major order, its right edge then its down edge."""
    edges = []
    for row in range(N):
        for col in range(N):
            v = row * N + col
            if col + 1 < N:
                edges.append((v, v + 1))
            if row + 1 < N:
                edges.append((v, v + N))
    return edges


def _assemble(n: int, edges, b) -> np.ndarray:
    A = np.zeros((n, n), dtype=np.uint8)
    for i, j in edges:
        A[i, j] = 1
        A[j, i] = 1
    A[np.arange(n), np.arange(n)] = np.asarray(b, dtype=np.uint8)
    return A


def b_from_string(s: str) -> np.ndarray:
    """The paper's diagonal strings b = b_1 b_2 ... b_n, written left to right
    (§4: "b = 1011"), as a uint8 vector indexed by 0-based vertex."""
    s = s.strip()
    if any(ch not in "01" for ch in s):
        raise ValueError(f"not a bit string: {s!r}")
    return np.frombuffer(s.encode(), dtype=np.uint8) - ord("0")


def paper_b_patterns(n: int) -> list[str]:
    """The three diagonals the paper runs on every all-connected grid size
    (§4 and App. C): 0^(n), 0^(n-1)1 and 0^(n-2)11."""
    return ["0" * n, "0" * (n - 1) + "1", "0" * (n - 2) + "11"]


def all_connected(N: int, b) -> np.ndarray:
    """All-connected N x N grid (every nearest-neighbour edge present, §3 and
    App. B) with diagonal b (a bit string or a 0/1 vector of length N*N)."""
    n = N * N
    if isinstance(b, str):
        b = b_from_string(b)
    b = np.asarray(b, dtype=np.uint8)
    if b.shape != (n,):
        raise ValueError(f"diagonal of length {b.shape} for n={n}")
    return _assemble(n, grid_edges(N), b)


def grid_instance(N: int, p: float, seed: int, *, b=None) -> np.ndarray:
    """Random N x N grid: each edge present with probability p, then (unless b
    is given) a Bernoulli(1/2) diagonal. p = 1 gives the all-connected grid."""
    rng = _rng(seed)
    edges = grid_edges(N)
    keep = rng.random(len(edges)) < p
    present = [e for e, k in zip(edges, keep) if k]
    n = N * N
    if b is None:
        b = (rng.random(n) < 0.5).astype(np.uint8)
    elif isinstance(b, str):
        b = b_from_string(b)
    return _assemble(n, present, b)


def random_symmetric(n: int, density: float, seed: int) -> np.ndarray:
    """A symmetric 0/1 matrix that is not a grid (§5: the scheme holds for any
    symmetric A): each upper-triangle entry and each diagonal entry is 1 with
    probability `density`."""
    rng = _rng(seed)
    U = (rng.random((n, n)) < density).astype(np.uint8)
    U = np.triu(U, 1)
    A = U | U.T
    A[np.arange(n), np.arange(n)] = (rng.random(n) < density).astype(np.uint8)
    return A


def random_regular(n: int, d: int, seed: int, *, b=None) -> np.ndarray:
    """A random simple d-regular graph on n vertices (§5: any symmetric A),
    drawn by sequential pairing: n*d points (d per vertex) are matched two at
    a time at random, a pair that would make a loop or a repeated edge is
    redrawn, and a dead end restarts the draw. The diagonal is Bernoulli(1/2)
    unless b is given."""
    if (n * d) % 2 or d >= n:
        raise ValueError("need n*d even and d < n")
    rng = _rng(seed)
    for _ in range(1000):
        pts = list(np.repeat(np.arange(n), d))
        edges = set()
        ok = True
        while pts:
            for _ in range(200):
                i, j = rng.integers(0, len(pts), size=2)
                u, v = int(pts[i]), int(pts[j])
                if i != j and u != v and (min(u, v), max(u, v)) not in edges:
                    break
            else:
                ok = False
                break
            edges.add((min(u, v), max(u, v)))
            for k in sorted((int(i), int(j)), reverse=True):
                pts[k] = pts[-1]
                pts.pop()
        if ok:
            if b is None:
                b = (rng.random(n) < 0.5).astype(np.uint8)
            return _assemble(n, sorted(edges), b)
    raise RuntimeError("could not draw a simple regular graph")


def window_offset(seed: int, space_log2: int, count: int) -> int:
    """A window start drawn uniformly from [0, 2^space_log2 - count]; the
    caller passes space_log2 = min(r, 64) and a count that fits."""
    space = 1 << space_log2
    if count > space:
        raise ValueError("window longer than the index space")
    hi = space - count  # inclusive upper bound, < 2^64 + 1
    rng = _rng(seed)
    # two 32-bit draws give a uniform 64-bit integer; reduce by rejection
    span = hi + 1
    while True:
        x = int(rng.integers(0, 1 << 32, dtype=np.uint64)) << 32
        x |= int(rng.integers(0, 1 << 32, dtype=np.uint64))
        if span >= (1 << 64):
            return x
        lim = (1 << 64) - ((1 << 64) % span)
        if x < lim:
            return x % span


def sample_indices(seed: int, m: int, lo: int, hi: int) -> np.ndarray:
    """m indices drawn uniformly (with replacement) from [lo, hi), as uint64."""
    if hi <= lo:
        raise ValueError("empty range")
    rng = _rng(seed)
    span = hi - lo
    if span <= (1 << 62):
        return (rng.integers(0, span, size=m, dtype=np.uint64) + np.uint64(lo)).astype(np.uint64)
    hi32 = rng.integers(0, 1 << 32, size=m, dtype=np.uint64)
    lo32 = rng.integers(0, 1 << 32, size=m, dtype=np.uint64)
    x = (hi32 << np.uint64(32)) | lo32
    return np.array([lo + int(v) % span for v in x], dtype=np.uint64)


def batch_instances(count: int, N_lo: int, N_hi: int, p: float, seed: int) -> list[np.ndarray]:
    """`count` random grids with N uniform in [N_lo, N_hi] (the batched
    workload: 4096 grids, N in 4..16, p = 1/2). Instance k uses seed
    (seed, k) so that any one instance can be rebuilt alone."""
    rng = _rng(seed)
    Ns = rng.integers(N_lo, N_hi + 1, size=count)
    out = []
    for k, N in enumerate(Ns):
        sub = int(np.random.SeedSequence([seed, k]).generate_state(1)[0])
        out.append(grid_instance(int(N), p, sub))
    return out


def poisson_stream(count: int, rate_per_s: float, N_lo: int, N_hi: int, p: float,
                   win_log2_lo: int, win_log2_hi: int, seed: int) -> list[dict]:
    """A served request stream: Poisson arrivals at `rate_per_s`, grids with N
    uniform in [N_lo, N_hi], edge probability p, and windows whose length is
    log-uniform in [2^win_log2_lo, 2^win_log2_hi]. Each request carries
    `t_arrival` (s), `A`, `want` (requested window length) and `u` (a uniform
    64-bit integer from which the window start is taken once the instance's
    index space is known)."""
    rng = _rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=count)
    t = np.cumsum(gaps) - gaps[0]
    Ns = rng.integers(N_lo, N_hi + 1, size=count)
    logs = rng.uniform(win_log2_lo, win_log2_hi, size=count)
    us = rng.integers(0, 1 << 63, size=count, dtype=np.uint64)
    reqs = []
    for k in range(count):
        sub = int(np.random.SeedSequence([seed, k]).generate_state(1)[0])
        reqs.append({
            "id": k,
            "t_arrival": float(t[k]),
            "A": grid_instance(int(Ns[k]), p, sub),
            "want": int(2.0 ** logs[k]),
            "u": int(us[k]),
        })
    return reqs
