"""Batched factorisation + reduction of many matrices in one persistent
launch (hlf_batch_*, hlf_factor_batched, hlf_enumerate_batched in
include/hlf.h), with CUDA-graph capture and the plain one-launch-per-matrix
path it is compared with.

Packing the matrices into one device buffer (rows back to back, a word
offset and n per matrix) is argument marshalling; all solver work runs in
the library's batch kernel.
"""

from __future__ import annotations

import os

import numpy as np

from . import hlf


def spin_limit_from_env() -> int | None:
    """HLF_SPIN_LIMIT: the bound on a chunk's polls for its matrix (see
    hlf_batch_set_spin_limit), for every plan this module creates; unset
    keeps the library's default."""
    v = os.environ.get("HLF_SPIN_LIMIT", "")
    if not v:
        return None
    limit = int(v, 0)
    if not 1 <= limit < 1 << 32:
        raise ValueError("HLF_SPIN_LIMIT must be in [1, 2^32)")
    return limit


class Batch:
    """Device-resident batch of matrices and its plan (workspace)."""

    def __init__(self, mats: list[np.ndarray], device: str = "cuda"):
        import torch

        self.count = len(mats)
        self.ns = np.array([A.shape[0] for A in mats], dtype=np.int32)
        if np.any(self.ns > hlf.BATCH_MAX_N) or np.any(self.ns < 1):
            raise ValueError(f"batched matrices need 1 <= n <= {hlf.BATCH_MAX_N}")
        self.Ws = (self.ns + 63) // 64
        sizes = self.ns.astype(np.int64) * self.Ws
        self.offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)  # [count + 1]
        self.word_off = self.offsets[:-1].copy()
        packed = np.concatenate([hlf.pack_rows(A).ravel() for A in mats]) if mats else np.zeros(0, np.uint64)
        self.A_dev = torch.from_numpy(packed.view(np.int64)).to(device)
        self.off_dev = torch.from_numpy(self.word_off).to(device)
        self.offsets_dev = torch.from_numpy(self.offsets).to(device)
        self.n_dev = torch.from_numpy(self.ns).to(device)
        self.r_dev = torch.empty(self.count, dtype=torch.int32, device=device)
        self.red_dev = torch.empty((self.count, hlf.REDUCE_WORDS), dtype=torch.int64, device=device)
        self.plan = hlf.hlf_batch_create(max(self.count, 1))
        self.tiles = (8, 0, 1 << 16)
        self.graph = None
        limit = spin_limit_from_env()
        if limit is not None:
            hlf.hlf_batch_set_spin_limit(self.plan, limit)

    def set_tiles(self, warps_per_item: int, ctas_per_sm: int, chunk: int):
        hlf.hlf_batch_set_tiles(self.plan, warps_per_item, ctas_per_sm, chunk)
        self.tiles = (warps_per_item, ctas_per_sm, chunk)

    def run(self, cap: int, stream=None):
        """Enqueue one fused launch: factor every matrix, reduce solutions
        [0, min(2^r, cap)) of each."""
        hlf.hlf_batch_factor_reduce(self.plan, self.A_dev, self.off_dev, self.n_dev, self.count, cap,
                                    self.r_dev, self.red_dev, stream)

    def factor(self, stream=None):
        """Stage 1 of every matrix (hlf_factor_batched, offsets table [count + 1])."""
        hlf.hlf_factor_batched(self.plan, self.A_dev, self.offsets_dev, self.count, self.r_dev, stream)

    def reduce(self, cap: int, stream=None):
        """Stage 2 reduce of the factored matrices into red_dev."""
        hlf.hlf_enumerate_batched(self.plan, cap, red_dev=self.red_dev, stream=stream)

    def store(self, cap: int, out_dev, out_offsets_dev, stream=None):
        """Stage 2 store of the factored matrices into out_dev at out_offsets_dev."""
        hlf.hlf_enumerate_batched(self.plan, cap, out_dev=out_dev, out_offsets_dev=out_offsets_dev, stream=stream)

    def capture(self, cap: int):
        """Capture run(cap) into a CUDA graph; replay() re-runs it."""
        import torch

        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.run(cap, s)  # warm-up outside the graph
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            self.run(cap, s)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def status(self) -> int:
        return hlf.hlf_batch_get_status(self.plan)

    def results(self):
        """(ranks int32[count], list of ReduceResult)."""
        r = self.r_dev.cpu().numpy()
        red = self.red_dev.cpu().numpy()
        return r, [hlf.ReduceResult.from_words(red[b], int(self.Ws[b])) for b in range(self.count)]

    def close(self):
        if self.plan:
            hlf.hlf_batch_destroy(self.plan)
            self.plan = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PlainPath:
    """The plain path the batched launch is compared with: for each matrix,
    one factor launch (hlf_factor) and one reduce launch of [0, min(2^r, cap))
    (hlf_enumerate_reduce_upto, which reads r on the device), all enqueued on
    one stream with no host wait; the matrices are staged on the device once,
    before any timing."""

    def __init__(self, mats: list[np.ndarray], device: str = "cuda"):
        import torch

        self.count = len(mats)
        self.ns = [A.shape[0] for A in mats]
        packed = np.concatenate([hlf.pack_rows(A).ravel() for A in mats]) if mats else np.zeros(0, np.uint64)
        self.A_dev = torch.from_numpy(packed.view(np.int64)).to(device)
        self.views = []
        at = 0
        for n in self.ns:
            W = hlf.words(n)
            self.views.append(self.A_dev[at: at + n * W].view(n, W))
            at += n * W
        self.red_dev = torch.empty((self.count, hlf.REDUCE_WORDS), dtype=torch.int64, device=device)

    def run(self, cap: int, stream=None, ranks: bool = False):
        """Enqueue every matrix's two launches; with ranks=True also wait for
        and return each rank (for tests; the timed path does not)."""
        out = np.zeros(self.count, dtype=np.int32) if ranks else None
        for b in range(self.count):
            h = hlf.hlf_factor(self.views[b], self.ns[b], stream)
            hlf.hlf_enumerate_reduce_upto(h, cap, self.red_dev[b], stream)
            if ranks:
                out[b] = hlf.hlf_get_rank(h)
            hlf.hlf_destroy(h)
        return out


def per_instance(mats: list[np.ndarray], cap: int, device: str = "cuda"):
    """The plain path run once: (ranks, reduce tensor [count, 18])."""
    p = PlainPath(mats, device)
    ranks = p.run(cap, ranks=True)
    return ranks, p.red_dev


def main(argv=None):
    """Run the batched workload (or its first `--count` grids) once and
    print launch time and throughput; `--tiles WARPS CTAS CHUNK` skips the
    autotuner."""
    import argparse
    import time

    import torch

    from synth import workloads as wl

    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--count", type=int, default=4096)
    ap.add_argument("--cap-log2", type=int, default=wl.BATCH_CAP_LOG2)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--tiles", type=int, nargs=3, default=None)
    a = ap.parse_args(argv)
    mats = wl.batch()[: a.count]
    cap = 1 << a.cap_log2
    B = Batch(mats)
    if a.tiles:
        B.set_tiles(a.tiles[0], a.tiles[1], a.tiles[2])
    else:
        from . import autotune

        autotune.autotune(B, cap, reps=1)
    B.run(cap)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(a.reps):
        B.run(cap)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / a.reps
    st = B.status()
    r, red = B.results()
    sols = sum(x.count for x in red)
    print(f"{len(mats)} grids, tiles {B.tiles}: {1e3 * dt:.3f} ms/launch, {len(mats) / dt:.3e} inst/s, "
          f"{sols / dt:.3e} solutions/s, status {st}")
    B.close()
    return 0 if st == 0 else 1


if __name__ == "__main__":
    import os
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    raise SystemExit(main())
