"""The N > 1 path on CPU with gloo, world size 2: shards of a window reduce
on separate ranks and combine, over a real process group, to the unsharded
reduce; the benchmark's reference arm prints exactly one line under two
ranks."""

import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2103_00693_gb300.shard import (allgather_combine, pack_partial, reduce_shard, shard_items, shard_range,
                                          unpack_partial)
from tests.conftest import ROOT


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_range_partitions():
    for count in (0, 1, 7, 100, 12345):
        for world in (1, 2, 3, 8):
            parts = [shard_range(50, count, r, world) for r in range(world)]
            assert sum(c for _, c in parts) == count
            at = 50
            for off, c in parts:
                assert off == at
                at += c
    assert shard_items(10, 1, 3) == [1, 4, 7]


def _worker(rank, world, port, out, n, p, seed, off, cnt):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import synth
    from oracle import cpu as oc

    F = oc.factor(synth.grid_instance(n, p, seed))
    # the benchmark's sharded mode runs exactly these two calls, with
    # hlf_enumerate_reduce in place of the oracle's reduce
    part = reduce_shard(lambda o, c: oc.reduce(F, o, c, 1), off, cnt, rank, world)
    got = allgather_combine(part, F.W, world, "cpu")
    out.put((rank, got[0], got[1], got[2].tolist()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("n,p,seed,off,cnt", [(6, 0.5, 42, 1000, 200000), (9, 0.5, 7, 12345, 300001),
                                              (11, 0.5, 3, 0, 99999)])
def test_gloo_two_ranks_combine(n, p, seed, off, cnt):
    """Two gloo ranks each reduce their shard with the oracle and exchange the
    partials with the benchmark's all-gather and combine; both ranks end with
    the unsharded reduce (W = 1 and W = 2)."""
    import synth
    from oracle import cpu as oc

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q, n, p, seed, off, cnt)) for r in range(2)]
    for pr in procs:
        pr.start()
    got = [q.get(timeout=120) for _ in range(2)]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    F = oc.factor(synth.grid_instance(n, p, seed))
    want = oc.reduce(F, off, cnt, 1)
    for _, c, h, f in got:
        assert (c, h) == want[:2] and np.array_equal(np.array(f, dtype=np.uint64), want[2])


def test_partial_pack_round_trip():
    rng = np.random.default_rng(1)
    for W in (1, 3, 16):
        f = rng.integers(0, 1 << 63, size=W, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
        part = ((1 << 64) - 5, (1 << 63) + 7, f)
        c, h, g = unpack_partial(pack_partial(part, W), W)
        assert (c, h) == part[:2] and np.array_equal(g, f)


def test_bench_reference_arm_two_ranks():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={port}", "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
