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

from paper_2103_00693_gb300.shard import combine_reduce, shard_items, shard_range
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import synth
    from oracle import cpu as oc

    F = oc.factor(synth.grid_instance(6, 0.5, 42))
    off, cnt = 1000, 200000
    o, c = shard_range(off, cnt, rank, world)
    mine = oc.reduce(F, o, c, 1)
    got = [None] * world
    dist.all_gather_object(got, (mine[0], mine[1], mine[2].tolist()))
    if rank == 0:
        out.put(got)
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_two_ranks_combine():
    import synth
    from oracle import cpu as oc

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    c, h, f = combine_reduce(got)
    F = oc.factor(synth.grid_instance(6, 0.5, 42))
    want = oc.reduce(F, 1000, 200000, 1)
    assert (c, h) == want[:2] and np.array_equal(f, want[2])


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
