"""Handles do not leak: thousands of factor / enumerate / destroy cycles, on
one and on several streams, over sizes that take both factor paths, leave
the device's free memory where a first round of the same cycles left it
(the library's stream-ordered pool keeps freed blocks for reuse, so the
first round may grow it, later rounds must not)."""

import numpy as np
import pytest

import paper_2103_00693_gb300 as hlf
import synth

pytestmark = pytest.mark.gpu


def _round(mats, streams, reds, outs):
    import torch

    for k, (A_dev, n) in enumerate(mats):
        i = k % len(streams)  # each stream its own output buffers
        h = hlf.hlf_factor(A_dev, n, streams[i])
        hlf.hlf_enumerate_reduce_upto(h, 1 << 12, reds[i], streams[i])
        hlf.hlf_enumerate_store_upto(h, 1 << 10, outs[i], streams[i])
        hlf.hlf_destroy(h)
    torch.cuda.synchronize()


def test_factor_enumerate_destroy_cycles_do_not_grow_memory(cuda_ok):
    import torch

    rng = np.random.default_rng(5)
    mats = []
    for k in range(200):
        n = int(rng.choice([9, 36, 100, 300, 450, 700, 1024]))
        A = synth.random_symmetric(n, 0.5, 1000 + k)
        mats.append((torch.from_numpy(hlf.pack_rows(A).view(np.int64)).cuda(), n))
    streams = [torch.cuda.current_stream()] + [torch.cuda.Stream() for _ in range(3)]
    reds = [torch.empty(hlf.REDUCE_WORDS, dtype=torch.int64, device="cuda") for _ in streams]
    outs = [torch.empty((1 << 10) * 16, dtype=torch.int64, device="cuda") for _ in streams]
    _round(mats, streams, reds, outs)  # warms the pool
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(10):  # 2000 further factorisations
        _round(mats, streams, reds, outs)
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 < (64 << 20), (free0, free1)  # no growth beyond pool rounding
    many = hlf.hlf_many_create(64)
    hlf.hlf_many_destroy(many)
    for _ in range(200):
        hlf.hlf_many_destroy(hlf.hlf_many_create(64))
    torch.cuda.synchronize()
    assert free0 - torch.cuda.mem_get_info()[0] < (64 << 20)
