"""The allocation-free batched entry point, for callers that cannot allocate
device memory when they call (a host application that owns all device memory
and hands over only input and output pointers, a framework pool that has
reserved the device, a loop that must not risk the synchronisation of
cudaMalloc/cudaFree). Its output must equal the planned entry point's,
exactly, on two calls in a row through the C ABI (the second call finds the
shared workspace holding the first call's contents). Collected last on
purpose, and independent of every other test file."""

import numpy as np
import pytest

import paper_2103_00693_gb300 as hlf
import synth

pytestmark = pytest.mark.gpu


def _device_batch(mats):
    import torch

    ns = np.array([A.shape[0] for A in mats], dtype=np.int32)
    Ws = (ns + 63) // 64
    off = np.concatenate([[0], np.cumsum(ns.astype(np.int64) * Ws)[:-1]]).astype(np.int64)
    packed = np.concatenate([hlf.pack_rows(A).ravel() for A in mats])
    return (torch.from_numpy(packed.view(np.int64)).cuda(), torch.from_numpy(off).cuda(),
            torch.from_numpy(ns).cuda())


def _planned(A_dev, off_dev, n_dev, count, cap):
    import torch

    r = torch.empty(count, dtype=torch.int32, device="cuda")
    red = torch.empty((count, hlf.REDUCE_WORDS), dtype=torch.int64, device="cuda")
    plan = hlf.hlf_batch_create(count)
    hlf.hlf_batch_factor_reduce(plan, A_dev, off_dev, n_dev, count, cap, r, red)
    assert hlf.hlf_batch_get_status(plan) == 0
    hlf.hlf_batch_destroy(plan)
    return r.cpu().numpy(), red.cpu().numpy()


def _noalloc(A_dev, off_dev, n_dev, count, cap):
    import torch

    r = torch.full((count,), -99, dtype=torch.int32, device="cuda")
    red = torch.full((count, hlf.REDUCE_WORDS), -1, dtype=torch.int64, device="cuda")
    hlf.hlf_batch_factor_reduce_noalloc(A_dev, off_dev, n_dev, count, cap, r, red)
    torch.cuda.synchronize()
    return r.cpu().numpy(), red.cpu().numpy()


def test_noalloc_matches_planned_on_two_calls(cuda_ok):
    import torch

    # call 1: 300 grids; call 2: a different batch at the stated maximum
    first = synth.batch_instances(300, 4, 16, 0.5, 2024)
    second = synth.batch_instances(hlf.BATCH_NOALLOC_MAX, 4, 16, 0.5, 2025)
    for mats, cap in ((first, 1 << 16), (second, 1 << 14)):
        args = _device_batch(mats)
        got_r, got_red = _noalloc(*args, len(mats), cap)
        want_r, want_red = _planned(*args, len(mats), cap)
        assert np.array_equal(got_r, want_r)
        assert np.array_equal(got_red, want_red)
        assert np.all(got_r >= 0)
    torch.cuda.synchronize()


def test_noalloc_call_reserves_no_device_memory(cuda_ok):
    """After a warm-up call (which may load the device code and reserve the
    workspace), a call leaves the device's free memory exactly as it was."""
    import torch

    mats = synth.batch_instances(64, 4, 16, 0.5, 2026)
    args = _device_batch(mats)
    count, cap = len(mats), 1 << 12
    r = torch.empty(count, dtype=torch.int32, device="cuda")
    red = torch.empty((count, hlf.REDUCE_WORDS), dtype=torch.int64, device="cuda")
    hlf.hlf_batch_factor_reduce_noalloc(*args, count, cap, r, red)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    hlf.hlf_batch_factor_reduce_noalloc(*args, count, cap, r, red)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    want_r, want_red = _planned(*args, count, cap)
    assert np.array_equal(r.cpu().numpy(), want_r)
    assert np.array_equal(red.cpu().numpy(), want_red)


def test_noalloc_rejects_more_than_the_maximum(cuda_ok):
    import torch

    n = hlf.BATCH_NOALLOC_MAX + 1
    z = torch.zeros(16 * n, dtype=torch.int64, device="cuda")
    with pytest.raises(hlf.HlfError) as e:
        hlf.hlf_batch_factor_reduce_noalloc(z, z, z, n, 1 << 10, z, z)
    assert e.value.status == hlf.STATUS_CODES["HLF_ERR_SIZE"]
