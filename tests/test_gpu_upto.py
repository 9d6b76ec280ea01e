"""hlf_enumerate_store_upto (every solution of a small instance, the rank read
on the device) against the oracle, bit-exact: the first min(2^r, cap) rows
equal the oracle's window [0, min(2^r, cap)), the rest of the buffer is
untouched, a failed factorisation writes nothing, and a second stream waits
for the factor kernel."""

import numpy as np
import pytest

import paper_2103_00693_gb300 as hlf
import synth
from oracle import cpu as oc

pytestmark = pytest.mark.gpu

SENTINEL = 0x5A5A5A5A5A5A5A5A


def _cases():
    c = [("grid3", synth.grid_instance(3, 0.5, 5)), ("grid4", synth.grid_instance(4, 1.0, 1)),
         ("zero6", np.zeros((6, 6), dtype=np.uint8)), ("eye1", np.eye(1, dtype=np.uint8))]
    for N, b in ((2, "0000"), (3, "101010101")):
        c.append((f"paper{N}", synth.all_connected(N, b)))
    c.append(("sym70", synth.random_symmetric(70, 0.03, 70)))  # W = 2, r = 58
    c.append(("sym130", synth.random_symmetric(130, 0.01, 130)))  # W = 3, r = 82
    rng = np.random.default_rng(3)
    X = rng.integers(0, 2, size=(1000, 10), dtype=np.int64)
    c.append(("lowrank1000", ((X @ X.T) & 1).astype(np.uint8)))  # W = 16, every solution
    return c


def _run(A, cap, stream=None, order=None):
    import torch

    G = hlf.Factorization.from_dense(A)
    try:
        if order is not None:
            G.set_order(order)
        out = torch.full((max(cap, 1), G.W), SENTINEL, dtype=torch.int64, device="cuda")
        hlf.hlf_enumerate_store_upto(G.h, cap, out, stream)
        torch.cuda.synchronize()
        return oc.factor(A), G.rank, out.cpu().numpy().view(np.uint64)
    finally:
        G.close()


@pytest.mark.parametrize("name,A", _cases(), ids=[c[0] for c in _cases()])
def test_upto_all_solutions(cuda_ok, name, A):
    F = oc.factor(A)
    space = 1 << min(F.r, 16)  # all solutions up to r = 16, a prefix above
    for cap in sorted({1, 3, min(space, 64), space, space + 5}):
        F, r, got = _run(A, cap)
        cnt = min(1 << r, cap)
        assert np.array_equal(got[:cnt], oc.window(F, 0, cnt)), (name, cap)
        assert (got[cnt:] == np.uint64(SENTINEL)).all(), (name, cap)


def test_upto_paper_order(cuda_ok):
    A = synth.all_connected(3, "101010101")
    F, r, got = _run(A, 1 << 9, order=hlf.ORDER_PAPER)
    assert np.array_equal(got[:1 << r], oc.paper_order(F, 0, 1 << r))


def test_upto_failed_factor_writes_nothing(cuda_ok):
    import torch

    A = np.zeros((8, 8), dtype=np.uint8)
    A[0, 1] = 1  # not symmetric
    G = hlf.Factorization.from_dense(A)
    try:
        out = torch.full((16, 1), SENTINEL, dtype=torch.int64, device="cuda")
        hlf.hlf_enumerate_store_upto(G.h, 16, out)
        torch.cuda.synchronize()
        assert (out.cpu().numpy().view(np.uint64) == np.uint64(SENTINEL)).all()
        assert G.status() == 3  # HLF_ERR_NOT_SYMMETRIC
    finally:
        G.close()


def test_upto_other_stream_waits_for_factor(cuda_ok):
    import torch

    A = synth.grid_instance(32, 0.5, 9)  # n = 1024: a factor kernel long enough to race
    F = oc.factor(A)
    G = hlf.Factorization.from_dense(A)
    try:
        s = torch.cuda.Stream()
        out = torch.zeros((1 << 12, G.W), dtype=torch.int64, device="cuda")
        hlf.hlf_enumerate_store_upto(G.h, 1 << 12, out, s)
        s.synchronize()
        assert np.array_equal(out.cpu().numpy().view(np.uint64), oc.window(F, 0, 1 << 12))
    finally:
        G.close()


def test_upto_argument_checks(cuda_ok):
    import torch

    A = synth.grid_instance(3, 0.5, 5)
    G = hlf.Factorization.from_dense(A)
    try:
        out = torch.empty((4, 1), dtype=torch.int64, device="cuda")
        with pytest.raises(hlf.HlfError) as e:
            hlf.hlf_enumerate_store_upto(G.h, (1 << 24) + 1, out)
        assert e.value.status == 1
        hlf.hlf_enumerate_store_upto(G.h, 0, None)  # nothing to do
    finally:
        G.close()


def test_many_handles_recycle_status_slots(cuda_ok):
    """More handles than one slab of status slots (4096), created and
    destroyed in turn, half of them used on a second stream: every rank and
    every stored block stays right while slots are recycled."""
    import torch

    A = synth.grid_instance(3, 0.5, 5)
    F = oc.factor(A)
    want = oc.window(F, 0, 1 << F.r)
    A_dev = torch.from_numpy(hlf.pack_rows(A).view(np.int64)).cuda()
    side = torch.cuda.Stream()
    out = torch.empty((1 << 9, 1), dtype=torch.int64, device="cuda")
    for k in range(4500):
        h = hlf.hlf_factor(A_dev, 9)
        if k % 2:
            hlf.hlf_enumerate_store_upto(h, 1 << 9, out, side)
            side.synchronize()
        else:
            hlf.hlf_enumerate_store_upto(h, 1 << 9, out)
            torch.cuda.synchronize()
        assert hlf.hlf_get_rank(h) == F.r
        if k % 500 == 0:
            assert np.array_equal(out[:1 << F.r].cpu().numpy().view(np.uint64), want)
        hlf.hlf_destroy(h)


@pytest.mark.parametrize("order", [0, 1])
def test_reduce_upto_equals_reduce(cuda_ok, order):
    """hlf_enumerate_reduce_upto (r read on the device) equals
    hlf_enumerate_reduce over [0, min(2^r, cap)) in both orders, for caps
    below, at and above 2^r; a failed factorisation reduces to zeros and its
    fault stays in the status word."""
    import torch

    import paper_2103_00693_gb300 as hlf

    for A in (synth.grid_instance(3, 0.5, 5), synth.grid_instance(5, 0.5, 2), synth.grid_instance(9, 0.5, 1),
              synth.random_symmetric(150, 0.5, 3), np.zeros((7, 7), dtype=np.uint8)):
        F = oc.factor(A)
        G = hlf.Factorization.from_dense(A)
        hlf.hlf_set_order(G.h, order)
        space = 1 << min(F.r, 64)
        for cap in (c for c in (1, 1000, space, 3 * space + 5, 1 << 21) if c < 1 << 64):
            red = torch.empty(hlf.REDUCE_WORDS, dtype=torch.int64, device="cuda")
            hlf.hlf_enumerate_reduce_upto(G.h, cap, red)
            want = G.reduce(0, min(space, cap)).cpu().numpy()
            assert np.array_equal(red.cpu().numpy(), want), (A.shape[0], cap)
        if order == 0:  # the paper order's windows are checked through hlf_enumerate_reduce's own tests
            c, h, f = oc.reduce(F, 0, min(space, 1 << 21))
            got = hlf.ReduceResult.from_words(red.cpu().numpy(), F.W)
            assert (got.count, got.hsum) == (c, h) and np.array_equal(got.xor_fold, f)
        G.close()
    bad = synth.grid_instance(4, 0.5, 3)
    bad[0, 5] ^= 1
    Ab = torch.from_numpy(hlf.pack_rows(bad).view(np.int64)).cuda()
    h = hlf.hlf_factor(Ab, bad.shape[0])
    red = torch.full((hlf.REDUCE_WORDS,), -1, dtype=torch.int64, device="cuda")
    hlf.hlf_enumerate_reduce_upto(h, 1 << 10, red)
    torch.cuda.synchronize()
    assert not red.cpu().numpy().any()
    assert hlf.hlf_get_status(h) == hlf.STATUS_CODES["HLF_ERR_NOT_SYMMETRIC"]
    hlf.hlf_destroy(h)
