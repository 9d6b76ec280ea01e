"""Stage 2 on the GPU (store, reduce, chunked reduce, sample) against the
oracle, element by element and bit-exact, over windows that span many tiles
with ragged heads and tails, odd offsets, empty windows, tiny ranks, every
word count W = 1..16, and ranks above 64."""

import numpy as np
import pytest

import paper_2103_00693_gb300 as hlf
import synth
from oracle import cpu as oc

pytestmark = pytest.mark.gpu


def _instance(kind):
    if kind == "r0":
        return np.zeros((9, 9), dtype=np.uint8)
    if kind == "r1":
        A = np.zeros((6, 6), dtype=np.uint8)
        A[4, 4] = 1
        return A
    if kind == "r2":
        return synth.all_connected(2, "0000")
    if kind == "r5":
        A = np.zeros((8, 8), dtype=np.uint8)
        A[np.arange(5), np.arange(5)] = 1
        return A
    if kind == "grid6":
        return synth.grid_instance(6, 1.0, 3)
    if kind == "grid8":
        return synth.grid_instance(8, 0.5, 0)
    if kind.startswith("W"):  # a random grid whose rows take W words
        W = int(kind[1:])
        n = 64 * (W - 1) + 37 if W > 1 else 40
        A = synth.random_symmetric(n, 0.02, 77 + W)
        return A
    raise KeyError(kind)


KINDS = ["r0", "r1", "r2", "r5", "grid6", "grid8"] + [f"W{w}" for w in range(1, 17)]


@pytest.fixture(scope="module")
def factored(cuda_ok):
    out = {}
    for k in KINDS:
        A = _instance(k)
        out[k] = (oc.factor(A), hlf.Factorization.from_dense(A))
    yield out
    for _, G in out.values():
        G.close()


def _windows(space_log2):
    space = 1 << space_log2
    w = [(0, 0), (0, 1), (0, min(space, 5))]
    for off, cnt in ((0, 4096), (1, 4095), (3, 333), (63, 130), (64, 64), (65, 1000), (101, 20000),
                     (space - 1000, 1000), (space - 65, 65), (space // 3, 7777)):
        off = max(0, min(off, space - 1))
        cnt = max(0, min(cnt, space - off))
        w.append((off, cnt))
    w.append((0, space) if space <= (1 << 16) else (space - (1 << 16), 1 << 16))
    return w


@pytest.mark.parametrize("kind", KINDS)
def test_store_windows(factored, kind):
    import torch

    F, G = factored[kind]
    assert G.rank == F.r
    for off, cnt in _windows(F.space_log2()):
        out = torch.full((max(cnt, 1) + 1, F.W), -1, dtype=torch.int64, device="cuda")
        G.store(off, cnt, out)
        got = out.cpu().numpy().view(np.uint64)
        want = oc.window(F, off, cnt)
        assert np.array_equal(got[:cnt], want), (kind, off, cnt)
        assert np.all(got[cnt:] == np.uint64(0xFFFFFFFFFFFFFFFF)), "wrote past the window"
    assert G.status() == 0


@pytest.mark.parametrize("kind", KINDS)
def test_reduce_windows(factored, kind):
    F, G = factored[kind]
    for off, cnt in _windows(F.space_log2()) + [(0, min(1 << F.space_log2(), 1 << 22))]:
        red = G.reduce(off, cnt)
        got = hlf.ReduceResult.from_words(red.cpu().numpy(), F.W)
        c, h, f = oc.reduce(F, off, cnt)
        assert (got.count, got.hsum) == (c, h), (kind, off, cnt)
        assert np.array_equal(got.xor_fold, f), (kind, off, cnt)
        assert not red.cpu().numpy()[2 + F.W:].any()


@pytest.mark.parametrize("kind", ["r2", "r5", "grid6", "grid8", "W1", "W3", "W16"])
def test_reduce_chunks(factored, kind):
    F, G = factored[kind]
    space = 1 << F.space_log2()
    for chunk, n_chunks in ((1, 7), (5, 3), (1000, 37), (4096, 16)):
        if chunk * n_chunks > space:
            continue
        off = (space - chunk * n_chunks) // 2
        red = G.reduce_chunks(off, chunk, n_chunks).cpu().numpy()
        total = hlf.ReduceResult.from_words(G.reduce(off, chunk * n_chunks).cpu().numpy(), F.W)
        C, H, X = 0, 0, np.zeros(F.W, dtype=np.uint64)
        for c in range(n_chunks):
            got = hlf.ReduceResult.from_words(red[c], F.W)
            want = oc.reduce(F, off + c * chunk, chunk, 1)
            assert (got.count, got.hsum) == want[:2] and np.array_equal(got.xor_fold, want[2])
            C, H, X = C + got.count, (H + got.hsum) % (1 << 64), X ^ got.xor_fold
        assert (C, H) == (total.count, total.hsum) and np.array_equal(X, total.xor_fold)


@pytest.mark.parametrize("kind", ["r0", "r1", "r5", "grid6", "grid8", "W2", "W7", "W16"])
def test_sample(factored, kind):
    import torch

    F, G = factored[kind]
    space_log2 = F.space_log2()
    idx = synth.sample_indices(8, 3000, 0, 1 << space_log2)
    idx[:3] = [0, (1 << space_log2) - 1, (1 << space_log2) // 2]
    out = G.sample(torch.from_numpy(idx.view(np.int64)).cuda()).cpu().numpy().view(np.uint64)
    for t, i in enumerate(idx):
        assert np.array_equal(out[t], oc.window(F, int(i), 1)[0]), (kind, int(i))
    assert G.status() == 0


def test_sample_out_of_range_sets_status(factored):
    import torch

    F, G = factored["r5"]  # r = 5: indices 0..31
    idx = torch.tensor([3, 32, 5], dtype=torch.int64, device="cuda")
    out = G.sample(idx).cpu().numpy().view(np.uint64)
    assert np.array_equal(out[0], oc.window(F, 3, 1)[0])
    assert not out[1].any()
    assert G.status() == 5
    assert G.status() == 0  # cleared once read


def test_range_errors(factored):
    import torch

    F, G = factored["r5"]
    out = torch.empty((64, 1), dtype=torch.int64, device="cuda")
    for off, cnt in ((0, 33), (32, 1), (31, 2), (2 ** 63, 1)):
        with pytest.raises(hlf.HlfError) as e:
            G.store(off, cnt, out)
        assert e.value.status == 5
        with pytest.raises(hlf.HlfError):
            G.reduce(off, cnt)
    with pytest.raises(hlf.HlfError):
        G.reduce_chunks(0, 16, 3)
    with pytest.raises(hlf.HlfError):
        G.reduce_chunks(0, 0, 3)


def test_rank_above_64_uses_first_64_rows(cuda_ok):
    """r > 64: the index space is [0, 2^64); windows that end exactly at 2^64
    and windows straddling 2^63 match the oracle."""
    import torch

    A = synth.grid_instance(20, 0.5, 1234)
    F = oc.factor(A)
    assert F.r > 64
    G = hlf.Factorization.from_dense(A)
    top = 1 << 64
    for off, cnt in ((top - 1000, 1000), (top - 64, 64), (top - 129, 129), ((1 << 63) - 700, 1400)):
        out = torch.empty((cnt, F.W), dtype=torch.int64, device="cuda")
        G.store(off, cnt, out)
        assert np.array_equal(out.cpu().numpy().view(np.uint64), oc.window(F, off, cnt))
        got = hlf.ReduceResult.from_words(G.reduce(off, cnt).cpu().numpy(), F.W)
        c, h, f = oc.reduce(F, off, cnt)
        assert (got.count, got.hsum) == (c, h) and np.array_equal(got.xor_fold, f)
    with pytest.raises(hlf.HlfError):
        G.store(top - 5, 6, torch.empty((6, F.W), dtype=torch.int64, device="cuda"))
    G.close()


def test_unaligned_output_rejected(factored):
    import torch

    _, G = factored["grid6"]
    buf = torch.empty(64, dtype=torch.int64, device="cuda")
    with pytest.raises(hlf.HlfError) as e:
        hlf.hlf_enumerate_store(G.h, 0, 4, buf[1:])  # 8-byte aligned only
    assert e.value.status == 1


def test_streams_and_events(factored):
    """Work issued on a side stream is ordered by that stream."""
    import torch

    F, G = factored["grid8"]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        out = torch.empty((100000, 1), dtype=torch.int64, device="cuda")
        G.store(12345, 100000, out, stream=s)
        red = G.reduce(12345, 100000, stream=s)
    s.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint64), oc.window(F, 12345, 100000))
    got = hlf.ReduceResult.from_words(red.cpu().numpy(), 1)
    assert (got.count, got.hsum) == oc.reduce(F, 12345, 100000)[:2]
