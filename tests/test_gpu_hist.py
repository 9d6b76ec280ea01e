"""The on-device histogram of a bit field over a window, against the oracle,
exactly: narrow and wide fields (shared-memory and global bins), fields that
straddle word boundaries, both orders, and the paper's 4 x 4 instance."""

import numpy as np
import pytest

import paper_2103_00693_gb300 as hlf
import synth
from oracle import cpu as oc

pytestmark = pytest.mark.gpu


CASES = [
    ("paper4x4-11", synth.all_connected(4, "0" * 14 + "11"), [(0, 8), (8, 8), (0, 16), (3, 1)]),
    ("grid6", synth.grid_instance(6, 1.0, 3), [(0, 12), (20, 16), (30, 6)]),
    ("grid9", synth.grid_instance(9, 0.5, 4), [(60, 8), (63, 2), (0, 20), (70, 11)]),
    ("sym300", synth.random_symmetric(300, 0.02, 8), [(120, 15), (250, 14), (191, 4)]),
]


@pytest.mark.parametrize("name,A,fields", CASES, ids=[c[0] for c in CASES])
def test_histogram_windows(cuda_ok, name, A, fields):
    F = oc.factor(A)
    G = hlf.Factorization.from_dense(A)
    space = 1 << F.space_log2()
    for order in ("gray", "paper"):
        G.set_order(hlf.ORDER_PAPER if order == "paper" else hlf.ORDER_GRAY)
        for off, cnt in ((0, min(space, 1 << 16)), (max(0, space // 2 - 5000), 30001)):
            cnt = min(cnt, space - off)
            for lo, nb in fields:
                got = G.histogram(off, cnt, lo, nb).cpu().numpy().view(np.uint64)
                want = oc.histogram(F, off, cnt, lo, nb, order)
                assert np.array_equal(got, want), (name, order, off, cnt, lo, nb)
    G.close()


def test_histogram_argument_checks(cuda_ok):
    import torch

    G = hlf.Factorization.from_dense(synth.grid_instance(3, 0.5, 5))  # n = 9
    out = torch.empty(1 << 20, dtype=torch.int64, device="cuda")
    for lo, nb in ((0, 0), (0, 21), (5, 5), (-1, 3)):
        with pytest.raises(hlf.HlfError):
            hlf.hlf_enumerate_histogram(G.h, 0, 4, lo, nb, out)
    G.close()


def _first_rows_independent(F, lo, nb, rows):
    """Whether the field bits [lo, lo + nb) of the enumeration rows 0..4 are
    linearly independent over GF(2) (the kernel then walks lane-interleaved)."""
    vecs = [int(sum(int(b) << j for j, b in enumerate(r[lo:lo + nb]))) for r in rows[:5]]
    if len(vecs) < 5:
        return False
    basis = []
    for v in vecs:
        for b in basis:
            v = min(v, v ^ b)
        if v == 0:
            return False
        basis.append(v)
    return True


@pytest.mark.parametrize("order", ["gray", "paper"])
def test_histogram_both_walks(cuda_ok, order):
    """Fields whose bits over the first five enumeration rows are independent
    (the lane-interleaved walk) and fields where they are not (per-thread
    runs), each against the oracle over windows with ragged ends."""
    A = synth.grid_instance(7, 0.5, 21)
    F = oc.factor(A)
    G = hlf.Factorization.from_dense(A)
    G.set_order(hlf.ORDER_PAPER if order == "paper" else hlf.ORDER_GRAY)
    if order == "gray":  # the enumeration rows are the basis rows B_k
        rows = oc.unpack_rows(F.basis_words(), F.n)
    else:  # row k is T_0 ^ ... ^ T_k, T_l = A's column at the pivot p_{r-1-l}
        rows = np.cumsum(F.A[F.piv[::-1]].astype(np.int64), axis=0) % 2
    seen = set()
    space = 1 << F.space_log2()
    for lo, nb in ((0, 10), (0, 14), (30, 12), (40, 9), (3, 5)):
        seen.add(_first_rows_independent(F, lo, nb, rows))
        for off, cnt in ((0, min(space, 1 << 17)), (12345, 70001)):
            cnt = min(cnt, space - off)
            got = G.histogram(off, cnt, lo, nb).cpu().numpy().view(np.uint64)
            assert np.array_equal(got, oc.histogram(F, off, cnt, lo, nb, order)), (order, lo, nb, off, cnt)
    assert seen == {True, False}, "both walks should be exercised"
    G.close()


def test_histogram_window_ending_at_2_64(cuda_ok):
    """r > 64: the index space is [0, 2^64), and a window may end exactly at
    2^64 (the end wraps to 0 in 64-bit arithmetic); both walks."""
    A = synth.random_symmetric(100, 0.02, 140)
    F = oc.factor(A)
    assert F.r > 64
    G = hlf.Factorization.from_dense(A)
    for cnt in (1, 31, 32, 33, 5000, 70001):
        off = (1 << 64) - cnt
        for lo, nb in ((0, 12), (70, 9), (40, 14)):
            got = G.histogram(off, cnt, lo, nb).cpu().numpy().view(np.uint64)
            assert np.array_equal(got, oc.histogram(F, off, cnt, lo, nb)), (cnt, lo, nb)
    G.close()


def test_atomic_probe_counts_every_atomic(cuda_ok):
    """The shared-memory atomic microbenchmark behind the histogram's
    roofline performs exactly the atomics it reports."""
    import torch

    s = torch.empty(1, dtype=torch.int64, device="cuda")
    for iters in (16, 1 << 10):
        n = hlf.hlf_probe_smem_atomics(iters, s)
        assert int(s.item()) == n > 0
    with pytest.raises(hlf.HlfError):
        hlf.hlf_probe_smem_atomics(15, s)
