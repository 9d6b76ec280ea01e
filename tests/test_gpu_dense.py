"""The dense bit-stream store (n bits per solution back to back) against the
oracle's definition of the layout, bit-exact: every word count W = 1..16,
odd and unaligned offsets, partial last groups, tiny ranks, r > 64, and the
paper order."""

import numpy as np
import pytest

import paper_2103_00693_gb300 as hlf
import synth
from oracle import cpu as oc

pytestmark = pytest.mark.gpu


def _mats():
    out = [("r0", np.zeros((9, 9), dtype=np.uint8)), ("grid3", synth.grid_instance(3, 0.5, 5)),
           ("grid6", synth.grid_instance(6, 1.0, 3)), ("grid8", synth.grid_instance(8, 0.5, 0)),
           ("grid20", synth.grid_instance(20, 0.5, 1234))]
    for n in (1, 7, 63, 64, 65, 100, 127, 128, 129, 200, 333, 512, 700, 1000, 1024):
        out.append((f"sym{n}", synth.random_symmetric(n, 0.02, 40 + n)))
    return out


MATS = _mats()


@pytest.mark.parametrize("name,A", MATS, ids=[m[0] for m in MATS])
def test_dense_store(cuda_ok, name, A):
    import torch

    F = oc.factor(A)
    G = hlf.Factorization.from_dense(A)
    space = 1 << F.space_log2()
    cases = [(0, 0), (0, 1), (0, min(space, 64)), (0, min(space, 65)), (1, min(space - 1, 200))]
    for off, cnt in ((space // 3, 3001), (space - 777, 777), (5, 4096)):
        off = max(0, min(off, space - 1))
        cases.append((off, min(cnt, space - off)))
    for off, cnt in cases:
        words = hlf.dense_words(cnt, F.n)
        out = torch.full((words + 2,), -1, dtype=torch.int64, device="cuda")
        G.store_dense(off, cnt, out)
        got = out.cpu().numpy().view(np.uint64)
        assert np.array_equal(got[:words], oc.window_dense(F, off, cnt)), (name, off, cnt)
        assert np.all(got[words:] == np.uint64(0xFFFFFFFFFFFFFFFF)), "wrote past the stream"
    G.close()


def test_dense_paper_order(cuda_ok):
    A = synth.grid_instance(7, 0.5, 77)
    F = oc.factor(A)
    G = hlf.Factorization.from_dense(A)
    G.set_order(hlf.ORDER_PAPER)
    got = G.store_dense(1000, 5000).cpu().numpy().view(np.uint64)
    want = oc.dense_stream(oc.unpack_rows(oc.paper_order(F, 1000, 5000), F.n))
    assert np.array_equal(got, want)
    G.close()


def test_dense_grid6_first_2_26(cuda_ok):
    """The grid6x6 store workload in dense form, 2^26 solutions: sampled
    blocks against the oracle."""
    F = oc.factor(synth.grid_instance(6, 1.0, 3))
    G = hlf.Factorization.from_dense(synth.grid_instance(6, 1.0, 3))
    cnt = 1 << 26
    out = G.store_dense(0, cnt).cpu().numpy().view(np.uint64)
    assert len(out) == cnt * 36 // 64
    rng = np.random.default_rng(3)
    for s in [0, cnt - 1024] + list(rng.integers(0, cnt // 1024 - 1, size=32) * 1024):
        s = int(s)
        want = oc.window_dense(F, s, 1024)  # 1024 * 36 bits = 576 whole words
        w0 = s * 36 // 64
        assert np.array_equal(out[w0:w0 + len(want)], want), s
    G.close()


@pytest.mark.parametrize("n", list(range(1, 65)))
def test_dense_one_word_rows(cuda_ok, n):
    """n <= 64, every n: lane runs of M = max(64 / gcd(n, 64), 16) solutions
    (16, 32 or 64), window offsets that are and are not multiples of M, a
    single solution, ragged last passes, and windows long enough that each
    warp walks several passes. Outputs that are 16-byte aligned (full passes
    leave as bulk stores; at n = 64 the packed store runs) and outputs that
    are only 8-byte aligned (the warp copies every pass out itself)."""
    import torch

    A = synth.random_symmetric(n, 0.3, 100 + n)
    F = oc.factor(A)
    G = hlf.Factorization.from_dense(A)
    space = 1 << F.space_log2()
    for k, cnt in enumerate((1, 511, 2049, 70001)):
        cnt = min(cnt, space)
        for aligned in (True, False):
            off = synth.window_offset(100 * n + k, F.space_log2(), cnt)
            off = off & ~63 if aligned else off | 1
            off = min(off, space - cnt)
            words = hlf.dense_words(cnt, n)
            for lead in (0, 1):
                buf = torch.full((words + 3,), -1, dtype=torch.int64, device="cuda")
                G.store_dense(off, cnt, buf[lead:])
                got = buf.cpu().numpy().view(np.uint64)
                assert np.array_equal(got[lead:lead + words], oc.window_dense(F, off, cnt)), (off, cnt, lead)
                assert np.all(got[lead + words:] == np.uint64(0xFFFFFFFFFFFFFFFF)), "wrote past the stream"
                assert np.all(got[:lead] == np.uint64(0xFFFFFFFFFFFFFFFF)), "wrote before the stream"
    G.close()


@pytest.mark.parametrize("n", [100, 129, 1000])
def test_dense_wide_rows_many_groups(cuda_ok, n):
    """n > 64 with windows long enough that every warp places many 64-solution
    groups (the per-lane Gray steps between groups), at an odd offset, with the
    bulk store (n even) and without (n odd): sampled groups against the oracle,
    and the ragged last group."""
    A = synth.random_symmetric(n, 0.02, 500 + n)
    F = oc.factor(A)
    G = hlf.Factorization.from_dense(A)
    cnt = (1 << 22) + 37
    off = synth.window_offset(n, F.space_log2(), cnt) | 1
    off = min(off, (1 << F.space_log2()) - cnt)
    out = G.store_dense(off, cnt).cpu().numpy().view(np.uint64)
    assert len(out) == hlf.dense_words(cnt, n)
    rng = np.random.default_rng(n)
    groups = cnt // 64
    for g in [0, groups - 1] + list(rng.integers(1, groups - 1, size=24)):
        g = int(g)
        want = oc.window_dense(F, off + 64 * g, 64)  # 64 solutions = n whole words
        assert np.array_equal(out[g * n:(g + 1) * n], want), g
    tail = cnt - 64 * groups
    want = oc.window_dense(F, off + 64 * groups, tail)
    assert np.array_equal(out[groups * n:], want)
    G.close()


@pytest.mark.parametrize("n", [65, 77, 100, 127, 128, 129, 130, 193, 200, 255, 256])
def test_dense_group_blocks_aligned(cuda_ok, n):
    """64 < n <= 256 at window offsets that are multiples of 64 (the
    group-block walk: each 64-solution block is the last one XOR a tiled
    step row). Windows from one solution to many groups per warp, ragged last
    groups, windows that cross a multiple of 2^k for large k (steps whose
    tiled row is formed on the fly), 8-byte and 16-byte aligned outputs; the
    whole stream against the oracle and nothing written around it."""
    import torch

    A = synth.random_symmetric(n, 0.3, 900 + n)
    F = oc.factor(A)
    G = hlf.Factorization.from_dense(A)
    lg = F.space_log2()
    space = 1 << lg
    cases = [(0, 1), (0, 63), (0, 64), (64, 65), (0, 70001)]
    for k in (16, 20, lg - 2):  # windows straddling the multiple 2^k of the index
        if k < lg:
            cases.append(((1 << k) - 64 * 300, 64 * 600 + 17))
    cases.append((space - 64 * 200, 64 * 200))  # up to the end of the index space
    for off, cnt in cases:
        assert off % 64 == 0 and off + cnt <= space
        words = hlf.dense_words(cnt, n)
        for lead in (0, 1):
            buf = torch.full((words + 3,), -1, dtype=torch.int64, device="cuda")
            G.store_dense(off, cnt, buf[lead:])
            got = buf.cpu().numpy().view(np.uint64)
            assert np.array_equal(got[lead:lead + words], oc.window_dense(F, off, cnt)), (n, off, cnt, lead)
            assert np.all(got[lead + words:] == np.uint64(0xFFFFFFFFFFFFFFFF)), "wrote past the stream"
            assert np.all(got[:lead] == np.uint64(0xFFFFFFFFFFFFFFFF)), "wrote before the stream"
    G.close()


@pytest.mark.parametrize("n", [65, 130, 256])
def test_dense_group_blocks_long_window(cuda_ok, n):
    """A long aligned window (2^22 + 37 solutions, many groups per warp):
    sampled groups and the ragged last group against the oracle."""
    A = synth.random_symmetric(n, 0.02, 700 + n)
    F = oc.factor(A)
    G = hlf.Factorization.from_dense(A)
    cnt = (1 << 22) + 37
    off = synth.window_offset(n, F.space_log2(), cnt) & ~63
    out = G.store_dense(off, cnt).cpu().numpy().view(np.uint64)
    assert len(out) == hlf.dense_words(cnt, n)
    rng = np.random.default_rng(n)
    groups = cnt // 64
    for g in [0, groups - 1] + list(rng.integers(1, groups - 1, size=24)):
        g = int(g)
        assert np.array_equal(out[g * n:(g + 1) * n], oc.window_dense(F, off + 64 * g, 64)), g
    tail = cnt - 64 * groups
    assert np.array_equal(out[groups * n:], oc.window_dense(F, off + 64 * groups, tail))
    G.close()


@pytest.mark.parametrize("n", [65, 96, 100, 128, 130, 193, 256])
def test_dense_group_blocks_any_offset(cuda_ok, n):
    """64 < n <= 256 at offsets that are not multiples of 64: the window
    starts (offset mod 64) * n bits into its first group block, and every
    stream word is funnel-shifted from two consecutive block words (the last
    from the next group's block). Several residues, windows within one group,
    across one boundary and across many, ending at the end of the index
    space; 8- and 16-byte aligned outputs."""
    import torch

    A = synth.random_symmetric(n, 0.3, 950 + n)
    F = oc.factor(A)
    G = hlf.Factorization.from_dense(A)
    lg = F.space_log2()
    space = 1 << lg
    cases = []
    for o in (1, 7, 33, 63):
        cases += [(o, 1), (o, 64 - o), (o, 65 - o), (64 * 3 + o, 64 * 40 + 11), (o, 70001)]
        cases.append(((1 << 20) + o - 64 * 300, 64 * 600 + 5))
        cases.append((space - 64 * 100 - o, 64 * 100 + o))  # ends at the end of the index space
    for off, cnt in cases:
        assert off % 64 and off + cnt <= space
        words = hlf.dense_words(cnt, n)
        for lead in (0, 1):
            buf = torch.full((words + 3,), -1, dtype=torch.int64, device="cuda")
            G.store_dense(off, cnt, buf[lead:])
            got = buf.cpu().numpy().view(np.uint64)
            assert np.array_equal(got[lead:lead + words], oc.window_dense(F, off, cnt)), (n, off, cnt, lead)
            assert np.all(got[lead + words:] == np.uint64(0xFFFFFFFFFFFFFFFF)), "wrote past the stream"
            assert np.all(got[:lead] == np.uint64(0xFFFFFFFFFFFFFFFF)), "wrote before the stream"
    G.close()


@pytest.mark.parametrize("n", [5, 17, 33, 36, 40, 47])
def test_dense_blocks_small_n_any_offset(cuda_ok, n):
    """n <= 48 at offsets that are not a multiple of the lane-run length:
    blocks of 64 * 2^s solutions (n 2^s words, 128 < n 2^s <= 256), the
    window's shift folded into the step rows. Windows inside one block,
    across one boundary and many, across large powers of two (rows formed on
    the fly) and up to the end of the index space; 8- and 16-byte aligned
    outputs; the whole stream against the oracle, nothing written around it."""
    import torch

    A = synth.random_symmetric(n, 0.5, 970 + n)
    F = oc.factor(A)
    lg = F.space_log2()
    space = 1 << lg
    s = 0
    while (n << (s + 1)) <= 256:
        s += 1
    G = 64 << s
    cases = []
    for o in (1, 3, G // 2 + 1, G - 1):
        for off, cnt in ((o, 1), (o, G - o), (o, G - o + 1), (3 * G + o, 5 * G + 11), (o, 70001)):
            if off + cnt <= space:
                cases.append((off, cnt))
        for k in (lg - 3, lg - 1):
            off = (1 << k) - 4 * G + o
            if k > 0 and off > 0 and off + 8 * G + 3 <= space:
                cases.append((off, 8 * G + 3))
        if space - 2 * G - o > 0:
            cases.append((space - 2 * G - o, 2 * G + o))
    assert cases
    H = hlf.Factorization.from_dense(A)
    for off, cnt in cases:
        words = hlf.dense_words(cnt, n)
        for lead in (0, 1):
            buf = torch.full((words + 3,), -1, dtype=torch.int64, device="cuda")
            H.store_dense(off, cnt, buf[lead:])
            got = buf.cpu().numpy().view(np.uint64)
            assert np.array_equal(got[lead:lead + words], oc.window_dense(F, off, cnt)), (n, off, cnt, lead)
            assert np.all(got[lead + words:] == np.uint64(0xFFFFFFFFFFFFFFFF)), "wrote past the stream"
            assert np.all(got[:lead] == np.uint64(0xFFFFFFFFFFFFFFFF)), "wrote before the stream"
    H.close()
