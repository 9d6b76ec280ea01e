"""The paper's own enumeration order on the GPU (Section 2, Eq. 3 with the
binary counter of Section 4; hlf_set_order(h, HLF_ORDER_PAPER)) against the
oracle's literal restatement (y = A R per counter value), bit-exact: stored
windows, reduces, samples and the many-window path. Over a full index space
the paper order and the Gray order give the same set."""

import numpy as np
import pytest

import paper_2103_00693_gb300 as hlf
import synth
from oracle import cpu as oc
from oracle import definitional as od

pytestmark = pytest.mark.gpu

KINDS = {
    "grid3": lambda: synth.grid_instance(3, 0.5, 5),
    "paper4-11": lambda: synth.all_connected(4, "0" * 14 + "11"),
    "grid6": lambda: synth.grid_instance(6, 1.0, 3),
    "grid8": lambda: synth.grid_instance(8, 0.5, 0),
    "sym100": lambda: synth.random_symmetric(100, 0.05, 9),
    "grid20_r_gt_64": lambda: synth.grid_instance(20, 0.5, 1234),
    "zero": lambda: np.zeros((7, 7), dtype=np.uint8),
}


@pytest.fixture(scope="module")
def pairs(cuda_ok):
    out = {}
    for k, mk in KINDS.items():
        A = mk()
        F = oc.factor(A)
        G = hlf.Factorization.from_dense(A)
        G.set_order(hlf.ORDER_PAPER)
        out[k] = (F, G)
    yield out
    for _, G in out.values():
        G.close()


def _reduce_of(rows):
    words = [tuple(int(x) for x in r) for r in rows]
    hs = sum(od.chain_hash(w) for w in words) % (1 << 64)
    fold = np.zeros(rows.shape[1], dtype=np.uint64)
    for r in rows:
        fold ^= r
    return len(words), hs, fold


@pytest.mark.parametrize("kind", list(KINDS))
def test_paper_order_windows(pairs, kind):
    import torch

    F, G = pairs[kind]
    space = 1 << F.space_log2()
    for off, cnt in ((0, 1), (0, 700), (3, 129), (space // 3, 4097), (space - 600, 600)):
        off = max(0, min(off, space - 1))
        cnt = min(cnt, space - off)
        want = oc.paper_order(F, off, cnt)
        out = G.store(off, cnt).cpu().numpy().view(np.uint64)
        assert np.array_equal(out, want), (kind, off, cnt)
        red = hlf.ReduceResult.from_words(G.reduce(off, cnt).cpu().numpy(), F.W)
        c, h, f = _reduce_of(want)
        assert (red.count, red.hsum) == (c, h) and np.array_equal(red.xor_fold, f)
        idx = np.array([off, off + cnt - 1, off + cnt // 2], dtype=np.uint64)
        smp = G.sample(torch.from_numpy(idx.view(np.int64)).cuda()).cpu().numpy().view(np.uint64)
        for t, i in enumerate(idx):
            assert np.array_equal(smp[t], oc.paper_order(F, int(i), 1)[0])
    assert G.status() == 0


@pytest.mark.parametrize("kind", ["grid3", "paper4-11", "zero"])
def test_paper_order_full_set_equals_gray_set(pairs, kind):
    F, G = pairs[kind]
    k = 1 << F.r
    paper = G.store(0, k).cpu().numpy().view(np.uint64)
    gray = oc.window(F, 0, k)
    assert sorted(map(tuple, paper.tolist())) == sorted(map(tuple, gray.tolist()))
    assert len(set(map(tuple, paper.tolist()))) == k


def test_paper_order_many_windows(pairs):
    import torch

    m = hlf.hlf_many_create(8)
    F, G = pairs["grid8"]
    F2, G2 = pairs["sym100"]
    outs = [torch.empty((5000, 1), dtype=torch.int64, device="cuda"),
            torch.empty((777, F2.W), dtype=torch.int64, device="cuda")]
    hlf.hlf_enumerate_store_many(m, [G.h, G2.h], [12345, 99], [5000, 777], outs)
    torch.cuda.synchronize()
    assert np.array_equal(outs[0].cpu().numpy().view(np.uint64), oc.paper_order(F, 12345, 5000))
    assert np.array_equal(outs[1].cpu().numpy().view(np.uint64), oc.paper_order(F2, 99, 777))
    hlf.hlf_many_destroy(m)


def test_order_switch_back_to_gray(pairs):
    F, G = pairs["grid6"]
    G.set_order(hlf.ORDER_GRAY)
    assert np.array_equal(G.store(100, 300).cpu().numpy().view(np.uint64), oc.window(F, 100, 300))
    G.set_order(hlf.ORDER_PAPER)
    with pytest.raises(hlf.HlfError):
        hlf.hlf_set_order(G.h, 7)
