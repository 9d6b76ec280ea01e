"""Many windows of many factorisations (any W) in one launch, against the
oracle window by window, bit-exact."""

import numpy as np
import pytest

import paper_2103_00693_gb300 as hlf
import synth
from oracle import cpu as oc

pytestmark = pytest.mark.gpu


def test_store_many_matches_oracle(cuda_ok):
    import torch

    mats = [synth.grid_instance(N, 0.5, 300 + N) for N in (2, 3, 5, 8, 9, 12, 16, 20, 25, 32)]
    mats += [np.zeros((7, 7), dtype=np.uint8), synth.random_symmetric(130, 0.05, 2)]
    Fs = [oc.factor(A) for A in mats]
    Gs = [hlf.Factorization.from_dense(A) for A in mats]
    m = hlf.hlf_many_create(64)
    rng = np.random.default_rng(1)
    handles, offs, cnts, outs, want = [], [], [], [], []
    for F, G in zip(Fs, Gs):
        space = 1 << F.space_log2()
        for _ in range(3):
            cnt = int(min(space, rng.integers(0, 5000)))
            off = synth.window_offset(int(rng.integers(0, 1 << 30)), F.space_log2(), cnt)
            handles.append(G.h)
            offs.append(off)
            cnts.append(cnt)
            outs.append(torch.full((max(cnt, 1), F.W), -1, dtype=torch.int64, device="cuda"))
            want.append(oc.window(F, off, cnt))
    for rep in range(3):  # the plan's two staging buffers are reused
        for o in outs:
            o.fill_(-1)
        hlf.hlf_enumerate_store_many(m, handles, offs, cnts, outs)
        torch.cuda.synchronize()
        for j, o in enumerate(outs):
            got = o.cpu().numpy().view(np.uint64)
            assert np.array_equal(got[:cnts[j]], want[j]), (rep, j)
    with pytest.raises(hlf.HlfError) as e:
        hlf.hlf_enumerate_store_many(m, [Gs[0].h], [0], [1 << 20], [outs[0]])
    assert e.value.status == 5
    hlf.hlf_many_destroy(m)
    for G in Gs:
        G.close()
