"""A seeded sweep over random symmetric matrices (a stand-in for
property-based fuzzing, which the GPU machine's Python lacks): n drawn over
[1, 1024] with the word boundaries and the two factor paths' boundary
favoured, densities from nearly empty to nearly full. Each instance is
checked against the oracle, bit-exact: stage 1 (r, pivots, basis, z^a), a
random window stored and reduced, random sampled indices, and, where the
rank allows, a window that straddles index 2^32."""

import numpy as np
import pytest

import paper_2103_00693_gb300 as hlf
import synth
from oracle import cpu as oc

pytestmark = pytest.mark.gpu

_BOUNDARY_N = [1, 2, 63, 64, 65, 127, 128, 129, 255, 256, 257, 383, 384, 385, 511, 512, 513, 1023, 1024]


def _cases(count=48, seed=2103):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(rng.choice(_BOUNDARY_N)) if k % 3 == 0 else int(rng.integers(1, 1025))
        p = float(rng.choice([0.002, 0.02, 0.1, 0.5, 0.9, 0.995]))
        out.append((k, n, p, int(rng.integers(1 << 30))))
    return out


def _window(rng, space_log2, cap):
    space = 1 << space_log2
    cnt = int(min(space, rng.integers(1, cap + 1)))
    off = int.from_bytes(rng.bytes(9), "little") % (space - cnt + 1)  # spaces up to 2^64
    return off, cnt


@pytest.mark.parametrize("k,n,p,seed", _cases(), ids=[f"{k}-n{n}-p{p}" for k, n, p, _ in _cases()])
def test_random_instance_against_oracle(cuda_ok, k, n, p, seed):
    import torch

    A = synth.random_symmetric(n, p, seed)
    F = oc.factor(A)
    G = hlf.Factorization.from_dense(A)
    rng = np.random.default_rng(seed)
    try:
        assert G.rank == F.r
        piv, z0, basis = G.factor_host()
        assert np.array_equal(piv, F.piv) and np.array_equal(z0, F.z0_words())
        assert np.array_equal(basis, F.basis_words())
        s = F.space_log2()
        windows = [_window(rng, s, 5000), _window(rng, s, 70)]
        if s >= 33:  # a window across index 2^32
            windows.append(((1 << 32) - 1500, 3000))
        for off, cnt in windows:
            out = G.store(off, cnt)
            assert np.array_equal(out.cpu().numpy().view(np.uint64), oc.window(F, off, cnt)), (off, cnt)
            got = hlf.ReduceResult.from_words(G.reduce(off, cnt).cpu().numpy(), F.W)
            c, h, f = oc.reduce(F, off, cnt, 1)
            assert (got.count, got.hsum) == (c, h) and np.array_equal(got.xor_fold, f), (off, cnt)
        idx = synth.sample_indices(seed % 1000, 64, 0, 1 << s)
        smp = G.sample(torch.from_numpy(idx.view(np.int64)).cuda()).cpu().numpy().view(np.uint64)
        for t, i in enumerate(idx):
            assert np.array_equal(smp[t], oc.window(F, int(i), 1)[0]), int(i)
        assert G.status() == 0
    finally:
        G.close()
