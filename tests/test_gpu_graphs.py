"""Beyond grids (§5: the scheme holds for any symmetric A) and at full size.

* App. B's closed form on the GPU for every all-connected grid up to 32 x 32
  (n = 1024): r = n - N for b = 0, and n - N <= r <= n for random b. This
  needs no oracle.
* Random d-regular graphs up to n = 1024, factored and enumerated on the GPU,
  against the oracle."""

import numpy as np
import pytest

import paper_2103_00693_gb300 as hlf
import synth
from oracle import cpu as oc

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N", list(range(2, 33)))
def test_appB_rank_on_gpu(cuda_ok, N):
    n = N * N
    G = hlf.Factorization.from_dense(synth.all_connected(N, "0" * n))
    assert G.rank == n - N
    G.close()
    for seed in range(2):
        G = hlf.Factorization.from_dense(synth.grid_instance(N, 1.0, 1000 * N + seed))
        assert n - N <= G.rank <= n
        G.close()


@pytest.mark.parametrize("n,d", [(16, 3), (64, 3), (65, 4), (200, 3), (511, 4), (1024, 3), (1000, 6)])
def test_random_regular_against_oracle(cuda_ok, n, d):
    import torch

    A = synth.random_regular(n, d, n + d)
    F = oc.factor(A)
    G = hlf.Factorization.from_dense(A)
    assert G.rank == F.r
    piv, z0, basis = G.factor_host()
    assert np.array_equal(basis, F.basis_words()) and np.array_equal(z0, F.z0_words())
    space = 1 << F.space_log2()
    off = space // 7
    cnt = min(20000, space - off)
    assert np.array_equal(G.store(off, cnt).cpu().numpy().view(np.uint64), oc.window(F, off, cnt))
    red = hlf.ReduceResult.from_words(G.reduce(off, cnt).cpu().numpy(), F.W)
    c, h, f = oc.reduce(F, off, cnt)
    assert (red.count, red.hsum) == (c, h) and np.array_equal(red.xor_fold, f)
    G.close()
