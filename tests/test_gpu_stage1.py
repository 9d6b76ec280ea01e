"""Stage 1 on the GPU (hlf_factor) against the oracle, bit-exact: rank,
pivot columns, RREF basis rows and z^a, plus the device-side input checks."""

import numpy as np
import pytest

import paper_2103_00693_gb300 as hlf
import synth
from oracle import cpu as oc

pytestmark = pytest.mark.gpu


def _cases():
    c = []
    for N in (2, 3, 4, 5, 6, 8, 11, 16, 23, 32):
        c.append((f"grid{N}-p.5", synth.grid_instance(N, 0.5, 10 + N)))
        c.append((f"grid{N}-full", synth.grid_instance(N, 1.0, 20 + N)))
    for N in (2, 3, 4, 5):
        for b in synth.paper_b_patterns(N * N):
            c.append((f"paper{N}-{b[-2:]}", synth.all_connected(N, b)))
    # W boundaries and general symmetric matrices (§5: any symmetric A)
    for n in (1, 2, 31, 32, 33, 63, 64, 65, 127, 128, 129, 200, 511, 512, 513, 777, 1023, 1024):
        c.append((f"sym{n}", synth.random_symmetric(n, 0.3, n)))
    for n in (1, 64, 100, 1024):
        c.append((f"zero{n}", np.zeros((n, n), dtype=np.uint8)))
        c.append((f"eye{n}", np.eye(n, dtype=np.uint8)))
    for n in (192, 193, 250, 256, 257, 320):  # the one-CTA path's last widths (W <= 4), the panel path's first
        c.append((f"sym{n}", synth.random_symmetric(n, 0.5, n)))
    # pivots only among late rows: the first rows and columns are zero
    for n, z in ((40, 33), (100, 50), (256, 200), (700, 600)):
        A = synth.random_symmetric(n, 0.5, n + z)
        A[:z, :] = 0
        A[:, :z] = 0
        c.append((f"late{n}-{z}", A))
    # low rank: A = X X^T mod 2 with X of k columns
    rng = np.random.default_rng(7)
    for n, k in ((64, 5), (200, 17), (1024, 40)):
        X = rng.integers(0, 2, size=(n, k), dtype=np.int64)
        c.append((f"lowrank{n}-{k}", ((X @ X.T) & 1).astype(np.uint8)))
    c.append(("sparse300", synth.random_symmetric(300, 0.01, 3)))
    c.append(("dense1000", synth.random_symmetric(1000, 0.9, 4)))
    # the panel path from its lower end (W = 5: n = 257..320) to W = 8, and
    # the word boundaries on the way
    for N in (17, 18, 20, 22):
        c.append((f"grid{N}-p.5", synth.grid_instance(N, 0.5, 30 + N)))
        c.append((f"grid{N}-full", synth.grid_instance(N, 1.0, 40 + N)))
    for n in (258, 288, 321, 384, 385, 448, 449):
        c.append((f"sym{n}", synth.random_symmetric(n, 0.5, n)))
    A = synth.random_symmetric(300, 0.5, 71)
    A[:270, :] = 0
    A[:, :270] = 0
    c.append(("late300-270", A))
    X = np.random.default_rng(9).integers(0, 2, size=(280, 10), dtype=np.int64)
    c.append(("lowrank280-10", ((X @ X.T) & 1).astype(np.uint8)))
    c.append(("zero260", np.zeros((260, 260), dtype=np.uint8)))
    c.append(("eye330", np.eye(330, dtype=np.uint8)))
    A = synth.random_symmetric(500, 0.5, 77)
    A[:400, :] = 0
    A[:, :400] = 0
    c.append(("late500-400", A))
    X = np.random.default_rng(8).integers(0, 2, size=(450, 12), dtype=np.int64)
    c.append(("lowrank450-12", ((X @ X.T) & 1).astype(np.uint8)))
    c.append(("zero400", np.zeros((400, 400), dtype=np.uint8)))
    c.append(("eye450", np.eye(450, dtype=np.uint8)))
    return c


CASES = _cases()


@pytest.mark.parametrize("name,A", CASES, ids=[c[0] for c in CASES])
def test_factor_parity(cuda_ok, name, A):
    F = oc.factor(A)
    G = hlf.Factorization.from_dense(A)
    try:
        assert G.rank == F.r
        piv, z0, basis = G.factor_host()
        assert np.array_equal(piv, F.piv)
        assert np.array_equal(z0, F.z0_words())
        assert np.array_equal(basis, F.basis_words())
        assert G.status() == 0
    finally:
        G.close()


def test_factor_rejects_non_symmetric(cuda_ok):
    A = synth.grid_instance(5, 0.5, 1)
    A[3, 17] ^= 1
    G = hlf.Factorization.from_dense(A)
    with pytest.raises(hlf.HlfError) as e:
        G.rank
    assert e.value.status == 3
    G.close()


ASYM = [(64, 0, 63), (64, 40, 7), (100, 99, 64), (100, 64, 99), (100, 70, 10),
        (1000, 0, 999), (1000, 999, 0), (1000, 500, 501), (1000, 37, 485), (1000, 63, 64),
        (1000, 960, 999), (1000, 33, 2), (1024, 1023, 1022), (1024, 96, 1000),
        (300, 299, 257), (300, 10, 290)]


@pytest.mark.parametrize("n,i,j", ASYM, ids=[f"n{n}-{i}-{j}" for n, i, j in ASYM])
def test_factor_finds_one_asymmetric_bit(cuda_ok, n, i, j):
    """A single flipped bit A[i][j] (i != j) is found wherever it lies: in a
    diagonal or off-diagonal 64 x 64 block, above or below the diagonal, in
    either half of a block's rows, next to the padding."""
    A = synth.random_symmetric(n, 0.3, n + i)
    A[i, j] ^= 1
    G = hlf.Factorization.from_dense(A)
    try:
        with pytest.raises(hlf.HlfError) as e:
            G.rank
        assert e.value.status == 3
    finally:
        G.close()


def test_factor_padding_wins_over_asymmetry(cuda_ok):
    import torch

    n = 1000
    A = synth.random_symmetric(n, 0.3, 11)
    A[5, 900] ^= 1  # not symmetric
    packed = hlf.pack_rows(A)
    packed[999, 15] |= np.uint64(1) << np.uint64(63)  # and a padding bit (column 1023)
    h = hlf.hlf_factor(torch.from_numpy(packed.view(np.int64)).cuda(), n)
    try:
        with pytest.raises(hlf.HlfError) as e:
            hlf.hlf_get_rank(h)
        assert e.value.status == 4
    finally:
        hlf.hlf_destroy(h)


def test_factor_rejects_padding_bits(cuda_ok):
    import torch

    A = synth.grid_instance(5, 0.5, 2)  # n = 25, one word per row
    packed = hlf.pack_rows(A)
    packed[7, 0] |= np.uint64(1) << np.uint64(40)
    A_dev = torch.from_numpy(packed.view(np.int64)).cuda()
    h = hlf.hlf_factor(A_dev, 25)
    with pytest.raises(hlf.HlfError) as e:
        hlf.hlf_get_rank(h)
    assert e.value.status == 4
    hlf.hlf_destroy(h)


def test_factor_size_limits(cuda_ok):
    import torch

    A_dev = torch.zeros((1025, 17), dtype=torch.int64, device="cuda")
    with pytest.raises(hlf.HlfError) as e:
        hlf.hlf_factor(A_dev, 1025)
    assert e.value.status == 2
    with pytest.raises(hlf.HlfError):
        hlf.hlf_factor(A_dev, 0)


def test_many_handles_independent(cuda_ok):
    """Several factorisations in flight on one stream stay independent."""
    mats = [synth.grid_instance(N, 0.5, 900 + N) for N in (3, 7, 12, 20, 31)]
    Gs = [hlf.Factorization.from_dense(A) for A in mats]
    for A, G in zip(mats, Gs):
        F = oc.factor(A)
        piv, z0, basis = G.factor_host()
        assert G.rank == F.r and np.array_equal(basis, F.basis_words()) and np.array_equal(z0, F.z0_words())
        G.close()
