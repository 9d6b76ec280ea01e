"""The single-instance workloads at full size, in the launch configuration
the benchmark times.

* grid3x3: every solution, against the oracle and the brute-force set, on
  the headline seed (r = n) and on a seed with r = 6 and z^a != 0, where the
  brute-force comparison is not trivially every string.
* grid6x6: the full 2^36 reduce against the oracle's full reduce (all host
  cores) and the closed forms (count 2^r, XOR-fold 0); the first 2^30
  solutions stored to HBM, checked on sampled blocks against the oracle and on
  a 2^20 sample for validity and index recovery. The same two tests run on a
  seed with r = 34 and z^a != 0 (full 2^34 reduce, first 2^30 stored).
* grid8x8: the 2^40 window reduced whole and in 2^24-solution chunks; chunks
  combine to the whole; 64 seeded chunks against the oracle; 2^20 sampled
  indices checked for validity against Ker(A) and for index recovery on the
  CPU, 4096 of them against the oracle directly.
"""

import numpy as np
import pytest

import paper_2103_00693_gb300 as hlf
import synth
from oracle import cpu as oc
from oracle import definitional as od
from synth import workloads as wl

pytestmark = pytest.mark.gpu


def gray_inverse(g: np.ndarray) -> np.ndarray:
    i = g.copy()
    s = 1
    while s < 64:
        i ^= i >> np.uint64(s)
        s <<= 1
    return i


def check_valid_and_indexed(F, Z_words: np.ndarray, idx: np.ndarray):
    """Every row is a solution (z . x_f = q(x_f)/2 on the oracle's kernel
    basis) and the inverse Gray code of z on P is its index."""
    Zb = oc.unpack_rows(Z_words, F.n)
    par = (Zb.astype(np.int32) @ F.X.T.astype(np.int32)) % 2
    assert np.array_equal(par, np.broadcast_to((F.q // 2).astype(np.int32), par.shape))
    g = np.zeros(len(Zb), dtype=np.uint64)
    for k, p in enumerate(F.piv[:64]):
        g |= Zb[:, p].astype(np.uint64) << np.uint64(k)
    assert np.array_equal(gray_inverse(g), idx.astype(np.uint64))


@pytest.mark.parametrize("which", ["headline", "lowrank"])
def test_grid3x3_all_solutions(cuda_ok, which):
    A = wl.grid3() if which == "headline" else wl.grid3_lowrank()
    F = oc.factor(A)
    G = hlf.Factorization.from_dense(A)
    assert G.rank == F.r
    if which == "lowrank":
        assert F.r == 6 and F.z0.any()
    out = G.store(0, 1 << F.r).cpu().numpy().view(np.uint64)
    assert np.array_equal(out, oc.window(F, 0, 1 << F.r))
    S = od.solutions_bruteforce(A)
    assert sorted(map(od.string_of, hlf.unpack_rows(out, F.n))) == sorted(map(od.string_of, S))
    G.close()


@pytest.fixture(scope="module", params=["headline", "lowrank"])
def grid6(cuda_ok, request):
    A = wl.grid6() if request.param == "headline" else wl.grid6_lowrank()
    F = oc.factor(A)
    if request.param == "lowrank":
        assert F.r == 34 and F.z0.any()
    else:
        assert F.r == 36
    G = hlf.Factorization.from_dense(A)
    yield F, G
    G.close()


def test_grid6x6_full_reduce(grid6):
    F, G = grid6
    assert G.rank == F.r
    got = hlf.ReduceResult.from_words(G.reduce(0, 1 << F.r).cpu().numpy(), F.W)
    assert got.count == 1 << F.r
    assert not got.xor_fold.any()  # affine space of dimension >= 2
    c, h, f = oc.reduce(F, 0, 1 << F.r)
    assert (got.count, got.hsum) == (c, h) and np.array_equal(got.xor_fold, f)


def test_grid6x6_store_first_2_30(grid6):
    import torch

    F, G = grid6
    cnt = 1 << wl.GRID6_STORE_LOG2
    out = torch.empty((cnt, F.W), dtype=torch.int64, device="cuda")
    G.store(0, cnt, out)
    rng = np.random.default_rng(6)
    starts = [0, cnt - 4096] + list(rng.integers(0, cnt - 4096, size=64))
    for s in starts:
        blk = out[int(s):int(s) + 4096].cpu().numpy().view(np.uint64)
        assert np.array_equal(blk, oc.window(F, int(s), 4096)), int(s)
    idx = np.sort(rng.choice(cnt, size=1 << 20, replace=False)).astype(np.int64)
    rows = out[torch.from_numpy(idx).cuda()].cpu().numpy().view(np.uint64)
    check_valid_and_indexed(F, rows, idx.astype(np.uint64))
    del out
    torch.cuda.empty_cache()


def test_grid8x8_window_reduce_and_sample(cuda_ok):
    import torch

    A = wl.grid8()
    F = oc.factor(A)
    G = hlf.Factorization.from_dense(A)
    assert G.rank == F.r
    off, cnt = wl.grid8_window(F.space_log2())
    total = hlf.ReduceResult.from_words(G.reduce(off, cnt).cpu().numpy(), F.W)
    assert total.count == cnt
    chunk = 1 << 24
    nch = cnt // chunk
    parts = G.reduce_chunks(off, chunk, nch).cpu().numpy()
    C, H, X = 0, 0, np.zeros(F.W, dtype=np.uint64)
    for row in parts:
        p = hlf.ReduceResult.from_words(row, F.W)
        C, H, X = C + p.count, (H + p.hsum) % (1 << 64), X ^ p.xor_fold
    assert (C, H) == (total.count, total.hsum) and np.array_equal(X, total.xor_fold)
    rng = np.random.default_rng(8)
    for c in rng.choice(nch, size=64, replace=False):
        p = hlf.ReduceResult.from_words(parts[c], F.W)
        want = oc.reduce(F, off + int(c) * chunk, chunk)
        assert (p.count, p.hsum) == want[:2] and np.array_equal(p.xor_fold, want[2]), int(c)
    idx = wl.grid8_samples(off, cnt)
    out = G.sample(torch.from_numpy(idx.view(np.int64)).cuda()).cpu().numpy().view(np.uint64)
    check_valid_and_indexed(F, out, idx)
    for t in rng.choice(len(idx), size=4096, replace=False):
        assert np.array_equal(out[t], oc.window(F, int(idx[t]), 1)[0])
    assert G.status() == 0
    G.close()


def test_resumable_job_on_the_gpu(cuda_ok):
    """A grid8x8 reduce run as a resumable job: stopped after two chunks,
    checkpointed to JSON, resumed on a fresh factorisation, finished; equal to
    the one-launch reduce of the whole window and to the oracle's."""
    from paper_2103_00693_gb300.job import ReduceJob, gpu_reduce_fn

    A = wl.grid8()
    F = oc.factor(A)
    off, cnt = 12345, (1 << 28) + 77
    job = ReduceJob.start(A, off, cnt, 1 << 26)
    fn, close = gpu_reduce_fn(job)
    job.advance(fn, 2)
    close()
    text = job.to_json()
    resumed = ReduceJob.from_json(text)
    fn2, close2 = gpu_reduce_fn(resumed)
    while not resumed.done():
        resumed.advance(fn2, 3)
    close2()
    c, h, f = resumed.result()
    G = hlf.Factorization.from_dense(A)
    whole = hlf.ReduceResult.from_words(G.reduce(off, cnt).cpu().numpy(), F.W)
    G.close()
    assert (c, h) == (whole.count, whole.hsum) and np.array_equal(f, whole.xor_fold)
    want = oc.reduce(F, off, cnt)
    assert (c, h) == want[:2] and np.array_equal(f, want[2])
