"""The batched persistent launch against the oracle and against the plain
one-matrix-per-launch path: every matrix's result is the same alone and in
the mix (exact), under graph replay, and for bad matrices mixed in; bounded
waits that run out report HLF_ERR_TIMEOUT and leave the context usable."""

import numpy as np
import pytest

import paper_2103_00693_gb300 as hlf
import synth
from oracle import cpu as oc
from paper_2103_00693_gb300 import autotune
from paper_2103_00693_gb300.batch import Batch, per_instance
from synth import workloads as wl

pytestmark = pytest.mark.gpu


def _mix():
    mats = synth.batch_instances(48, 4, 16, 0.5, 77)
    mats += [synth.all_connected(4, b) for b in synth.paper_b_patterns(16)]
    mats += [np.zeros((20, 20), dtype=np.uint8), np.eye(256, dtype=np.uint8), synth.random_symmetric(1, 1.0, 1)]
    mats += [synth.random_symmetric(n, 0.3, n) for n in (63, 64, 65, 128, 129, 200, 255, 256)]
    return mats


def _oracle_expect(A, cap):
    F = oc.factor(A)
    total = min(1 << min(F.r, 64), cap)
    c, h, f = oc.reduce(F, 0, total)
    return F.r, c, h, f


def test_batch_matches_oracle(cuda_ok):
    mats = _mix()
    cap = 1 << 14
    B = Batch(mats)
    B.run(cap)
    assert B.status() == 0
    r, red = B.results()
    for b, A in enumerate(mats):
        rr, c, h, f = _oracle_expect(A, cap)
        assert r[b] == rr, b
        assert (red[b].count, red[b].hsum) == (c, h), b
        assert np.array_equal(red[b].xor_fold, f), b
    B.close()


def test_batch_bad_matrices_fail_alone(cuda_ok):
    good = synth.batch_instances(6, 4, 8, 0.5, 5)
    bad_sym = synth.grid_instance(5, 0.5, 9)
    bad_sym[0, 7] ^= 1
    mats = good[:3] + [bad_sym] + good[3:]
    cap = 1 << 12
    B = Batch(mats)
    B.run(cap)
    assert B.status() == 0
    r, red = B.results()
    assert r[3] == -3
    for b in (0, 1, 2, 4, 5, 6):
        A = mats[b]
        rr, c, h, f = _oracle_expect(A, cap)
        assert r[b] == rr and (red[b].count, red[b].hsum) == (c, h)
    B.close()


def test_batch_tiles_do_not_change_results(cuda_ok):
    mats = synth.batch_instances(64, 4, 16, 0.5, 3)
    cap = 1 << 16
    B = Batch(mats)
    ref = None
    for cps, chunk in ((0, 1 << 16), (1, 1 << 13), (2, 1 << 17), (3, 256)):
        B.set_tiles(cps, chunk)
        B.run(cap)
        assert B.status() == 0
        got = B.red_dev.cpu().numpy().copy()
        if ref is None:
            ref = got
        assert np.array_equal(got, ref)
    B.close()


def test_batch_graph_replay(cuda_ok):
    import torch

    mats = synth.batch_instances(32, 4, 16, 0.5, 8)
    cap = 1 << 15
    B = Batch(mats)
    B.run(cap)
    torch.cuda.synchronize()
    want = B.red_dev.cpu().numpy().copy()
    B.red_dev.zero_()
    B.capture(cap)
    for _ in range(3):
        B.red_dev.fill_(-1)
        B.replay()
        torch.cuda.synchronize()
        assert np.array_equal(B.red_dev.cpu().numpy(), want)
    B.close()


def test_batch_timeout_reports_and_recovers(cuda_ok):
    """Every chunk waits on a flag that nothing sets (the factor items are
    skipped); the bounded waits run out, the status says so, and the next
    normal launch on the same context is exact."""
    mats = synth.batch_instances(4, 4, 6, 0.5, 11)
    B = Batch(mats)
    hlf.hlf_batch_set_spin_limit(B.plan, 200)
    hlf.hlf_batch_set_debug(B.plan, 1)
    B.run(1 << 12)
    assert B.status() == hlf.STATUS_CODES["HLF_ERR_TIMEOUT"]
    hlf.hlf_batch_set_debug(B.plan, 0)
    hlf.hlf_batch_set_spin_limit(B.plan, 1 << 23)
    B.run(1 << 12)
    assert B.status() == 0
    r, red = B.results()
    for b, A in enumerate(mats):
        rr, c, h, _ = _oracle_expect(A, 1 << 12)
        assert r[b] == rr and (red[b].count, red[b].hsum) == (c, h)
    B.close()


def test_batch4096_alone_and_in_the_mix(cuda_ok):
    """The batched workload at full size: 4096 grids, N in 4..16, cap 2^20.
    The one launch equals the per-matrix path for every matrix (exact), and a
    seeded sample of 256 matrices equals the oracle."""
    mats = wl.batch()
    cap = 1 << wl.BATCH_CAP_LOG2
    B = Batch(mats)
    autotune.autotune(B, cap, reps=1, use_cache=False)
    B.run(cap)
    assert B.status() == 0
    r, red = B.results()
    ranks, red_plain = per_instance(mats, cap)
    assert np.array_equal(r, ranks)
    assert np.array_equal(B.red_dev.cpu().numpy(), red_plain.cpu().numpy())
    rng = np.random.default_rng(4096)
    for b in rng.choice(len(mats), size=256, replace=False):
        rr, c, h, f = _oracle_expect(mats[b], cap)
        assert r[b] == rr and (red[b].count, red[b].hsum) == (c, h) and np.array_equal(red[b].xor_fold, f)
    B.close()
