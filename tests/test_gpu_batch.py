"""The batched persistent launches against the oracle and against the plain
one-matrix-per-launch path: every matrix's result is the same alone and in
the mix (exact), in the fused launch and in the two separate calls
(hlf_factor_batched with an offsets table, then hlf_enumerate_batched
reducing or storing), under every launch shape, under graph replay, and for
bad matrices mixed in; bounded waits that run out report HLF_ERR_TIMEOUT and
leave the context usable."""

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
    for warps, cps, chunk in ((8, 0, 1 << 16), (8, 1, 1 << 13), (4, 2, 1 << 17), (2, 3, 256), (2, 0, 1 << 14),
                              (4, 0, 1 << 15)):
        B.set_tiles(warps, cps, chunk)
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


def test_spin_limit_from_the_environment(cuda_ok, monkeypatch):
    """HLF_SPIN_LIMIT sets the bound of every plan the module creates: with
    200 polls and the factor items skipped, the waits run out at once."""
    monkeypatch.setenv("HLF_SPIN_LIMIT", "200")
    B = Batch(synth.batch_instances(4, 4, 6, 0.5, 12))
    hlf.hlf_batch_set_debug(B.plan, 1)
    B.run(1 << 12)
    assert B.status() == hlf.STATUS_CODES["HLF_ERR_TIMEOUT"]
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


@pytest.mark.parametrize("warps", [2, 4, 8])
def test_split_calls_equal_fused_and_oracle(cuda_ok, warps):
    """hlf_factor_batched (n from the offsets table) + hlf_enumerate_batched
    reduce equal the fused launch and the oracle for every matrix of the mix
    (n = 1 .. 256, W = 1 .. 4, rank 0 .. n)."""
    mats = _mix()
    cap = 1 << 13
    B = Batch(mats)
    B.set_tiles(warps, 0, 1 << 12)
    B.run(cap)
    assert B.status() == 0
    fused_r = B.r_dev.cpu().numpy().copy()
    fused = B.red_dev.cpu().numpy().copy()
    B.r_dev.fill_(-99)
    B.red_dev.fill_(-1)
    B.factor()
    B.reduce(cap)
    assert B.status() == 0
    assert np.array_equal(B.r_dev.cpu().numpy(), fused_r)
    assert np.array_equal(B.red_dev.cpu().numpy(), fused)
    r, red = B.results()
    for b in range(0, len(mats), 3):
        rr, c, h, f = _oracle_expect(mats[b], cap)
        assert r[b] == rr and (red[b].count, red[b].hsum) == (c, h) and np.array_equal(red[b].xor_fold, f), b
    B.close()


@pytest.mark.parametrize("warps", [2, 8])
def test_batched_store_against_oracle(cuda_ok, warps):
    """hlf_enumerate_batched storing: matrix b writes z(i), i < min(2^r_b,
    cap, room_b), at its offset, W_b words each; nothing past that is
    touched. A ragged cap (not a multiple of 32), rooms smaller than the cap
    and an empty room are included; the same factorisations are reduced
    first and stored after."""
    import torch

    mats = _mix()
    cap = 1000
    B = Batch(mats)
    B.set_tiles(warps, 0, 256)
    B.factor()
    B.reduce(cap)
    want_red = B.red_dev.cpu().numpy().copy()
    Ws = B.Ws.astype(np.int64)
    rooms = np.full(len(mats), cap, dtype=np.int64)
    rooms[1], rooms[4], rooms[7], rooms[-1] = 37, 0, 100, 999
    spare = np.full(len(mats), 5, dtype=np.int64)  # extra words: a room may exceed what is written
    spare[4] = 0  # instance 4 gets an empty region
    sizes = rooms * Ws + spare
    table = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)  # [count + 1]
    out = torch.full((int(table[-1]),), -1, dtype=torch.int64, device="cuda")
    B.store(cap, out, torch.from_numpy(table).cuda())
    assert B.status() == 0
    got = out.cpu().numpy().view(np.uint64)
    starts = table
    for b, A in enumerate(mats):
        F = oc.factor(A)
        room_b = (int(table[b + 1]) - int(table[b])) // int(Ws[b])
        k = min(1 << min(F.r, 64), cap, room_b)
        if b == 4:
            assert k == 0
        if k:
            blk = got[starts[b]: starts[b] + k * Ws[b]].reshape(k, Ws[b])
            assert np.array_equal(blk, oc.window(F, 0, k)), b
        rest = got[starts[b] + k * Ws[b]: starts[b + 1]]
        assert np.all(rest == np.uint64(0xFFFFFFFFFFFFFFFF)), b
    # the store left the factorisations and the earlier reduce intact
    B.reduce(cap)
    assert np.array_equal(B.red_dev.cpu().numpy(), want_red)
    B.close()


def test_factor_batched_bad_sizes_fail_alone(cuda_ok):
    """A matrix whose word count is n * ceil(n/64) for no n <= 256 fails
    alone with HLF_ERR_SIZE; the others are exact."""
    import torch

    mats = synth.batch_instances(5, 4, 8, 0.5, 12)
    packed = [hlf.pack_rows(A).ravel() for A in mats]
    junk = np.zeros(65, dtype=np.uint64)  # 65 words: no n has that size
    parts = packed[:2] + [junk] + packed[2:]
    sizes = [len(p) for p in parts]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    A_dev = torch.from_numpy(np.concatenate(parts).view(np.int64)).cuda()
    plan = hlf.hlf_batch_create(len(parts))
    r = torch.empty(len(parts), dtype=torch.int32, device="cuda")
    red = torch.empty((len(parts), hlf.REDUCE_WORDS), dtype=torch.int64, device="cuda")
    hlf.hlf_factor_batched(plan, A_dev, torch.from_numpy(offs).cuda(), len(parts), r)
    hlf.hlf_enumerate_batched(plan, 1 << 10, red_dev=red)
    assert hlf.hlf_batch_get_status(plan) == 0
    rr = r.cpu().numpy()
    assert rr[2] == -hlf.STATUS_CODES["HLF_ERR_SIZE"]
    assert not red[2].cpu().numpy().any()
    for b, A in zip([0, 1, 3, 4, 5, 6], mats):
        want = _oracle_expect(A, 1 << 10)
        got = hlf.ReduceResult.from_words(red[b].cpu().numpy(), hlf.words(A.shape[0]))
        assert rr[b] == want[0] and (got.count, got.hsum) == want[1:3], b
    hlf.hlf_batch_destroy(plan)


def test_enumerate_batched_needs_a_factorisation(cuda_ok):
    import torch

    plan = hlf.hlf_batch_create(4)
    red = torch.empty((4, hlf.REDUCE_WORDS), dtype=torch.int64, device="cuda")
    with pytest.raises(hlf.HlfError) as e:
        hlf.hlf_enumerate_batched(plan, 16, red_dev=red)
    assert e.value.status == hlf.STATUS_CODES["HLF_ERR_ARG"]
    hlf.hlf_batch_destroy(plan)
