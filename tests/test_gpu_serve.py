"""The continuous-batching request loop: every served result equals the
plain one-request-at-a-time path (alone) and the oracle, bit-exact, whatever
else was in flight with it (in the mix)."""

import numpy as np
import pytest

import synth
from oracle import cpu as oc
from paper_2103_00693_gb300 import serve

pytestmark = pytest.mark.gpu


def _stream(count, rate, seed, N_hi=12, lo=4, hi=12):
    return synth.poisson_stream(count, rate, 3, N_hi, 0.5, lo, hi, seed)


def test_served_equals_alone_and_oracle(cuda_ok):
    reqs = _stream(80, 5000.0, 7)
    srv = serve.Server(device_bytes=64 << 20, host_bytes=64 << 20)
    st, done = srv.run(reqs)
    srv.close()
    assert st.n_requests == len(done) == len(reqs)
    assert st.launches < len(reqs)  # windows were batched together
    st_plain, alone = serve.run_plain(reqs)
    by_id = {q.id: q for q in alone}
    for q in done:
        a = by_id[q.id]
        assert (q.r, q.offset, q.count) == (a.r, a.offset, a.count)
        assert np.array_equal(q.result, a.result), q.id
        F = oc.factor(q.A)
        off, cnt = serve.window_of(F.r, q.want, q.u)
        assert (F.r, off, cnt) == (q.r, q.offset, q.count)
        assert np.array_equal(q.result, oc.window(F, off, cnt)), q.id


def test_sparse_stream_equals_plain_and_oracle(cuda_ok):
    """A sparse stream (the server idle between most arrivals, one request
    per tick): every result equals the plain path and the oracle."""
    reqs = _stream(24, 300.0, 11)
    srv = serve.Server(device_bytes=64 << 20, host_bytes=64 << 20)
    st, done = srv.run(reqs)
    srv.close()
    assert len(done) == len(reqs) and all(q.outcome == "ok" for q in done)
    _, alone = serve.run_plain(reqs)
    by_id = {q.id: q for q in alone}
    for q in done:
        assert np.array_equal(q.result, by_id[q.id].result), q.id
        F = oc.factor(q.A)
        assert np.array_equal(q.result, oc.window(F, q.offset, q.count)), q.id


def test_served_under_tight_memory_budget(cuda_ok):
    """A budget that fits only a few windows at once still serves everything
    exactly (requests wait for admission)."""
    reqs = _stream(40, 20000.0, 9, N_hi=20, lo=8, hi=14)
    srv = serve.Server(device_bytes=1 << 20, host_bytes=4 << 20)
    st, done = srv.run(reqs)
    srv.close()
    assert len(done) == len(reqs)
    for q in done[:: 5]:
        F = oc.factor(q.A)
        assert np.array_equal(q.result, oc.window(F, q.offset, q.count))


def test_served_large_windows_mixed_sizes(cuda_ok):
    """The served workload's own mix (N up to 32, windows up to 2^24), a
    short stream: results equal the plain path."""
    from synth import workloads as wl

    reqs = wl.stream(12, 200.0)
    srv = serve.Server(device_bytes=4 << 30, host_bytes=4 << 30)
    st, done = srv.run(reqs)
    srv.close()
    _, alone = serve.run_plain(reqs)
    by_id = {q.id: q for q in alone}
    for q in done:
        assert np.array_equal(q.result, by_id[q.id].result)


def _planted_stream(seed=21, rate=4000.0):
    """A Poisson stream with malformed, oversized and cancelled requests
    planted among good ones. Returns (stream, expected outcome by id, ids to
    cancel at admission, ids to cancel once factored, ids whose factor call
    gets an injected allocation failure)."""
    import paper_2103_00693_gb300 as hlf

    reqs = _stream(70, rate, seed)
    expect = {}
    # requests 0 and 1 reach hlf_factor first: their allocations are failed
    nomem = [0, 1]
    for i in nomem:
        expect[i] = ("failed", 6)
    # not symmetric: found by the factor kernel
    A = reqs[5]["A"].copy()
    A[0, A.shape[0] - 1] ^= 1
    reqs[5]["A"] = A
    expect[5] = ("failed", 3)
    # a padding bit past column n in packed rows: found by the factor kernel
    A = reqs[9]["A"]
    w = hlf.pack_rows(A).copy()
    w[2, -1] |= np.uint64(1) << np.uint64(63)
    reqs[9] = dict(reqs[9], A=None, A_words=w, n=A.shape[0])
    assert A.shape[0] % 64
    expect[9] = ("failed", 4)
    # host-side checks
    reqs[13] = dict(reqs[13], A=np.zeros((1100, 1100), dtype=np.uint8))
    expect[13] = ("failed", 2)
    reqs[17] = dict(reqs[17], A=np.ones((4, 5), dtype=np.uint8))
    expect[17] = ("failed", 1)
    reqs[19] = dict(reqs[19], want=0)
    expect[19] = ("failed", 1)
    # a window larger than the device ring: refused, not raised
    reqs[23] = dict(reqs[23], A=synth.grid_instance(10, 0.5, 4), want=1 << 24)
    expect[23] = ("refused", 6)
    # cancelled while waiting (before it arrives)
    for i in (29, 31):
        reqs[i] = dict(reqs[i], t_cancel=reqs[i]["t_arrival"] - 1e-4)
        expect[i] = ("cancelled", 0)
    at_admit, at_factored = [37, 41], [43, 47]
    for i in at_admit + at_factored:
        expect[i] = ("cancelled", 0)
    return reqs, expect, at_admit, at_factored, nomem


@pytest.mark.parametrize("rate", [4000.0, 300.0], ids=["busy", "idle"])
def test_served_failures_and_cancellations(cuda_ok, rate):
    """Malformed, oversized, cancelled and allocation-failed requests in a
    Poisson stream each end alone with their status; every other result is
    bit-exact against the oracle; the rings are empty afterwards and the
    same server then serves a clean stream exactly. No case involves a GPU
    fault: bad inputs are caught by host checks or reported in the request's
    own device status word."""
    import paper_2103_00693_gb300 as hlf

    reqs, expect, at_admit, at_factored, nomem = _planted_stream(rate=rate)
    srv = serve.Server(device_bytes=64 << 20, host_bytes=64 << 20)

    def on_event(kind, q):
        if (kind == "admitted" and q.id in at_admit) or (kind == "factored" and q.id in at_factored):
            srv.cancel(q.id)

    hlf.hlf_debug_fail_allocs(len(nomem))
    try:
        st, done = srv.run(reqs, on_event=on_event)
    finally:
        hlf.hlf_debug_fail_allocs(0)
    assert sorted(q.id for q in done) == [q["id"] for q in reqs]
    by_id = {q.id: q for q in done}
    for i, (outcome, status) in expect.items():
        assert (by_id[i].outcome, by_id[i].status) == (outcome, status), i
        assert by_id[i].result is None
    good = [q for q in done if q.id not in expect]
    assert all(q.outcome == "ok" for q in good)
    assert len(good) == len(reqs) - len(expect)
    assert (st.failed, st.refused, st.cancelled) == (
        sum(o == "failed" for o, _ in expect.values()), sum(o == "refused" for o, _ in expect.values()),
        sum(o == "cancelled" for o, _ in expect.values()))
    for q in good:
        F = oc.factor(q.A)
        off, cnt = serve.window_of(F.r, q.want, q.u)
        assert (q.r, q.offset, q.count) == (F.r, off, cnt)
        assert np.array_equal(q.result, oc.window(F, off, cnt)), q.id
    for ring in (srv.dev_ring, srv.host_ring, srv.in_ring, srv.mat_ring):
        assert ring.used == 0
    # the same server still serves exactly
    clean = _stream(20, 5000.0, 99)
    st2, done2 = srv.run(clean)
    srv.close()
    assert st2.failed == st2.cancelled == st2.refused == 0
    for q in done2:
        F = oc.factor(q.A)
        assert np.array_equal(q.result, oc.window(F, q.offset, q.count)), q.id


def test_plain_path_reports_the_same_failures(cuda_ok):
    """The plain one-at-a-time path ends the same malformed and oversized
    requests with the same statuses (cancellations at admission or once
    factored exist only in the continuous loop)."""
    reqs, expect, at_admit, at_factored, nomem = _planted_stream()
    st, done = serve.run_plain(reqs, device_bytes=64 << 20, host_bytes=64 << 20)
    by_id = {q.id: q for q in done}
    for i, (outcome, status) in expect.items():
        if i in at_admit + at_factored + nomem:
            continue
        assert (by_id[i].outcome, by_id[i].status) == (outcome, status), i
    for q in done:
        if q.id not in expect:
            assert q.outcome == "ok"
