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
