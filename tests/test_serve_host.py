"""Host-side logic of the request loop (no GPU): window placement inside the
index space, memory accounting, statistics."""

import numpy as np

from paper_2103_00693_gb300 import serve
from synth import workloads as wl


def test_window_of_inside_space():
    rng = np.random.default_rng(0)
    for _ in range(2000):
        r = int(rng.integers(0, 200))
        want = int(rng.integers(1, 1 << 24))
        u = int(rng.integers(0, 1 << 63))
        off, cnt = serve.window_of(r, want, u)
        space = 1 << min(r, 64)
        assert cnt == min(want, space)
        assert 0 <= off and off + cnt <= space


def test_window_of_small_spaces():
    assert serve.window_of(0, 100, 12345) == (0, 1)
    assert serve.window_of(3, 100, 7) == (0, 8)
    assert serve.window_of(3, 5, 7) == (7 % 4, 5)


def test_handle_bytes_grows_with_n():
    assert serve.handle_bytes(9) < serve.handle_bytes(64) < serve.handle_bytes(1024)


def test_stats_summary():
    st = serve.Stats(n_requests=3, solutions=300, bytes_out=2400, makespan_s=2.0,
                     latencies_ms=[1.0, 2.0, 3.0], busy_s=1.0, ticks=2, launches=2)
    s = st.summary()
    assert s["solutions_per_s"] == 150.0 and s["p50_ms"] == 2.0 and s["busy_frac"] == 0.5


def test_stream_workload_shape():
    reqs = wl.stream(50, 1000.0)
    assert len(reqs) == 50
    assert all(9 <= q["A"].shape[0] <= 1024 for q in reqs)
    assert all((1 << 10) <= q["want"] <= (1 << 24) for q in reqs)


def test_ring_blocks_never_overlap():
    """Random allocate/free sequences on the FIFO arena: live blocks stay in
    bounds and disjoint, and everything is reclaimed at the end."""
    import torch

    rng = np.random.default_rng(3)
    ring = serve.Ring(torch.empty(10_240, dtype=torch.int64))
    live = []
    for step in range(20000):
        if live and (rng.random() < 0.45 or len(live) > 40):
            blk = live.pop(int(rng.integers(0, len(live))))
            ring.free(blk)
        else:
            n = int(rng.integers(1, 3000))
            blk = ring.alloc(n)
            if blk is not None:
                assert blk[1] >= n
                live.append(blk)
        spans = sorted((b[0], b[0] + b[1]) for b in live)
        for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
            assert a1 <= b0
        assert all(0 <= a and b <= ring.size for a, b in spans)
    for blk in live:
        ring.free(blk)
    assert ring.used == 0 and ring.alloc(ring.size) is not None


def test_ring_fifo_reuse_and_refusal():
    import torch

    ring = serve.Ring(torch.empty(1024, dtype=torch.int64))
    a = ring.alloc(500)
    b = ring.alloc(500)
    assert a[0] == 0 and b[0] == 512
    assert ring.alloc(100) is None  # full
    ring.free(b)                    # freed out of order: still held by a
    assert ring.alloc(100) is None
    ring.free(a)
    assert ring.alloc(1024)[0] == 0


def test_check_request_statuses():
    """Host-side request checks: each malformed form maps to its status
    before anything reaches the GPU; symmetry and padding are left to the
    factor kernel."""
    ok = np.eye(5, dtype=np.uint8)

    def req(**kw):
        base = dict(id=0, t_arrival=0.0, A=ok, want=4, u=0)
        base.update(kw)
        return serve._mk_reqs([base])[0]

    assert serve.check_request(req())[0] == 0
    assert serve.check_request(req(want=0))[0] == 1
    assert serve.check_request(req(A=np.ones((3, 4), dtype=np.uint8)))[0] == 1
    assert serve.check_request(req(A=2 * ok))[0] == 1
    assert serve.check_request(req(A=np.zeros((0, 0), dtype=np.uint8)))[0] == 2
    assert serve.check_request(req(A=np.zeros((1100, 1100), dtype=np.uint8)))[0] == 2
    asym = ok.copy()
    asym[0, 3] = 1
    assert serve.check_request(req(A=asym))[0] == 0  # the kernel reports it
    words = np.zeros((70, 2), dtype=np.uint64)
    assert serve.check_request(req(A=None, A_words=words, n=70))[0] == 0
    assert serve.check_request(req(A=None, A_words=words, n=71))[0] == 1
    assert serve.check_request(req(A=None, A_words=words[:, :1], n=70))[0] == 1
    assert serve.check_request(req(A=None, A_words=np.zeros((2000, 32), np.uint64), n=2000))[0] == 2
    assert serve.check_request(req(A=None))[0] == 1
