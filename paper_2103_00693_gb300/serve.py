"""Request loop for the served workload: continuous batching of enumeration
windows on one GPU, and the plain one-request-at-a-time path it is compared
with.

A request carries a matrix A, a wanted window length and a 64-bit draw u.
Once its factorisation is known (rank r), the window is
    count  = min(want, 2^min(r, 64)),
    offset = u mod (2^min(r, 64) - count + 1),
and the solutions z(offset) .. z(offset + count - 1) are returned to the host.

Continuous batching (Server.run):
  * admission in arrival order: a request that has arrived is checked on the
    host (a square 0/1 matrix, n in [1, 1024], want >= 1), its packed matrix
    is carved from a device ring, and its factorisation is launched on one of
    several high-priority factor streams, in turn. A stream's factor kernels
    finish in order, so the loop keeps one queue per factor stream and asks
    only each queue's head whether it is done;
  * admission by device memory: once the rank r is known, the request's
    output window (min(want, 2^min(r,64)) x W words, no more) is reserved in
    the device staging ring and the pinned host ring, in factorisation order;
    a window that does not fit yet waits for earlier ones to leave, and the
    factorisation stays resident (one handle) meanwhile;
  * every tick, all factored windows that got their memory are
    materialised by ONE hlf_enumerate_store_many launch on the enumeration
    stream (hlf_enumerate_store when the tick has one window), into the
    staging ring, while earlier ticks' windows are still being copied out
    and later requests are being factored;
  * each window is copied to its slot of a pinned host ring on a copy stream;
    a request completes when its copy event has fired
    (latency = completion - arrival).
Both rings are allocated once, up front, so the loop itself never allocates
or frees memory (allocation can synchronise the device); handles use the
stream-ordered pool. All solver work runs in the library's kernels; this
module only schedules.

Failure paths. Every request ends in exactly one outcome, and one request's
failure never disturbs another's result:
  * "ok": the window reached the host (q.result);
  * "failed": q.status is the hlf_status that ended it -- a host-side check
    (HLF_ERR_ARG, HLF_ERR_SIZE), a fault the factor kernel found
    (HLF_ERR_NOT_SYMMETRIC, HLF_ERR_PADDING: the problem of Section 1 is
    defined for symmetric A only), or an allocation the library could not
    make (HLF_ERR_NOMEM);
  * "refused": the request can never fit the rings (its packed matrix or its
    window is larger than the ring), status HLF_ERR_NOMEM;
  * "cancelled": Server.cancel(id), or the request's own t_cancel time,
    reached it before its window was launched (waiting, being factored, or
    factored and waiting for memory). A request already launched completes
    normally.
Whatever a request held (ring blocks, its handle) is released when it ends.
"""

from __future__ import annotations

import collections
import contextlib
import gc
import time
from dataclasses import dataclass, field

import numpy as np

from . import hlf


def window_of(r: int, want: int, u: int) -> tuple[int, int]:
    """(offset, count) of a request's window inside [0, 2^min(r, 64))."""
    space = 1 << min(r, 64)
    count = min(want, space)
    return u % (space - count + 1), count


def handle_bytes(n: int) -> int:
    W = hlf.words(n)
    return 64 + 4 * n + 8 * 66 * W + 8 * n * W + 1024


class Ring:
    """FIFO arena over one preallocated 1-D int64 tensor. Blocks are carved
    at the head and reclaimed from the tail in allocation order (a block
    freed early stays reserved until the blocks before it are freed)."""

    ALIGN = 32  # words (256 bytes)

    def __init__(self, buf):
        self.buf = buf
        self.size = buf.numel()
        self.head = 0
        self.tail = 0
        self.live = collections.deque()  # [start, nwords, freed]

    @property
    def used(self) -> int:
        if not self.live:
            return 0
        return (self.head - self.tail) % self.size or self.size

    def alloc(self, nwords: int):
        n = max(self.ALIGN, (nwords + self.ALIGN - 1) // self.ALIGN * self.ALIGN)
        if n > self.size:
            return None
        if not self.live:
            self.head = self.tail = 0
        if self.live and self.head <= self.tail:        # wrapped: free space is [head, tail)
            if self.tail - self.head < n:
                return None
            start = self.head
        elif self.size - self.head >= n:                # free: [head, size) and [0, tail)
            start = self.head
        elif self.tail >= n and self.live:
            start = 0
        else:
            return None
        self.head = start + n
        if self.head == self.size:
            self.head = 0
        blk = [start, n, False]
        self.live.append(blk)
        return blk

    def view(self, blk, nwords: int):
        return self.buf[blk[0]: blk[0] + nwords]

    def free(self, blk):
        blk[2] = True
        while self.live and self.live[0][2]:
            self.live.popleft()
        if self.live:
            self.tail = self.live[0][0]
        else:
            self.head = self.tail = 0


OK, FAILED, CANCELLED, REFUSED = "ok", "failed", "cancelled", "refused"
_ERR_ARG = 1
_ERR_SIZE = 2
_ERR_NOMEM = 6


@dataclass
class Req:
    id: int
    t_arrival: float
    A: np.ndarray | None
    want: int
    u: int
    A_words: np.ndarray | None = None  # packed rows [n][W], given instead of A
    t_cancel: float | None = None
    n: int = 0
    W: int = 0
    r: int = -1
    offset: int = 0
    count: int = 0
    t_done: float = 0.0
    result: np.ndarray | None = None
    outcome: str = ""
    status: int = 0
    state: str = "waiting"  # waiting, factoring, pending, launched, done
    cancel_requested: bool = False
    h: int = 0
    blk_dev: list | None = None
    blk_host: list | None = None
    blk_in: list | None = None
    blk_mat: list | None = None
    A_dev: object = None
    ev_factor: object = None
    ev_copy: object = None
    lane: int = 0  # which factor stream
    packed: np.ndarray | None = None  # the checked, packed rows (set at the first admission attempt)


@dataclass
class Stats:
    n_requests: int = 0
    solutions: int = 0
    bytes_out: int = 0
    makespan_s: float = 0.0
    latencies_ms: list = field(default_factory=list)
    busy_s: float = 0.0
    ticks: int = 0
    launches: int = 0
    failed: int = 0
    cancelled: int = 0
    refused: int = 0

    def summary(self) -> dict:
        lat = np.array(self.latencies_ms) if self.latencies_ms else np.zeros(1)
        return {"requests": self.n_requests, "solutions": self.solutions,
                "solutions_per_s": self.solutions / self.makespan_s if self.makespan_s else 0.0,
                "gb_per_s_to_host": self.bytes_out / self.makespan_s / 1e9 if self.makespan_s else 0.0,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "makespan_s": self.makespan_s,
                "busy_frac": self.busy_s / self.makespan_s if self.makespan_s else 0.0,
                "ticks": self.ticks, "launches": self.launches,
                "failed": self.failed, "cancelled": self.cancelled, "refused": self.refused}


_SPIN_S = 150e-6  # the last stretch before a known arrival is spun, not slept


def _wait_until(t0: float, t: float, cap_s: float = float("inf")):
    """Wait until perf_counter() - t0 >= t, or return after cap_s when t is
    further away: sleep to within _SPIN_S of t, spin the rest. A sleep wakes
    tens of microseconds late, which would add to the latency of the request
    arriving at t. Both the served and the plain loop wait this way."""
    dt = t - (time.perf_counter() - t0)
    if dt > cap_s + _SPIN_S:  # not due yet: one sleep, the caller comes back
        time.sleep(cap_s)
        return
    if dt > _SPIN_S:
        time.sleep(dt - _SPIN_S)
    while time.perf_counter() - t0 < t:
        pass


@contextlib.contextmanager
def _no_gc_pauses():
    """Python's cyclic collector can pause the loop for tens of milliseconds
    when many objects are alive; latency-critical loops keep it off and
    collect afterwards."""
    was = gc.isenabled()
    gc.collect()
    gc.disable()
    try:
        yield
    finally:
        if was:
            gc.enable()


def _mk_reqs(stream: list[dict]) -> list[Req]:
    return [Req(id=q["id"], t_arrival=q["t_arrival"], A=q.get("A"), want=q["want"], u=q["u"],
                A_words=q.get("A_words"), n=int(q.get("n", 0)), t_cancel=q.get("t_cancel"))
            for q in stream]


def check_request(q: Req) -> tuple[int, np.ndarray | None]:
    """Host-side checks of a request before anything is launched: (status,
    packed rows). A dense A must be a square 0/1 matrix; packed rows must be
    [n][W] words; n must lie in [1, 1024]; want must be >= 1. Symmetry and
    padding bits are left to the factor kernel, which reports them in the
    request's own status word."""
    if q.want < 1:
        return _ERR_ARG, None
    if q.A_words is not None:
        w = np.asarray(q.A_words)
        if w.ndim != 2 or w.dtype.itemsize != 8:
            return _ERR_ARG, None
        if not 1 <= q.n <= hlf.MAX_N:
            return _ERR_SIZE, None
        if w.shape != (q.n, hlf.words(q.n)):
            return _ERR_ARG, None
        return 0, np.ascontiguousarray(w).view(np.int64)
    if q.A is None:
        return _ERR_ARG, None
    A = np.asarray(q.A)
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        return _ERR_ARG, None
    q.n = A.shape[0]
    if not 1 <= q.n <= hlf.MAX_N:
        return _ERR_SIZE, None
    if A.size and (A.min() < 0 or A.max() > 1):
        return _ERR_ARG, None
    return 0, hlf.pack_rows(A).view(np.int64)


class Server:
    """Continuous-batching server on the current CUDA device.

    device_bytes: the staging ring (the admission budget for output windows);
    host_bytes:   the pinned host ring the results land in.
    """

    def __init__(self, device_bytes: int = 8 << 30, host_bytes: int = 8 << 30, max_batch: int = 4096,
                 keep_results: bool = True, matrix_bytes: int = 64 << 20):
        import torch

        self.keep = keep_results
        # factorisations: several high-priority streams, so single-CTA factor
        # kernels run side by side and get SMs ahead of the bulk stores
        self.s_factors = [torch.cuda.Stream(priority=-1) for _ in range(4)]
        self._next_factor = 0
        self.s_enum = torch.cuda.Stream()
        self.s_copy = torch.cuda.Stream()
        self.max_batch = max_batch
        self.many = hlf.hlf_many_create(max_batch)
        self.dev_ring = Ring(torch.empty(device_bytes // 8, dtype=torch.int64, device="cuda"))
        self.host_ring = Ring(torch.empty(host_bytes // 8, dtype=torch.int64, pin_memory=True))
        self.in_ring = Ring(torch.empty(matrix_bytes // 8, dtype=torch.int64, pin_memory=True))
        # the packed matrices on the device: carved from a ring as well, so
        # the loop never reaches the allocator (which may synchronise)
        self.mat_ring = Ring(torch.empty(matrix_bytes // 8, dtype=torch.int64, device="cuda"))
        self._cancel: set = set()

    def close(self):
        if self.many:
            hlf.hlf_many_destroy(self.many)
            self.many = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def cancel(self, req_id: int):
        """Ask the running loop to cancel a request. It takes effect at the
        loop's next iteration if the request's window has not been launched
        yet; otherwise the request completes normally."""
        self._cancel.add(req_id)

    # ------------------------------------------------------------ internals

    def _release(self, q: Req):
        """Give back whatever q holds: its handle and its ring blocks."""
        if q.h:
            hlf.hlf_destroy(q.h)
            q.h = 0
        q.A_dev = None
        for ring, name in ((self.in_ring, "blk_in"), (self.mat_ring, "blk_mat"),
                           (self.dev_ring, "blk_dev"), (self.host_ring, "blk_host")):
            blk = getattr(q, name)
            if blk is not None:
                ring.free(blk)
                setattr(q, name, None)

    def _finish(self, q: Req, outcome: str, status: int, st: Stats, done: list, t: float):
        q.outcome, q.status, q.state, q.t_done = outcome, status, "done", t
        if outcome == OK:
            st.latencies_ms.append(1e3 * (q.t_done - q.t_arrival))
            st.solutions += q.count
            st.bytes_out += q.count * q.W * 8
        elif outcome == FAILED:
            st.failed += 1
        elif outcome == CANCELLED:
            st.cancelled += 1
        else:
            st.refused += 1
        done.append(q)
        if self._on_event:
            self._on_event("done", q)

    def _admit(self, q: Req, st: Stats, done: list, t: float) -> bool:
        """Try to admit the head of the waiting queue. Returns False if it
        must wait for ring space; True if it left the queue (admitted, or
        ended by a host-side check or a failed launch)."""
        import torch

        if q.packed is None:  # checked and packed once, not on every retry while the rings are full
            status, q.packed = check_request(q)
            if status:
                self._finish(q, FAILED, status, st, done, t)
                return True
        packed = q.packed
        q.W = hlf.words(q.n)
        nw = q.n * q.W
        if nw > self.in_ring.size or nw > self.mat_ring.size:
            self._finish(q, REFUSED, _ERR_NOMEM, st, done, t)
            return True
        bi = self.in_ring.alloc(nw)
        bm = self.mat_ring.alloc(nw) if bi is not None else None
        if bm is None:
            if bi is not None:
                self.in_ring.free(bi)
            return False
        q.blk_in, q.blk_mat = bi, bm
        staged = self.in_ring.view(bi, nw)
        staged.copy_(torch.from_numpy(packed.ravel()))
        q.lane = self._next_factor
        sf = self.s_factors[q.lane]
        self._next_factor = (self._next_factor + 1) % len(self.s_factors)
        with torch.cuda.stream(sf):
            q.A_dev = self.mat_ring.view(bm, nw).view(q.n, q.W)
            q.A_dev.view(-1).copy_(staged, non_blocking=True)
            try:
                q.h = hlf.hlf_factor(q.A_dev, q.n, sf)
            except hlf.HlfError as e:
                # the copy above may still be reading the staged rows
                sf.synchronize()
                self._release(q)
                self._finish(q, FAILED, e.status, st, done, t)
                return True
            q.ev_factor = torch.cuda.Event()
            q.ev_factor.record(sf)
        q.state = "factoring"
        if self._on_event:
            self._on_event("admitted", q)
        return True

    def _apply_cancels(self, by_id, waiting, pending, st, done, t):
        """End the requests asked to be cancelled that have not been
        launched: a waiting or factored one at once, one being factored once
        its factor kernel is done (its handle and matrix are in use)."""
        if not self._cancel:
            return
        ids, self._cancel = self._cancel, set()
        for i in ids:
            q = by_id.get(i)
            if q is None or q.state in ("launched", "done"):
                continue
            if q.state == "waiting":
                waiting.remove(q)
                self._finish(q, CANCELLED, 0, st, done, t)
            elif q.state == "factoring":
                q.cancel_requested = True
            elif q.state == "pending":
                pending.remove(q)
                self._release(q)
                self._finish(q, CANCELLED, 0, st, done, t)

    def run(self, stream: list[dict], on_event=None) -> tuple[Stats, list[Req]]:
        """Serve `stream` (dicts with id, t_arrival, A or A_words + n, want, u,
        and optionally t_cancel). on_event(kind, req), if given, is called
        with kind "admitted", "factored", "launched" and "done". Returns the
        statistics and every request, in completion order."""
        self._on_event = on_event
        with _no_gc_pauses():
            try:
                return self._run(stream)
            finally:
                self._on_event = None

    def _run(self, stream: list[dict]) -> tuple[Stats, list[Req]]:
        import torch

        reqs = _mk_reqs(stream)
        by_id = {q.id: q for q in reqs}
        waiting = collections.deque(reqs)
        cancels = sorted((q.t_cancel, q.id) for q in reqs if q.t_cancel is not None)
        next_cancel = 0
        # one FIFO per factor stream: a stream's factor kernels finish in
        # order, so only each queue's head needs an event query
        factoring = [collections.deque() for _ in self.s_factors]
        pending: collections.deque = collections.deque()  # factored, waiting for window memory
        copying: list[Req] = []
        done: list[Req] = []
        st = Stats(n_requests=len(reqs))
        t0 = time.perf_counter()
        busy_since = None
        while waiting or any(factoring) or pending or copying:
            now = time.perf_counter() - t0
            # ---- cancellations (timed ones, then those asked through cancel())
            while next_cancel < len(cancels) and cancels[next_cancel][0] <= now:
                self._cancel.add(cancels[next_cancel][1])
                next_cancel += 1
            self._apply_cancels(by_id, waiting, pending, st, done, now)
            # ---- admission: host checks, matrix memory, factor launch
            while waiting and waiting[0].t_arrival <= now:
                if not self._admit(waiting[0], st, done, now):
                    break
                q = waiting.popleft()
                if q.state == "factoring":
                    factoring[q.lane].append(q)
                    if busy_since is None:
                        busy_since = now
            # ---- finished factorisations: rank, or the kernel's fault
            progressed = False
            for fq in factoring:
                while fq and fq[0].ev_factor.query():
                    q = fq.popleft()
                    progressed = True
                    # the factor kernel has read the matrix: its blocks are free
                    self.in_ring.free(q.blk_in)
                    self.mat_ring.free(q.blk_mat)
                    q.blk_in = q.blk_mat = None
                    q.A_dev = None
                    t = time.perf_counter() - t0
                    if q.cancel_requested:
                        self._release(q)
                        self._finish(q, CANCELLED, 0, st, done, t)
                        continue
                    try:
                        q.r = hlf.hlf_get_rank(q.h)
                    except hlf.HlfError as e:
                        self._release(q)
                        self._finish(q, FAILED, e.status, st, done, t)
                        continue
                    q.offset, q.count = window_of(q.r, q.want, q.u)
                    q.state = "pending"
                    pending.append(q)
                    if self._on_event:
                        self._on_event("factored", q)
            # ---- window memory, reserved for the window's actual size
            if self._cancel:
                self._apply_cancels(by_id, waiting, pending, st, done, time.perf_counter() - t0)
            ready = []
            while pending and len(ready) < self.max_batch:
                q = pending[0]
                words = q.count * q.W
                if words > self.dev_ring.size or words > self.host_ring.size:
                    pending.popleft()
                    self._release(q)
                    self._finish(q, REFUSED, _ERR_NOMEM, st, done, time.perf_counter() - t0)
                    continue
                bd = self.dev_ring.alloc(words)
                if bd is None:
                    break
                bh = self.host_ring.alloc(words)
                if bh is None:
                    self.dev_ring.free(bd)
                    break
                q.blk_dev, q.blk_host = bd, bh
                ready.append(pending.popleft())
            if ready:
                torch.cuda.nvtx.range_push("serve.tick")  # one window launch and its copies
                try:
                    if len(ready) == 1:  # one window: the single-window call marshals less
                        q = ready[0]
                        hlf.hlf_enumerate_store(q.h, q.offset, q.count, self.dev_ring.view(q.blk_dev, q.count * q.W),
                                                self.s_enum)
                    else:
                        hlf.hlf_enumerate_store_many(
                            self.many, [q.h for q in ready], [q.offset for q in ready], [q.count for q in ready],
                            [self.dev_ring.view(q.blk_dev, q.count * q.W) for q in ready], self.s_enum)
                except hlf.HlfError as e:
                    t = time.perf_counter() - t0
                    for q in ready:
                        self._release(q)
                        self._finish(q, FAILED, e.status, st, done, t)
                    ready = []
                    torch.cuda.nvtx.range_pop()
            if ready:
                st.ticks += 1
                st.launches += 1
                ev = torch.cuda.Event()
                ev.record(self.s_enum)
                self.s_copy.wait_event(ev)
                with torch.cuda.stream(self.s_copy):
                    for q in ready:
                        words = q.count * q.W
                        self.host_ring.view(q.blk_host, words).copy_(self.dev_ring.view(q.blk_dev, words),
                                                                     non_blocking=True)
                        q.ev_copy = torch.cuda.Event()
                        q.ev_copy.record(self.s_copy)
                        q.state = "launched"
                        if self._on_event:
                            self._on_event("launched", q)
                copying.extend(ready)
                torch.cuda.nvtx.range_pop()
            finished = 0
            while copying and copying[0].ev_copy.query():  # copies complete in stream order
                q = copying.pop(0)
                finished += 1
                if self.keep:
                    q.result = self.host_ring.view(q.blk_host, q.count * q.W).numpy().view(np.uint64)\
                        .reshape(q.count, q.W).copy()
                self._release(q)
                q.packed = None
                self._finish(q, OK, 0, st, done, time.perf_counter() - t0)
            if busy_since is not None and not (any(factoring) or pending or copying):
                st.busy_s += (time.perf_counter() - t0) - busy_since
                busy_since = None
            if not ready and not finished and not progressed:
                if waiting and not any(factoring) and not pending and not copying:
                    dt = waiting[0].t_arrival - (time.perf_counter() - t0)
                    if dt > 0:
                        _wait_until(t0, waiting[0].t_arrival, 0.001)
                elif not pending:
                    # only events to wait for: poll just those until one
                    # fires, the next request or timed cancellation is due,
                    # or a cancel() comes in; a whole pass of the loop per
                    # poll would add its cost to the request's latency. (With
                    # work in flight the loop never sleeps: a sleep of a few
                    # microseconds lasts ~60 us on Linux.)
                    evs = [fq[0].ev_factor for fq in factoring if fq]
                    if copying:
                        evs.append(copying[0].ev_copy)
                    t_next = waiting[0].t_arrival if waiting else float("inf")
                    if next_cancel < len(cancels):
                        t_next = min(t_next, cancels[next_cancel][0])
                    while (not self._cancel and time.perf_counter() - t0 < t_next
                           and not any(e.query() for e in evs)):
                        pass
        st.makespan_s = time.perf_counter() - t0
        if busy_since is not None:
            st.busy_s += st.makespan_s - busy_since
        return st, done


def run_plain(stream: list[dict], keep_results: bool = True, host_bytes: int = 2 << 30,
              device_bytes: int = 2 << 30) -> tuple[Stats, list[Req]]:
    """The plain path: requests served one at a time in arrival order, each
    with its own factor launch, window launch and copy to pinned host memory,
    waiting for each step. It uses the same kind of preallocated buffers, the
    same collector setting and the same outcomes (a request whose t_cancel
    has passed when its turn comes is cancelled), so it differs from
    Server.run only in scheduling."""
    with _no_gc_pauses():
        return _run_plain(stream, keep_results, host_bytes, device_bytes)


def _run_plain(stream, keep_results, host_bytes, device_bytes):
    import torch

    reqs = _mk_reqs(stream)
    st = Stats(n_requests=len(reqs))
    dev_buf = torch.empty(device_bytes // 8, dtype=torch.int64, device="cuda")
    host_buf = torch.empty(host_bytes // 8, dtype=torch.int64, pin_memory=True)
    in_buf = torch.empty((1 << 20) // 8, dtype=torch.int64, pin_memory=True)

    def end(q, outcome, status):
        q.outcome, q.status, q.state, q.t_done = outcome, status, "done", time.perf_counter() - t0
        if outcome == FAILED:
            st.failed += 1
        elif outcome == CANCELLED:
            st.cancelled += 1
        elif outcome == REFUSED:
            st.refused += 1

    t0 = time.perf_counter()
    for q in reqs:
        now = time.perf_counter() - t0
        if q.t_arrival > now:
            _wait_until(t0, q.t_arrival)
        t_start = time.perf_counter() - t0
        if q.t_cancel is not None and q.t_cancel <= t_start:
            end(q, CANCELLED, 0)
            continue
        status, packed = check_request(q)
        if status:
            end(q, FAILED, status)
            continue
        q.W = hlf.words(q.n)
        if q.n * q.W > in_buf.numel():
            end(q, REFUSED, _ERR_NOMEM)
            continue
        in_buf[: q.n * q.W].copy_(torch.from_numpy(packed.ravel()))
        A_dev = in_buf[: q.n * q.W].view(q.n, q.W).to("cuda", non_blocking=True)
        h = 0
        try:
            h = hlf.hlf_factor(A_dev, q.n)
            q.r = hlf.hlf_get_rank(h)
        except hlf.HlfError as e:
            if h:
                hlf.hlf_destroy(h)
            torch.cuda.current_stream().synchronize()
            end(q, FAILED, e.status)
            continue
        q.offset, q.count = window_of(q.r, q.want, q.u)
        words = q.count * q.W
        if words > dev_buf.numel() or words > host_buf.numel():
            hlf.hlf_destroy(h)
            end(q, REFUSED, _ERR_NOMEM)
            continue
        hlf.hlf_enumerate_store(h, q.offset, q.count, dev_buf[: max(words, 1)])
        host_buf[:words].copy_(dev_buf[:words])
        hlf.hlf_destroy(h)
        end(q, OK, 0)
        st.busy_s += q.t_done - t_start
        st.launches += 2
        st.latencies_ms.append(1e3 * (q.t_done - q.t_arrival))
        st.solutions += q.count
        st.bytes_out += words * 8
        if keep_results:
            q.result = host_buf[:words].numpy().view(np.uint64).reshape(q.count, q.W).copy()
    st.makespan_s = time.perf_counter() - t0
    st.ticks = len(reqs)
    return st, reqs
