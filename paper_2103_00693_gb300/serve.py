"""Request loop for the served workload: continuous batching of enumeration
windows on one GPU, and the plain one-request-at-a-time path it is compared
with.

A request carries a matrix A, a wanted window length and a 64-bit draw u.
Once its factorisation is known (rank r), the window is
    count  = min(want, 2^min(r, 64)),
    offset = u mod (2^min(r, 64) - count + 1),
and the solutions z(offset) .. z(offset + count - 1) are returned to the host.

Continuous batching (Server.run):
  * admission by device memory: a request is admitted, in arrival order, once
    it has arrived and its output window (want x W words) fits in the device
    staging ring; a window that does not fit waits for earlier ones to leave;
  * factorisations are launched on high-priority factor streams, in turn, as
    requests are admitted, and stay resident (one handle each) until their
    window has reached the host. A stream's factor kernels finish in order,
    so the loop keeps one queue per factor stream and asks only each queue's
    head whether it is done;
  * every tick, all admitted windows whose factorisation has finished are
    materialised by ONE hlf_enumerate_store_many launch on the enumeration
    stream, into the staging ring, while earlier ticks' windows are still
    being copied out and later requests are being factored;
  * each window is copied to its slot of a pinned host ring on a copy stream;
    a request completes when its copy event has fired
    (latency = completion - arrival).
Both rings are allocated once, up front, so the loop itself never allocates
or frees memory (allocation can synchronise the device); handles use the
stream-ordered pool. All solver work runs in the library's kernels; this
module only schedules.
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


@dataclass
class Req:
    id: int
    t_arrival: float
    A: np.ndarray
    want: int
    u: int
    n: int = 0
    W: int = 0
    r: int = -1
    offset: int = 0
    count: int = 0
    t_done: float = 0.0
    result: np.ndarray | None = None
    h: int = 0
    blk_dev: list | None = None
    blk_host: list | None = None
    blk_in: list | None = None
    blk_mat: list | None = None
    A_dev: object = None
    ev_factor: object = None
    ev_copy: object = None
    lane: int = 0  # which factor stream


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

    def summary(self) -> dict:
        lat = np.array(self.latencies_ms) if self.latencies_ms else np.zeros(1)
        return {"requests": self.n_requests, "solutions": self.solutions,
                "solutions_per_s": self.solutions / self.makespan_s if self.makespan_s else 0.0,
                "gb_per_s_to_host": self.bytes_out / self.makespan_s / 1e9 if self.makespan_s else 0.0,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "makespan_s": self.makespan_s,
                "busy_frac": self.busy_s / self.makespan_s if self.makespan_s else 0.0,
                "ticks": self.ticks, "launches": self.launches}


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
    return [Req(id=q["id"], t_arrival=q["t_arrival"], A=q["A"], want=q["want"], u=q["u"]) for q in stream]


class Server:
    """Continuous-batching server on the current CUDA device.

    device_bytes: the staging ring (the admission budget for output windows);
    host_bytes:   the pinned host ring the results land in.
    """

    def __init__(self, device_bytes: int = 8 << 30, host_bytes: int = 8 << 30, max_batch: int = 4096,
                 keep_results: bool = True):
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
        self.in_ring = Ring(torch.empty((64 << 20) // 8, dtype=torch.int64, pin_memory=True))
        # the packed matrices on the device: carved from a ring as well, so
        # the loop never reaches the allocator (which may synchronise)
        self.mat_ring = Ring(torch.empty((64 << 20) // 8, dtype=torch.int64, device="cuda"))

    def close(self):
        if self.many:
            hlf.hlf_many_destroy(self.many)
            self.many = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _admit(self, q: Req) -> bool:
        import torch

        q.n = q.A.shape[0]
        q.W = hlf.words(q.n)
        words = q.want * q.W
        bd = self.dev_ring.alloc(words)
        if bd is None:
            return False
        bh = self.host_ring.alloc(words)
        if bh is None:
            self.dev_ring.free(bd)
            return False
        bi = self.in_ring.alloc(q.n * q.W)
        bm = self.mat_ring.alloc(q.n * q.W) if bi is not None else None
        if bm is None:
            if bi is not None:
                self.in_ring.free(bi)
            self.dev_ring.free(bd)
            self.host_ring.free(bh)
            return False
        q.blk_dev, q.blk_host, q.blk_in, q.blk_mat = bd, bh, bi, bm
        staged = self.in_ring.view(bi, q.n * q.W)
        staged.copy_(torch.from_numpy(hlf.pack_rows(q.A).view(np.int64).ravel()))
        q.lane = self._next_factor
        sf = self.s_factors[q.lane]
        self._next_factor = (self._next_factor + 1) % len(self.s_factors)
        with torch.cuda.stream(sf):
            q.A_dev = self.mat_ring.view(bm, q.n * q.W).view(q.n, q.W)
            q.A_dev.view(-1).copy_(staged, non_blocking=True)
            q.h = hlf.hlf_factor(q.A_dev, q.n, sf)
            q.ev_factor = torch.cuda.Event()
            q.ev_factor.record(sf)
        return True

    def run(self, stream: list[dict]) -> tuple[Stats, list[Req]]:
        with _no_gc_pauses():
            return self._run(stream)

    def _run(self, stream: list[dict]) -> tuple[Stats, list[Req]]:
        import torch

        reqs = _mk_reqs(stream)
        waiting = collections.deque(reqs)
        # one FIFO per factor stream: a stream's factor kernels finish in
        # order, so only each queue's head needs an event query
        factoring = [collections.deque() for _ in self.s_factors]
        copying: list[Req] = []
        done: list[Req] = []
        st = Stats(n_requests=len(reqs))
        t0 = time.perf_counter()
        busy_since = None
        while waiting or any(factoring) or copying:
            now = time.perf_counter() - t0
            while waiting and waiting[0].t_arrival <= now:
                if not self._admit(waiting[0]):
                    if not (any(factoring) or copying):
                        raise RuntimeError(f"request {waiting[0].id} does not fit the rings")
                    break
                q = waiting.popleft()
                factoring[q.lane].append(q)
                if busy_since is None:
                    busy_since = now
            ready = []
            for fq in factoring:
                while fq and len(ready) < self.max_batch and fq[0].ev_factor.query():
                    ready.append(fq.popleft())
            if ready:
                for q in ready:
                    self.in_ring.free(q.blk_in)
                    q.r = hlf.hlf_get_rank(q.h)
                    q.offset, q.count = window_of(q.r, q.want, q.u)
                hlf.hlf_enumerate_store_many(
                    self.many, [q.h for q in ready], [q.offset for q in ready], [q.count for q in ready],
                    [self.dev_ring.view(q.blk_dev, max(q.count, 1) * q.W) for q in ready], self.s_enum)
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
                copying.extend(ready)
            finished = 0
            while copying and copying[0].ev_copy.query():  # copies complete in stream order
                q = copying.pop(0)
                finished += 1
                q.t_done = time.perf_counter() - t0
                st.latencies_ms.append(1e3 * (q.t_done - q.t_arrival))
                st.solutions += q.count
                st.bytes_out += q.count * q.W * 8
                if self.keep:
                    q.result = self.host_ring.view(q.blk_host, q.count * q.W).numpy().view(np.uint64)\
                        .reshape(q.count, q.W).copy()
                hlf.hlf_destroy(q.h)
                q.h = 0
                q.A_dev = None
                self.mat_ring.free(q.blk_mat)  # the factor kernel read it long before the copy ended
                self.dev_ring.free(q.blk_dev)
                self.host_ring.free(q.blk_host)
                done.append(q)
            if busy_since is not None and not (any(factoring) or copying):
                st.busy_s += (time.perf_counter() - t0) - busy_since
                busy_since = None
            if not ready and not finished:
                if waiting and not any(factoring) and not copying:
                    dt = waiting[0].t_arrival - (time.perf_counter() - t0)
                    if dt > 0:
                        time.sleep(min(dt, 0.001))
                # with work in flight the loop polls its events without
                # sleeping: a sleep of a few microseconds lasts ~60 us on
                # Linux, which would add to every request's latency
        st.makespan_s = time.perf_counter() - t0
        if busy_since is not None:
            st.busy_s += st.makespan_s - busy_since
        return st, done


def run_plain(stream: list[dict], keep_results: bool = True, host_bytes: int = 2 << 30,
              device_bytes: int = 2 << 30) -> tuple[Stats, list[Req]]:
    """The plain path: requests served one at a time in arrival order, each
    with its own factor launch, window launch and copy to pinned host memory,
    waiting for each step. It uses the same kind of preallocated buffers and
    the same collector setting, so it differs from Server.run only in
    scheduling."""
    with _no_gc_pauses():
        return _run_plain(stream, keep_results, host_bytes, device_bytes)


def _run_plain(stream, keep_results, host_bytes, device_bytes):
    import torch

    reqs = _mk_reqs(stream)
    st = Stats(n_requests=len(reqs))
    dev_buf = torch.empty(device_bytes // 8, dtype=torch.int64, device="cuda")
    host_buf = torch.empty(host_bytes // 8, dtype=torch.int64, pin_memory=True)
    in_buf = torch.empty((1 << 20) // 8, dtype=torch.int64, pin_memory=True)
    t0 = time.perf_counter()
    for q in reqs:
        now = time.perf_counter() - t0
        if q.t_arrival > now:
            time.sleep(q.t_arrival - now)
        t_start = time.perf_counter() - t0
        q.n = q.A.shape[0]
        q.W = hlf.words(q.n)
        in_buf[: q.n * q.W].copy_(torch.from_numpy(hlf.pack_rows(q.A).view(np.int64).ravel()))
        A_dev = in_buf[: q.n * q.W].view(q.n, q.W).to("cuda", non_blocking=True)
        h = hlf.hlf_factor(A_dev, q.n)
        q.r = hlf.hlf_get_rank(h)
        q.offset, q.count = window_of(q.r, q.want, q.u)
        words = q.count * q.W
        hlf.hlf_enumerate_store(h, q.offset, q.count, dev_buf[: max(words, 1)])
        host_buf[:words].copy_(dev_buf[:words])
        hlf.hlf_destroy(h)
        q.t_done = time.perf_counter() - t0
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
