"""Request loop for the served workload: continuous batching of enumeration
windows on one GPU, and the plain one-request-at-a-time path it is compared
with.

A request carries a matrix A, a wanted window length and a 64-bit draw u.
Once its factorisation is known (rank r), the window is
    count  = min(want, 2^min(r, 64)),
    offset = u mod (2^min(r, 64) - count + 1),
and the solutions z(offset) .. z(offset + count - 1) are returned to the host.

Continuous batching (Server.run):
  * admission: a request is admitted, in arrival order, once it has arrived
    and the device memory it will hold (its factorisation and its output
    window) fits in the budget; otherwise it waits;
  * factorisations are launched on a factor stream and stay resident until
    their window has been copied out;
  * every tick, all admitted windows whose factorisation has finished are
    materialised by ONE hlf_enumerate_store_many launch on the enumeration
    stream, while earlier ticks' results are still being copied out;
  * copies go to pinned host buffers on a copy stream; a request completes
    when its copy event has fired (latency = completion - arrival).
All solver work runs in the library's kernels; this module only schedules.
"""

from __future__ import annotations

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
    # device-side state
    h: int = 0
    A_dev: object = None
    out_dev: object = None
    ev_factor: object = None
    ev_copy: object = None
    host: object = None
    reserved: int = 0


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


def _mk_reqs(stream: list[dict]) -> list[Req]:
    return [Req(id=q["id"], t_arrival=q["t_arrival"], A=q["A"], want=q["want"], u=q["u"]) for q in stream]


class Server:
    """Continuous-batching server on the current CUDA device."""

    def __init__(self, mem_budget_bytes: int = 16 << 30, max_batch: int = 4096, keep_results: bool = True):
        import torch

        self.budget = mem_budget_bytes
        self.keep = keep_results
        self.s_factor = torch.cuda.Stream()
        self.s_enum = torch.cuda.Stream()
        self.s_copy = torch.cuda.Stream()
        self.max_batch = max_batch
        self.many = hlf.hlf_many_create(max_batch)

    def close(self):
        if self.many:
            hlf.hlf_many_destroy(self.many)
            self.many = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, stream: list[dict]) -> tuple[Stats, list[Req]]:
        import torch

        reqs = _mk_reqs(stream)
        waiting = list(reqs)           # not yet admitted, in arrival order
        factoring: list[Req] = []      # factor launched
        copying: list[Req] = []        # window launched and copy enqueued
        done: list[Req] = []
        used = 0
        st = Stats(n_requests=len(reqs))
        t0 = time.perf_counter()
        busy_since = None
        while waiting or factoring or copying:
            now = time.perf_counter() - t0
            # -- admission, in arrival order, by device memory
            while waiting and waiting[0].t_arrival <= now:
                q = waiting[0]
                q.n = q.A.shape[0]
                q.W = hlf.words(q.n)
                need = handle_bytes(q.n) + q.want * q.W * 8
                if used + need > self.budget and (factoring or copying):
                    break
                waiting.pop(0)
                q.reserved = need
                used += need
                packed = torch.from_numpy(hlf.pack_rows(q.A).view(np.int64)).pin_memory()
                with torch.cuda.stream(self.s_factor):
                    q.A_dev = packed.to("cuda", non_blocking=True)
                    q.h = hlf.hlf_factor(q.A_dev, q.n, self.s_factor)
                    q.ev_factor = torch.cuda.Event()
                    q.ev_factor.record(self.s_factor)
                factoring.append(q)
            # -- one launch for every window whose factorisation is done
            ready = [q for q in factoring if q.ev_factor.query()][: self.max_batch]
            if ready:
                if busy_since is None:
                    busy_since = now
                for q in ready:
                    factoring.remove(q)
                    q.r = hlf.hlf_get_rank(q.h)
                    q.offset, q.count = window_of(q.r, q.want, q.u)
                    used += q.count * q.W * 8 - q.want * q.W * 8  # shrink to the real window
                    q.reserved += q.count * q.W * 8 - q.want * q.W * 8
                    q.out_dev = torch.empty((max(q.count, 1), q.W), dtype=torch.int64, device="cuda")
                hlf.hlf_enumerate_store_many(self.many, [q.h for q in ready], [q.offset for q in ready],
                                             [q.count for q in ready], [q.out_dev for q in ready], self.s_enum)
                st.ticks += 1
                st.launches += 1
                ev = torch.cuda.Event()
                ev.record(self.s_enum)
                self.s_copy.wait_event(ev)
                with torch.cuda.stream(self.s_copy):
                    for q in ready:
                        q.host = torch.empty((max(q.count, 1), q.W), dtype=torch.int64, pin_memory=True)
                        q.host.copy_(q.out_dev, non_blocking=True)
                        q.ev_copy = torch.cuda.Event()
                        q.ev_copy.record(self.s_copy)
                copying.extend(ready)
            # -- completions
            still = []
            for q in copying:
                if q.ev_copy.query():
                    q.t_done = time.perf_counter() - t0
                    st.latencies_ms.append(1e3 * (q.t_done - q.t_arrival))
                    st.solutions += q.count
                    st.bytes_out += q.count * q.W * 8
                    if self.keep:
                        q.result = q.host.numpy()[: q.count].view(np.uint64).copy()
                    hlf.hlf_destroy(q.h)
                    q.h = 0
                    q.out_dev = q.A_dev = q.host = None
                    used -= q.reserved
                    done.append(q)
                else:
                    still.append(q)
            copying = still
            if busy_since is not None and not (factoring or copying):
                st.busy_s += (time.perf_counter() - t0) - busy_since
                busy_since = None
            if not ready and not (copying and copying[0].ev_copy.query()):
                if waiting and not factoring and not copying:
                    dt = waiting[0].t_arrival - (time.perf_counter() - t0)
                    if dt > 0:
                        time.sleep(min(dt, 0.002))
                else:
                    time.sleep(20e-6)
        st.makespan_s = time.perf_counter() - t0
        if busy_since is not None:
            st.busy_s += st.makespan_s - busy_since
        return st, done


def run_plain(stream: list[dict], keep_results: bool = True) -> tuple[Stats, list[Req]]:
    """The plain path: requests served one at a time in arrival order, each
    with its own factor launch, window launch and copy, synchronously."""
    import torch

    reqs = _mk_reqs(stream)
    st = Stats(n_requests=len(reqs))
    t0 = time.perf_counter()
    for q in reqs:
        now = time.perf_counter() - t0
        if q.t_arrival > now:
            time.sleep(q.t_arrival - now)
        t_start = time.perf_counter() - t0
        q.n = q.A.shape[0]
        q.W = hlf.words(q.n)
        A_dev = torch.from_numpy(hlf.pack_rows(q.A).view(np.int64)).cuda()
        h = hlf.hlf_factor(A_dev, q.n)
        q.r = hlf.hlf_get_rank(h)
        q.offset, q.count = window_of(q.r, q.want, q.u)
        out = torch.empty((max(q.count, 1), q.W), dtype=torch.int64, device="cuda")
        hlf.hlf_enumerate_store(h, q.offset, q.count, out)
        host = torch.empty((max(q.count, 1), q.W), dtype=torch.int64, pin_memory=True)
        host.copy_(out)
        hlf.hlf_destroy(h)
        q.t_done = time.perf_counter() - t0
        st.busy_s += q.t_done - t_start
        st.launches += 2
        st.latencies_ms.append(1e3 * (q.t_done - q.t_arrival))
        st.solutions += q.count
        st.bytes_out += q.count * q.W * 8
        if keep_results:
            q.result = host.numpy()[: q.count].view(np.uint64).copy()
    st.makespan_s = time.perf_counter() - t0
    st.ticks = len(reqs)
    return st, reqs
