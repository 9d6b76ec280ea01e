#!/usr/bin/env python
"""Throughput of the FS2D HLF hot path (arXiv 2103.00693) on GB300.

Workload: the all-connected 6 x 6 grid (n = 36, Bernoulli(1/2) diagonal,
seed 3, binary rank r = 36). One step is one pass over every part of the
path through the C ABI:
  hlf_factor (stage 1: GF(2) elimination, kernel basis, q, z^a)
  hlf_enumerate_reduce of all 2^r solutions (count, XOR-fold, hash sum)
  hlf_enumerate_store of the first 2^30 solutions into HBM (8 GiB)
  hlf_sample of 2^20 seeded indices.
value = 2^r solutions per step / step time (the store and the sample are
extra work inside the step and are not counted as solutions).

Other legs on the same JSON line: the dominant kernel's roofline, the store
kernel's HBM roofline, an end-to-end run through host buffers (e2e), SM
clocks sampled during the timed region, the widened rows (dense store,
histogram), the other single-instance workloads (grid3x3 latency, the grid8x8
2^40-solution window), the batched and served workloads, and the CPU oracle
timed on the host cores (cpu_baseline). `--impl reference` times the CPU
oracle alone.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FS2D HLF solutions/sec"
UNIT = "solutions/s"
# Minimal 32-bit integer instructions per solution of the reduce at W = 1:
# Gray step XOR 2, the SplitMix64 finalizer after its first (GF(2)-linear)
# layer, which the walk absorbs into the basis table: two 64 x 64 -> 64
# multiplies at 3 and two 64-bit xor-shifts at 4 (14), and the 64-bit add of
# the hash 2. The XOR-fold costs nothing per solution: over a whole aligned
# Gray block of 2^U >= 4 solutions it is zero, so only the partial blocks at
# the ends of a run are folded. Each further word adds its step XOR 2, the
# XOR into the chained hash 2 and a whole finalizer 18: 22W - 4 in all.
OPS_PER_SOLUTION_W1 = 18
ISSUE_LANES_PER_SM_CLK = 128  # 4 schedulers x 32 lanes
# The histogram walks the table projected onto the field: per solution one
# 32-bit XOR and one shared-memory atomic add.
HIST_OPS_PER_SOLUTION = 2
# Of the reduce's 18 operations per solution at W = 1, the 12 that only the
# ALU pipe executes (64 lanes per clock per SM): the step XOR 2, the two
# xor-shifts 8 and the 64-bit add 2. The multiplies run on the FMA pipe.
ALU_PIPE_OPS_PER_SOLUTION_W1 = 12
ALU_PIPE_LANES_PER_SM_CLK = 64
PROBE_ITERS = 1 << 14
STORE_LOG2 = 30
SAMPLE_LOG2 = 20
SAMPLE_SEED = 99

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# each roofline kernel in this bench's default configuration, recorded by hand
# from one ncu capture of this bench (not measured in the run). Each record
# carries a digest of the kernel's source files at capture time; once those
# sources change, the figure no longer describes the kernel and the line
# reports null.
KERNEL_SOURCES = {
    "reduce_kernel<1,6,1024>": ["enumerate.cu", "enum_impl.cuh", "hlf_internal.cuh"],
    "store_kernel<1,2>": ["enumerate.cu", "enum_impl.cuh", "hlf_internal.cuh"],
    "dense1_kernel<16,1,1>": ["dense.cu", "enum_impl.cuh", "hlf_internal.cuh"],
}
TRAFFIC = {  # kernel -> per-launch DRAM bytes (read + write) and the source digest at capture
    "reduce_kernel<1,6,1024>": {"bytes": 541440 + 1536, "sources": "0b975b98a6be7595"},
    "store_kernel<1,2>": {"bytes": 244992 + 8525198848, "sources": "0b975b98a6be7595"},
    "dense1_kernel<16,1,1>": {"bytes": 467200 + 4767411200, "sources": "2a92c04830996b04"},
}


def source_digest(kernel: str) -> str:
    import hashlib

    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2103_00693_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic(kernel: str):
    rec = TRAFFIC.get(kernel)
    if rec is None or rec["sources"] != source_digest(kernel):
        return None
    return rec["bytes"]


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["hlf", "reference"], default="hlf")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="target length of the CPU-oracle sample")
    p.add_argument("--reduce-log2", type=int, default=None,
                   help="reduce only the first 2^k solutions (small cases for profiling; the line says so)")
    p.add_argument("--store-log2", type=int, default=STORE_LOG2, help="solutions stored per step (log2)")
    p.add_argument("--no-batched", action="store_true", help="skip the batched (4096 grids) leg")
    p.add_argument("--no-served", action="store_true", help="skip the served (Poisson stream) leg")
    p.add_argument("--shard", action="store_true",
                   help="split ONE grid6x6 instance across the ranks (contiguous index ranges, one all-gather "
                        "of the partials; strong scaling) instead of one replica per GPU")
    return p.parse_args()


def ops_per_solution(W: int) -> int:
    """The reduce's minimal 32-bit integer operations per solution of W words."""
    return OPS_PER_SOLUTION_W1 + 22 * (W - 1)


def alu_pipe_ops_per_solution(W: int) -> int:
    """Of those, the ones only the ALU pipe executes: 12 at W = 1, and per
    further word its step XOR 2, the XOR into the running hash 2 and the
    three xor-shifts of its SplitMix64 round 12 (the round's two multiplies
    run on the FMA pipe)."""
    return ALU_PIPE_OPS_PER_SOLUTION_W1 + 16 * (W - 1)


def alu_pipe_peak(dev=None):
    """(peak ALU-pipe ops/s in T, its basis): 64 lanes per clock per SM."""
    import torch

    pk = peaks()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device() if dev is None else dev).multi_processor_count
    peak = sms * ALU_PIPE_LANES_PER_SM_CLK * pk["sm_max_mhz"] * 1e6 / 1e12
    return peak, f"{sms} SMs x {ALU_PIPE_LANES_PER_SM_CLK} ALU-pipe lanes/clk x {pk['sm_max_mhz']:.0f} MHz"


def int_peak(dev=None):
    """(peak 32-bit integer ops/s in T, its basis): every SM's four
    schedulers issuing one 32-lane instruction per clock at the maximum SM
    clock."""
    import torch

    pk = peaks()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device() if dev is None else dev).multi_processor_count
    peak = sms * ISSUE_LANES_PER_SM_CLK * pk["sm_max_mhz"] * 1e6 / 1e12
    return peak, f"{sms} SMs x {ISSUE_LANES_PER_SM_CLK} int32 lanes/clk x {pk['sm_max_mhz']:.0f} MHz (issue limit)"


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": d["hbm_gbs"], "sm_max_mhz": d.get("sm_max_mhz", 2070.0), "source": "measured"}
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi SM clock and throttle reasons, sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        # nvidia-smi's start-up (NVML initialisation) can stall the host's
        # launches and waits for tens of ms: let it write its first sample
        # before the caller opens the timed region (bounded wait)
        t_end = time.time() + 3.0
        while time.time() < t_end and self.proc.poll() is None and os.path.getsize(self.file.name) == 0:
            time.sleep(0.01)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [ln.split(",") for ln in self.file.read().strip().splitlines() if ln.strip()]
        os.unlink(self.file.name)
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            try:
                pw.append(float(r[3]))
            except ValueError:
                pass
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
               "samples": len(sm)}
        if pw:
            out["power_w"] = statistics.median(pw)
        return out


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        backend = "nccl" if (args.impl == "hlf" and torch.cuda.is_available()) else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ CPU oracle

def cpu_oracle_sample(target_s: float):
    """Time the oracle as it stands (factor + reduce of a leading window of
    the workload) on all host cores; the window is sized for ~target_s."""
    from oracle import cpu as oc
    from synth import workloads as wl

    cores = os.cpu_count() or 1
    A = wl.grid6()
    F = oc.factor(A)
    t0 = time.perf_counter()
    oc.reduce(F, 0, 1 << 24, cores)
    rate = (1 << 24) / max(time.perf_counter() - t0, 1e-6)
    k = 24
    while k < F.r and (1 << (k + 1)) / rate <= target_s:
        k += 1
    t0 = time.perf_counter()
    F = oc.factor(A)
    oc.reduce(F, 0, 1 << k, cores)
    dt = time.perf_counter() - t0
    # the same oracle on one thread, over a window sized for ~target_s / 4
    t0 = time.perf_counter()
    oc.reduce(F, 0, 1 << 20, 1)
    rate1 = (1 << 20) / max(time.perf_counter() - t0, 1e-6)
    k1 = 20
    while k1 < F.r and (1 << (k1 + 1)) / rate1 <= target_s / 4:
        k1 += 1
    t0 = time.perf_counter()
    oc.reduce(F, 0, 1 << k1, 1)
    dt1 = time.perf_counter() - t0
    return {"value": (1 << k) / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"oracle factor + reduce of solutions [0, 2^{k}) of the 2^{F.r} on {cores} threads "
                      f"({dt:.1f} s)",
            "single_thread": {"value": (1 << k1) / dt1, "unit": UNIT,
                              "sample": f"oracle reduce of solutions [0, 2^{k1}) on 1 thread ({dt1:.1f} s)"}}, k


def workload_config(r: int, reduce_n: int | None = None, store_n: int | None = None):
    reduce_n = reduce_n or (1 << r)
    store_n = store_n or (1 << STORE_LOG2)
    return {"workload": "grid6x6 all-connected (n=36, Bernoulli(1/2) diagonal, seed 3)",
            "n": 36, "r": r, "reduce_per_step": f"2^{reduce_n.bit_length() - 1}",
            "store_per_step": f"2^{store_n.bit_length() - 1}",
            "sample_per_step": f"2^{SAMPLE_LOG2}",
            "l2": "each step stores 8 GiB (> 129 MB L2) between reduces; no separate flush",
            "parallelism": "replicas (one independent instance per GPU)"}


def run_reference(args, world, rank):
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    from oracle import cpu as oc
    from synth import workloads as wl

    A = wl.grid6()
    F = oc.factor(A)
    # one step = oracle factor + reduce of a leading 2^k window (~4 s)
    t0 = time.perf_counter()
    oc.reduce(F, 0, 1 << 24, cores)
    rate = (1 << 24) / max(time.perf_counter() - t0, 1e-6)
    k = 24
    while k < F.r and (1 << (k + 1)) / rate <= 4.0:
        k += 1

    def step():
        G = oc.factor(A)
        oc.reduce(G, 0, 1 << k, cores)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = args.steps * (1 << k) / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": workload_config(F.r),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"per step: oracle factor + reduce of solutions [0, 2^{k}) of the "
                                       f"2^{F.r} on {cores} threads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU path

def run_hlf(args, world, rank, local):
    import numpy as np
    import torch

    import paper_2103_00693_gb300 as hlf
    import synth
    from synth import workloads as wl

    torch.cuda.set_device(local)
    hlf.load()
    dev = torch.device("cuda", local)
    A = wl.grid6()
    n = A.shape[0]
    W = hlf.words(n)
    packed = hlf.pack_rows(A).view(np.int64)
    A_dev = torch.from_numpy(packed).to(dev)
    h = hlf.hlf_factor(A_dev, n)
    r = hlf.hlf_get_rank(h)
    hlf.hlf_destroy(h)
    total = 1 << min(r, 64)
    if args.reduce_log2 is not None:
        total = min(total, 1 << args.reduce_log2)
    store_n = min(1 << args.store_log2, total)
    m = 1 << SAMPLE_LOG2
    idx_host = synth.sample_indices(SAMPLE_SEED, m, 0, total).view(np.int64)
    idx_dev = torch.from_numpy(idx_host).to(dev)
    out = torch.empty((store_n, W), dtype=torch.int64, device=dev)
    smp = torch.empty((m, W), dtype=torch.int64, device=dev)
    red = torch.empty(hlf.REDUCE_WORDS, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)
    fstream = torch.cuda.Stream(dev)
    nxt = {}

    def prefetch():
        # a step's factorisation is enqueued on its own stream at the end of
        # the step before, so it runs beside that step's kernels and its rank
        # is ready when the host asks for it: the host's wait for r (the
        # reduce's launch needs it) then never lets the device queue drain.
        # Every step still factors once. The first timed step's factorisation
        # is enqueued by the last warm-up step, before the region, and the
        # region ends after the one the last timed step enqueues: it holds
        # exactly K factor launches.
        nxt["h"] = hlf.hlf_factor(A_dev, n, fstream)
        nxt["ev"] = torch.cuda.Event()
        nxt["ev"].record(fstream)

    def step(evs=None):
        hh = nxt["h"]
        stream.wait_event(nxt["ev"])
        # the reduce needs r on the host: wait for it before the start
        # event, so that the event brackets the reduce kernel alone
        hlf.hlf_get_rank(hh)
        if evs:
            evs[0].record(stream)
        hlf.hlf_enumerate_reduce(hh, 0, total, red, stream)
        if evs:
            evs[1].record(stream)
        hlf.hlf_enumerate_store(hh, 0, store_n, out, stream)
        if evs:
            evs[2].record(stream)
        hlf.hlf_sample(hh, idx_dev, m, smp, stream)
        prefetch()
        hlf.hlf_destroy(hh)

    prefetch()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    res = hlf.ReduceResult.from_words(red.cpu().numpy(), W)
    if res.count != total:
        raise RuntimeError(f"reduce counted {res.count} solutions, expected {total}")

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize(dev)
    start.record(stream)
    for k in range(args.steps):
        step(evs[k])
    stream.wait_event(nxt["ev"])  # the last factorisation inside the region
    end.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    hlf.hlf_destroy(nxt.pop("h"))
    barrier(world)
    ms = start.elapsed_time(end)
    ms_max = max_over_ranks(ms, world)
    reduce_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    store_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in evs)
    value = world * args.steps * total / (ms_max / 1e3)

    pk = peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = sms * ISSUE_LANES_PER_SM_CLK * pk["sm_max_mhz"] * 1e6 / 1e12  # Tops/s
    ops = total * ops_per_solution(W)
    achieved = ops / (reduce_ms / 1e3) / 1e12
    store_bytes = store_n * W * 8
    store_gbs = store_bytes / (store_ms / 1e3) / 1e9

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": workload_config(r, total, store_n),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Tops/s",
                         "frac": achieved / alu_peak, "traffic": traffic("reduce_kernel<1,6,1024>"),
                         "kernel": "reduce_kernel<1,6,1024>",
                         "ms_per_launch": reduce_ms,
                         "peak_basis": f"{sms} SMs x {ISSUE_LANES_PER_SM_CLK} int32 lanes/clk x "
                                       f"{pk['sm_max_mhz']:.0f} MHz (issue limit)",
                         "ops_per_solution": ops_per_solution(W)},
            "roofline_alu_pipe": {
                "bound": "alu_pipe",
                "achieved": total * ALU_PIPE_OPS_PER_SOLUTION_W1 / (reduce_ms / 1e3) / 1e12,
                "peak": sms * ALU_PIPE_LANES_PER_SM_CLK * pk["sm_max_mhz"] * 1e6 / 1e12, "unit": "Tops/s",
                "frac": (total * ALU_PIPE_OPS_PER_SOLUTION_W1 / (reduce_ms / 1e3))
                        / (sms * ALU_PIPE_LANES_PER_SM_CLK * pk["sm_max_mhz"] * 1e6),
                "kernel": "reduce_kernel<1,6,1024>", "ops_per_solution": ALU_PIPE_OPS_PER_SOLUTION_W1,
                "peak_basis": f"{sms} SMs x {ALU_PIPE_LANES_PER_SM_CLK} ALU-pipe lanes/clk x "
                              f"{pk['sm_max_mhz']:.0f} MHz (the pipe that binds: W = 1 only)"} if W == 1 else None,
            "roofline_store": {"bound": "hbm", "achieved": store_gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                               "frac": store_gbs / pk["hbm_gbs"], "traffic": traffic("store_kernel<1,2>"),
                               "kernel": "store_kernel<1,2>", "ms_per_launch": store_ms,
                               "peak_source": pk["source"]},
            "gpu_launches": 4 * args.steps,
            "clocks": clk}

    # The e2e leg's pinned host buffers and the serving rings are pinned now,
    # after the timed step and well before their own legs: on a box that has
    # done much GPU work, host transfers and launches right after pinning
    # gigabytes of host memory were measured to run slow for a while.
    e2e_host = None if args.no_e2e else {
        "out": torch.empty((store_n, W), dtype=torch.int64, pin_memory=True),
        "smp": torch.empty((m, W), dtype=torch.int64, pin_memory=True),
        "red": torch.empty(hlf.REDUCE_WORDS, dtype=torch.int64, pin_memory=True)}
    server = None
    if not args.no_served:
        from paper_2103_00693_gb300 import serve
        server = serve.Server(keep_results=False)
    line["next_rows"] = run_next_rows(args, A_dev, n, W, store_n, pk, dev)
    line["configs"] = run_configs(dev)
    if not args.no_e2e:
        line["e2e"] = run_e2e(args, world, dev, A, r, total, store_n, idx_host, e2e_host)
    del out, smp
    torch.cuda.empty_cache()
    if not args.no_batched:
        line["batched"] = run_batched(args)
    if not args.no_served:
        line["served"] = run_served(args, server)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"], _ = cpu_oracle_sample(args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_next_rows(args, A_dev, n, W, store_n, pk, dev):
    """Throughput of the widened rows on the same grid: the dense bit-stream
    store (n = 36 bits per solution) of the 2^30 block, against HBM, and the
    on-device histogram of the first 14 bits over 2^32 solutions."""
    import torch

    import paper_2103_00693_gb300 as hlf

    hh = hlf.hlf_factor(A_dev, n)
    dense = torch.empty(hlf.dense_words(store_n, n), dtype=torch.int64, device=dev)
    hist = torch.empty(1 << 14, dtype=torch.int64, device=dev)
    hcount = 1 << 32

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / reps

    d_ms = timed(lambda: hlf.hlf_enumerate_store_dense(hh, 0, store_n, dense), max(3, args.steps))
    h_ms = timed(lambda: hlf.hlf_enumerate_histogram(hh, 0, hcount, 0, 14, hist), 3)
    hlf.hlf_destroy(hh)
    # the shared-memory atomic rate of this GPU (the histogram's denominator)
    psum = torch.empty(1, dtype=torch.int64, device=dev)
    n_atomics = hlf.hlf_probe_smem_atomics(PROBE_ITERS, psum)
    p_ms = timed(lambda: hlf.hlf_probe_smem_atomics(PROBE_ITERS, psum), 3)
    assert int(psum.item()) == n_atomics
    atomic_peak = n_atomics / (p_ms / 1e3) / 1e12
    h_rate = hcount / (h_ms / 1e3) / 1e12  # one shared-memory atomic per solution
    ipk, ipk_basis = int_peak(dev)
    dbytes = hlf.dense_words(store_n, n) * 8
    return {"dense_store": {"solutions": store_n, "bits_per_solution": n, "ms_per_launch": d_ms,
                            "solutions_per_s": store_n / (d_ms / 1e3),
                            "roofline": {"bound": "hbm", "achieved": dbytes / (d_ms / 1e3) / 1e9,
                                         "peak": pk["hbm_gbs"], "unit": "GB/s",
                                         "frac": dbytes / (d_ms / 1e3) / 1e9 / pk["hbm_gbs"],
                                         "kernel": "dense1_kernel<16,1,1>",
                                         "traffic": traffic("dense1_kernel<16,1,1>")}},
            "histogram": {"solutions": hcount, "field": "bits 0..13", "ms_per_launch": h_ms,
                          "solutions_per_s": hcount / (h_ms / 1e3),
                          "roofline": {"bound": "smem_atomic", "achieved": h_rate, "peak": atomic_peak,
                                       "unit": "T atomics/s", "frac": h_rate / atomic_peak,
                                       "kernel": "hist_interleaved_kernel<true>",
                                       "peak_basis": f"hlf_probe_smem_atomics: {n_atomics} conflict-free "
                                                     f"32-bit shared-memory atomics in {p_ms:.3f} ms"},
                          "roofline_issue": {"bound": "alu", "achieved": HIST_OPS_PER_SOLUTION * h_rate,
                                             "peak": ipk, "unit": "Tops/s",
                                             "frac": HIST_OPS_PER_SOLUTION * h_rate / ipk,
                                             "ops_per_solution": HIST_OPS_PER_SOLUTION, "peak_basis": ipk_basis}}}


def run_e2e(args, world, dev, A, r, total, store_n, idx_host, host_bufs=None):
    """The same step through the C ABI from host buffers: A and the sample
    indices are copied in from pinned memory, the 2^30 stored solutions, the
    samples and the reduce result are copied back, all inside the timed
    region."""
    import numpy as np
    import torch

    import paper_2103_00693_gb300 as hlf

    n = A.shape[0]
    W = hlf.words(n)
    A_host = torch.from_numpy(hlf.pack_rows(A).view(np.int64)).pin_memory()
    idx_pin = torch.from_numpy(idx_host).pin_memory()
    m = idx_pin.numel()
    A_dev = torch.empty_like(A_host, device=dev)
    idx_dev = torch.empty_like(idx_pin, device=dev)
    out = torch.empty((store_n, W), dtype=torch.int64, device=dev)
    smp = torch.empty((m, W), dtype=torch.int64, device=dev)
    red = torch.empty(hlf.REDUCE_WORDS, dtype=torch.int64, device=dev)
    if host_bufs is None:
        host_bufs = {"out": torch.empty((store_n, W), dtype=torch.int64, pin_memory=True),
                     "smp": torch.empty((m, W), dtype=torch.int64, pin_memory=True),
                     "red": torch.empty(hlf.REDUCE_WORDS, dtype=torch.int64, pin_memory=True)}
    out_host, smp_host, red_host = host_bufs["out"], host_bufs["smp"], host_bufs["red"]
    stream = torch.cuda.current_stream(dev)

    copy_stream = torch.cuda.Stream(dev)

    def step():
        # The 2^30 stored solutions go to the host on a copy stream while the
        # reduce runs: the copy needs the host link, the reduce the integer
        # pipes. Every byte still reaches host memory inside the step.
        A_dev.copy_(A_host, non_blocking=True)
        idx_dev.copy_(idx_pin, non_blocking=True)
        hh = hlf.hlf_factor(A_dev, n, stream)
        hlf.hlf_enumerate_store(hh, 0, store_n, out, stream)
        stored = torch.cuda.Event()
        stored.record(stream)
        copy_stream.wait_event(stored)
        with torch.cuda.stream(copy_stream):
            out_host.copy_(out, non_blocking=True)
        hlf.hlf_enumerate_reduce(hh, 0, total, red, stream)
        hlf.hlf_sample(hh, idx_dev, m, smp, stream)
        smp_host.copy_(smp, non_blocking=True)
        red_host.copy_(red, non_blocking=True)
        hlf.hlf_destroy(hh)
        torch.cuda.synchronize(dev)

    for _ in range(max(1, args.warmup)):
        step()
    link = d2h_gbs(out_host, out, copy_stream)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    barrier(world)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize(dev)
    dt = max_over_ranks(time.perf_counter() - t0, world)
    barrier(world)
    clk = clocks.stop()
    if int(red_host[0]) != total:
        raise RuntimeError("e2e reduce count mismatch")
    h2d = A_host.numel() * 8 + idx_pin.numel() * 8
    d2h = out_host.numel() * 8 + smp_host.numel() * 8 + red_host.numel() * 8
    return {"value": world * args.steps * total / dt, "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * dt / args.steps,
            "d2h_gbs": link, "clocks": clk}


def d2h_gbs(dst_host, src_dev, stream) -> float:
    """Device-to-host bandwidth into this pinned buffer right now (best of two
    copies, CUDA events). It varies with the state of the host, so the e2e and
    served figures are read against it."""
    import torch

    best = 0.0
    for _ in range(2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record()
            dst_host.copy_(src_dev, non_blocking=True)
            e1.record()
        e1.synchronize()
        best = max(best, src_dev.numel() * src_dev.element_size() / (e0.elapsed_time(e1) * 1e6))
    return best


def run_configs(dev):
    """The two other single-instance workloads, through the C ABI:
    grid3x3 (factor and store every solution, a latency) and grid8x8 (the
    2^40-solution window reduced on the device, and 2^20 samples of it)."""
    import statistics as st

    import numpy as np
    import torch

    from paper_2103_00693_gb300 import hlf
    from synth import workloads as wl

    out = {}
    # grid3x3: factor + store of all 2^r solutions + sync + rank, on the host
    # clock; the store reads r on the device (one host wait). The two-step
    # path (rank to the host, then a store of [0, 2^r)) is timed beside it.
    A3 = torch.from_numpy(hlf.pack_rows(wl.grid3()).view(np.int64)).to(dev)
    n3 = A3.shape[0]
    sols = torch.empty((1 << n3, 1), dtype=torch.int64, device=dev)
    lat, lat2 = [], []
    for k in range(70):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        h = hlf.hlf_factor(A3, n3)
        hlf.hlf_enumerate_store_upto(h, 1 << n3, sols)
        torch.cuda.synchronize(dev)
        r3 = hlf.hlf_get_rank(h)
        if k >= 10:
            lat.append(time.perf_counter() - t0)
        hlf.hlf_destroy(h)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        h = hlf.hlf_factor(A3, n3)
        r3b = hlf.hlf_get_rank(h)
        hlf.hlf_enumerate_store(h, 0, 1 << r3b, sols)
        torch.cuda.synchronize(dev)
        if k >= 10:
            lat2.append(time.perf_counter() - t0)
        hlf.hlf_destroy(h)
    out["grid3x3"] = {"workload": "3x3 grid, p=1/2, seed 5: factor + store every solution",
                      "r": r3, "solutions": 1 << r3, "us_p50": 1e6 * st.median(lat),
                      "us_min": 1e6 * min(lat),
                      "two_step_us_p50": 1e6 * st.median(lat2)}
    # grid8x8: reduce of the 2^40 window, and the 2^20 samples
    A8 = wl.grid8()
    n8 = A8.shape[0]
    h = hlf.hlf_factor(torch.from_numpy(hlf.pack_rows(A8).view(np.int64)).to(dev), n8)
    r8 = hlf.hlf_get_rank(h)
    off, cnt = wl.grid8_window(min(r8, 64))
    red = torch.empty(hlf.REDUCE_WORDS, dtype=torch.int64, device=dev)
    idx = torch.from_numpy(wl.grid8_samples(off, cnt).view(np.int64)).to(dev)
    smp = torch.empty(idx.numel(), dtype=torch.int64, device=dev)
    hlf.hlf_enumerate_reduce(h, off, 1 << 30, red)  # warm-up
    hlf.hlf_sample(h, idx, idx.numel(), smp)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize(dev)
    e[0].record()
    hlf.hlf_enumerate_reduce(h, off, cnt, red)
    e[1].record()
    hlf.hlf_sample(h, idx, idx.numel(), smp)
    e[2].record()
    torch.cuda.synchronize(dev)
    res = hlf.ReduceResult.from_words(red.cpu().numpy(), 1)
    if res.count != cnt:
        raise RuntimeError("grid8x8 window reduce miscounted")
    hlf.hlf_destroy(h)
    r_ms, s_ms = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
    out["grid8x8"] = {"workload": "8x8 grid, p=1/2, seed 0: 2^40-solution window at a seeded offset",
                      "r": r8, "solutions": cnt, "reduce_ms": r_ms, "solutions_per_s": cnt / (r_ms / 1e3),
                      "samples": idx.numel(), "sample_ms": s_ms}
    return out


def batched_ops(Ws, counts, per_solution=None) -> int:
    """Algorithmic 32-bit integer operations of the batched reduce: the
    single-instance reduce's 22W - 4 per solution (18 at W = 1), summed over
    the instances' solution counts; factorisation work is not counted.
    per_solution picks another count (the ALU-pipe one)."""
    f = per_solution or ops_per_solution
    return int(sum(int(c) * f(int(w)) for w, c in zip(Ws, counts)))


def run_batched(args):
    """The batched workload: 4096 grids (N in 4..16, p = 1/2), each reducing
    min(2^r, 2^20) solutions. One persistent launch per step, replayed from a
    CUDA graph with autotuned tiles (warps per item, CTAs per SM, chunk),
    against the same two stages as separate batched calls
    (hlf_factor_batched + hlf_enumerate_batched) and against the plain path
    (a factor launch and a reduce launch per grid, matrices staged on the
    device beforehand, no host wait in between)."""
    import numpy as np
    import torch

    from paper_2103_00693_gb300 import autotune
    from paper_2103_00693_gb300.batch import Batch, PlainPath
    from synth import workloads as wl

    mats = wl.batch()
    cap = 1 << wl.BATCH_CAP_LOG2
    B = Batch(mats)
    tune = autotune.autotune(B, cap, reps=2)
    B.capture(cap)
    for _ in range(max(1, args.warmup)):
        B.replay()
    torch.cuda.synchronize()
    reps = max(3, args.steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        B.replay()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    r, red = B.results()
    counts = [x.count for x in red]
    sols = sum(counts)
    ops = batched_ops(B.Ws, counts)
    ipk, ipk_basis = int_peak()
    alu_ops = batched_ops(B.Ws, counts, alu_pipe_ops_per_solution)
    apk, apk_basis = alu_pipe_peak()
    # the two-call form of the same work
    for _ in range(2):
        B.factor()
        B.reduce(cap)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        B.factor()
        B.reduce(cap)
    e1.record()
    torch.cuda.synchronize()
    split_ms = e0.elapsed_time(e1) / reps
    # the batched store: every grid's first min(2^r, 2^14) solutions, W words
    # each, into one buffer at per-grid offsets (an offsets table of B + 1)
    scap = 1 << 14
    room = np.minimum(np.left_shift(1, np.clip(r.astype(np.int64), 0, 62)), scap) * B.Ws.astype(np.int64)
    out_off = np.concatenate([[0], np.cumsum(room)]).astype(np.int64)
    out_dev = torch.empty(int(out_off[-1]), dtype=torch.int64, device="cuda")
    out_off_dev = torch.from_numpy(out_off).cuda()
    B.store(scap, out_dev, out_off_dev)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        B.store(scap, out_dev, out_off_dev)
    e1.record()
    torch.cuda.synchronize()
    store_ms = e0.elapsed_time(e1) / reps
    store_bytes = int(out_off[-1]) * 8
    del out_dev
    B.close()
    plain = PlainPath(mats)
    plain.run(cap)  # warm-up: pool, module load
    torch.cuda.synchronize()
    e0.record()
    plain.run(cap)
    e1.record()
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1)
    return {"workload": "4096 grids, N uniform 4..16, p=1/2, min(2^r, 2^20) solutions each",
            "ms_per_batch": ms, "inst_per_s": len(mats) / (ms / 1e3), "solutions_per_s": sols / (ms / 1e3),
            "solutions_per_batch": sols,
            "tiles": {"warps_per_item": tune["tiles"][0], "ctas_per_sm": tune["tiles"][1], "chunk": tune["tiles"][2]},
            "launch": "one persistent kernel (+3 memsets) replayed from a CUDA graph",
            "roofline": {"bound": "alu", "achieved": ops / (ms / 1e3) / 1e12, "peak": ipk,
                         "unit": "Tops/s", "frac": ops / (ms / 1e3) / 1e12 / ipk,
                         "ops_per_batch": ops, "ops_per_solution": "22W - 4 (18 at W = 1)",
                         "kernel": "batch_kernel", "peak_basis": ipk_basis},
            "roofline_alu_pipe": {"bound": "alu_pipe", "achieved": alu_ops / (ms / 1e3) / 1e12, "peak": apk,
                                  "unit": "Tops/s", "frac": alu_ops / (ms / 1e3) / 1e12 / apk,
                                  "ops_per_batch": alu_ops, "ops_per_solution": "16W - 4 (12 at W = 1)",
                                  "kernel": "batch_kernel", "peak_basis": apk_basis + " (the pipe that binds)"},
            "split_calls_ms_per_batch": split_ms,
            "store": {"what": "hlf_enumerate_batched storing min(2^r, 2^14) solutions of every grid",
                      "ms": store_ms, "bytes": store_bytes,
                      "roofline": {"bound": "hbm", "achieved": store_bytes / (store_ms / 1e3) / 1e9,
                                   "peak": peaks()["hbm_gbs"], "unit": "GB/s",
                                   "frac": store_bytes / (store_ms / 1e3) / 1e9 / peaks()["hbm_gbs"],
                                   "kernel": "batch_kernel (store chunks)"}},
            "plain_ms_per_batch": plain_ms, "plain_inst_per_s": len(mats) / (plain_ms / 1e3),
            "plain": "per grid: hlf_factor + hlf_enumerate_reduce_upto on one stream, no host wait",
            "speedup_vs_plain": plain_ms / ms}


def run_served(args, srv=None):
    """The served workload: Poisson arrivals, N uniform 3..32, windows
    log-uniform 2^10..2^24 solutions returned to pinned host memory. The
    continuous-batching server and the plain one-request-at-a-time path see
    the same streams at a low and a high arrival rate."""
    from paper_2103_00693_gb300 import serve
    from synth import workloads as wl

    out = {"workload": "Poisson stream, N uniform 3..32 (n <= 1024), p=1/2, windows 2^10..2^24 to host"}
    import torch

    warm = wl.stream(8, 1000.0, seed=1)
    if srv is None:
        srv = serve.Server(keep_results=False)
    srv.run(warm)
    serve.run_plain(warm, keep_results=False)
    words = (1 << 30) // 8
    src = torch.empty(words, dtype=torch.int64, device="cuda")
    out["host_ring_d2h_gbs"] = d2h_gbs(srv.host_ring.buf[:words], src, torch.cuda.Stream())
    del src
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    for name, rate, count in (("low_load", 50.0, 60), ("high_load", 2000.0, 200), ("overload", 5000.0, 300)):
        reqs = wl.stream(count, rate)
        st, _ = srv.run(reqs)
        pl, _ = serve.run_plain(reqs, keep_results=False)
        out[name] = {"rate_per_s": rate, "requests": count, "batched": st.summary(), "plain": pl.summary()}
    out["clocks"] = clocks.stop()
    srv.close()
    return out


def run_sharded(args, world, rank, local):
    """One grid6x6 instance split across the ranks. Each step, every rank
    copies A in from pinned host memory, factors it (microseconds, so it is
    replicated), reduces its contiguous slice of the 2^r indices with
    hlf_enumerate_reduce, reads its partial back, and the partials meet in one
    all-gather and combine (paper_2103_00693_gb300.shard, the code the gloo
    tests run on CPU ranks). Total work is fixed as N grows: strong scaling."""
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2103_00693_gb300 as hlf
    from paper_2103_00693_gb300 import shard
    from synth import workloads as wl

    torch.cuda.set_device(local)
    hlf.load()
    dev = torch.device("cuda", local)
    A = wl.grid6()
    n = A.shape[0]
    W = hlf.words(n)
    A_host = torch.from_numpy(hlf.pack_rows(A).view(np.int64)).pin_memory()
    A_dev = torch.empty_like(A_host, device=dev)
    red = torch.empty(hlf.REDUCE_WORDS, dtype=torch.int64, device=dev)
    red_host = torch.empty(hlf.REDUCE_WORDS, dtype=torch.int64, pin_memory=True)
    coll_dev = "cuda" if world > 1 and dist.get_backend() == "nccl" else "cpu"
    A_dev.copy_(A_host)
    h0 = hlf.hlf_factor(A_dev, n)
    r = hlf.hlf_get_rank(h0)
    hlf.hlf_destroy(h0)
    total = 1 << (r if args.reduce_log2 is None else min(r, args.reduce_log2))
    stream = torch.cuda.current_stream(dev)
    evs = []

    def step(record: bool):
        A_dev.copy_(A_host, non_blocking=True)
        h = hlf.hlf_factor(A_dev, n)

        def reduce_fn(o, c):
            e = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            e[0].record(stream)
            hlf.hlf_enumerate_reduce(h, o, c, red)
            e[1].record(stream)
            if record:
                evs.append(e)
            red_host.copy_(red, non_blocking=True)
            stream.synchronize()
            rr = hlf.ReduceResult.from_words(red_host.numpy(), W)
            return rr.count, rr.hsum, rr.xor_fold

        part = shard.reduce_shard(reduce_fn, 0, total, rank, world)
        got = shard.allgather_combine(part, W, world, coll_dev)
        hlf.hlf_destroy(h)
        return got

    for _ in range(max(3, args.warmup)):
        got = step(False)
    assert got[0] == total, got  # the shards cover the window exactly
    if total == 1 << r and r >= 2:
        assert not got[2].any()   # the full set is an affine space of dimension >= 2
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step(True)
    torch.cuda.synchronize(dev)
    barrier(world)
    dt = max_over_ranks(time.perf_counter() - t0, world)
    clk = clocks.stop()
    k_ms = max_over_ranks(statistics.mean(e[0].elapsed_time(e[1]) for e in evs), world)
    mine = shard.shard_range(0, total, rank, world)[1]
    ipk, ipk_basis = int_peak(dev)
    achieved = mine * ops_per_solution(W) / (k_ms / 1e3) / 1e12
    if rank != 0:
        return
    value = args.steps * total / dt
    cfg = workload_config(r, total)
    cfg["parallelism"] = (f"shards: contiguous index ranges of one instance over {world} GPU(s), "
                          f"one all-gather of {2 + W} words per rank per step")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "u64", "data": "synthetic", "config": cfg,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": ipk, "unit": "Tops/s",
                         "frac": achieved / ipk, "traffic": None, "kernel": "reduce_kernel<1,6,1024>",
                         "ms_per_launch": k_ms, "peak_basis": ipk_basis,
                         "ops_per_solution": ops_per_solution(W)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": A_host.numel() * 8,
                    "d2h_bytes_per_step": red_host.numel() * 8,
                    "note": "the step itself runs through host buffers: A in, the partial out, the exchange"},
            "gpu_launches": 2 * args.steps, "clocks": clk, "combined": {"count": got[0], "hsum": got[1]}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.shard:
        run_sharded(args, world, rank, local)
    else:
        run_hlf(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
