"""bench.py end to end on a small case: one JSON line with every key the
measurement contract asks for, and figures that make sense (no number is
checked against a target here; the values are whatever this GPU measures)."""

import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_line_has_every_field(cuda_ok):
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "3", "--warmup", "3",
           "--reduce-log2", "28", "--store-log2", "22", "--no-batched", "--no-served", "--cpu-seconds", "1"]
    res = subprocess.run(cmd, capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "roofline_store", "gpu_launches",
              "clocks", "e2e", "cpu_baseline", "next_rows", "configs"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 3 and d["warmup"] == 3
    assert d["value"] > 0 and d["higher_is_better"] is True
    for r in (d["roofline"], d["roofline_store"]):
        for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
            assert k in r, k
        assert 0 < r["frac"] < 1.5
    assert d["gpu_launches"] == 4 * d["steps"]
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    c = d["cpu_baseline"]
    assert c["kind"] == "oracle" and c["cores"] >= 1 and c["value"] > 0
    assert d["configs"]["grid8x8"]["solutions"] == 1 << 40
    assert d["configs"]["grid3x3"]["solutions"] == 512
    # a timed region this short may end before nvidia-smi's first sample
    assert d["clocks"] is None or set(d["clocks"]) >= {"sm_mhz", "sm_max_mhz", "reasons"}


def test_bench_sharded_mode_line(cuda_ok):
    """bench.py --shard on one GPU: the shard/all-gather/combine path the
    multi-GPU runs use (here with one rank), one JSON line with strong
    scaling and the combined reduce covering the whole window."""
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--shard", "--steps", "3", "--warmup", "3",
           "--reduce-log2", "30"]
    res = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["scaling"] == "strong" and d["n_gpus"] == 1 and d["value"] > 0
    assert d["combined"]["count"] == 1 << 30
    assert 0 < d["roofline"]["frac"] < 1.5 and d["gpu_launches"] == 6
    assert set(d["e2e"]) >= {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"}
