"""Host-side logic of bench.py that needs no GPU: the DRAM-traffic records are
keyed to the kernels' source files, and a record whose sources changed since
its capture is reported as null."""

import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_every_traffic_record_names_its_sources():
    b = _bench()
    assert set(b.TRAFFIC) <= set(b.KERNEL_SOURCES)
    for k, files in b.KERNEL_SOURCES.items():
        for f in files:
            assert os.path.exists(os.path.join(ROOT, "paper_2103_00693_gb300", "csrc", f)), (k, f)


def test_traffic_is_null_once_the_sources_change(monkeypatch):
    b = _bench()
    for k, rec in b.TRAFFIC.items():
        got = b.traffic(k)
        assert got is None or got == rec["bytes"]
        monkeypatch.setattr(b, "source_digest", lambda kernel: "0" * 16)
        assert b.traffic(k) is None
        monkeypatch.undo()
    assert b.traffic("no_such_kernel") is None


def test_operation_counts():
    """The reduce's op count per solution and its ALU-pipe part: 18 and 12 at
    W = 1; every word beyond the first adds 22, of which 16 on the ALU pipe
    (the other 6 are its round's two 64-bit multiplies, 3 IMAD each)."""
    b = _bench()
    assert b.ops_per_solution(1) == 18 and b.alu_pipe_ops_per_solution(1) == 12
    for W in range(1, 17):
        assert b.ops_per_solution(W) - b.alu_pipe_ops_per_solution(W) == 6 * W
    assert b.batched_ops([1, 2], [10, 10], b.alu_pipe_ops_per_solution) == 10 * 12 + 10 * 28
