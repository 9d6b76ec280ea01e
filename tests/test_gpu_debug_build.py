"""The debug build (libhlf_debug.so, compiled with -DHLF_DEBUG): every
solution store is checked against its output buffer, and the factor's and
the histogram's shared tables against their sizes. A failed check skips the
access and is recorded on the device (never a trap), so these runs cannot
fault the GPU; the kernels' own parity tests, rerun on the debug library,
must leave no record (the conftest hook checks after every test)."""

import os
import re
import subprocess
import sys

import pytest

from paper_2103_00693_gb300 import hlf

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DEBUG_RUN = ["tests/test_gpu_stage1.py", "tests/test_gpu_stage2.py", "tests/test_gpu_paper_order.py",
             "tests/test_gpu_dense.py", "tests/test_gpu_batch.py", "tests/test_gpu_hist.py",
             "tests/test_gpu_many.py", "tests/test_gpu_upto.py", "tests/test_gpu_fuzz.py"]


def _debug_env():
    env = dict(os.environ)
    env["HLF_DEBUG"] = "1"
    return env


@pytest.fixture(scope="module")
def debug_lib():
    from paper_2103_00693_gb300 import build

    return build.build(debug=True)


def test_probe_records_a_failed_check(cuda_ok, debug_lib):
    """An index inside [0, n) passes; the first one outside is recorded with
    its site and index, a later one is not, and reading the record clears it."""
    code = "\n".join([
        "from paper_2103_00693_gb300 import hlf",
        "assert hlf.hlf_debug_violation() == (0, True)",
        "hlf.hlf_debug_bounds_probe(2, 3)",
        "assert hlf.hlf_debug_violation() == (0, True)",
        "hlf.hlf_debug_bounds_probe(5, 3)",
        "hlf.hlf_debug_bounds_probe(-1, 3)",
        "v, d = hlf.hlf_debug_violation()",
        "assert d and v == (1 << 63) | (1 << 48) | 5, hex(v)",
        "assert hlf.hlf_debug_violation() == (0, True)",
    ])
    res = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=_debug_env(), capture_output=True,
                         text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]


def test_release_build_checks_nothing(cuda_ok):
    if hlf.debug_requested():
        pytest.skip("this process runs the debug library")
    hlf.hlf_debug_bounds_probe(5, 3)
    assert hlf.hlf_debug_violation() == (0, False)


def test_kernels_pass_their_bounds_checks(cuda_ok, debug_lib):
    """The stage-1, stage-2, paper-order, dense, batched, histogram, many,
    upto and random-sweep parity tests on the debug library: all pass, no
    check fails."""
    if hlf.debug_requested():
        pytest.skip("already inside the debug run")
    cmd = [sys.executable, "-m", "pytest", *DEBUG_RUN, "-x", "-q", "-m", "gpu", "-p", "no:cacheprovider"]
    res = subprocess.run(cmd, cwd=ROOT, env=_debug_env(), capture_output=True, text=True, timeout=2400)
    assert res.returncode == 0, res.stdout[-3000:] + res.stderr[-2000:]
    ran = re.search(r"(\d+) passed", res.stdout)
    assert ran and int(ran.group(1)) >= 350, res.stdout[-500:]  # the files hold ~370 GPU tests
