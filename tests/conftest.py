import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libhlf.so")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def expand_b(s: str) -> str:
    """Expand the paper's shorthand 0^(m) / 1^(m) in a diagonal string."""
    out, i = [], 0
    while i < len(s):
        if i + 2 < len(s) and s[i + 1] == "^" and s[i + 2] == "(":
            j = s.index(")", i)
            out.append(s[i] * int(s[i + 3:j]))
            i = j + 1
        else:
            out.append(s[i])
            i += 1
    return "".join(out)


def read_golden(name: str):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append(line.split())
    return rows


@pytest.fixture(scope="session")
def cuda_ok():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return True


@pytest.fixture(autouse=True)
def _debug_build_bounds(request):
    """Under HLF_DEBUG=1 (the bounds-checked debug library) a GPU test also
    fails if a kernel it ran recorded a failed bounds check."""
    yield
    if os.environ.get("HLF_DEBUG") != "1" or request.node.get_closest_marker("gpu") is None:
        return
    from paper_2103_00693_gb300 import hlf

    first, is_debug = hlf.hlf_debug_violation()
    assert is_debug, "HLF_DEBUG=1 but the loaded library is the release build"
    assert first == 0, f"failed bounds check: site {(first >> 48) & 0x7fff}, index {first & ((1 << 48) - 1)}"
