"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/hlf.h declares. Only host-side paths run here (no GPU calls): status
strings and argument checks that return before any CUDA work."""

import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2103_00693_gb300 as hlf
from paper_2103_00693_gb300 import build as hbuild
from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "hlf.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hlf_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    hbuild.build()
    return hlf.load()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("hlf_factor", "hlf_get_rank", "hlf_get_factor", "hlf_enumerate_store",
                 "hlf_enumerate_reduce", "hlf_sample", "hlf_destroy"):
        assert name in syms


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", hbuild.LIB], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (hlf_[a-z0-9_]+)$", out, flags=re.M))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, f"declared but not exported: {missing}"
    for s in declared_symbols():
        assert hasattr(lib, s)
        assert s in hlf.SIGNATURES, f"binding lacks {s}"


def test_library_is_sm103a_only():
    """The build targets exactly compute_103a / sm_103a."""
    assert hbuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_status_strings(lib):
    for code, name in hlf.STATUS.items():
        assert hlf.hlf_status_string(code)
    assert "symmetric" in hlf.hlf_status_string(3)


def test_host_side_argument_checks(lib):
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: checks fail first
    assert lib.hlf_factor(None, 4, None, ctypes.byref(h)) == 1  # HLF_ERR_ARG
    assert lib.hlf_factor(fake, 0, None, ctypes.byref(h)) == 2  # HLF_ERR_SIZE
    assert lib.hlf_factor(fake, 1025, None, ctypes.byref(h)) == 2
    assert lib.hlf_factor(fake, 4, None, None) == 1
    assert h.value is None
    r = ctypes.c_int32()
    assert lib.hlf_get_rank(None, ctypes.byref(r)) == 1
    assert lib.hlf_enumerate_store(None, 0, 1, fake, None) == 1
    assert lib.hlf_enumerate_store_upto(None, 1, fake, None) == 1
    assert lib.hlf_enumerate_reduce(None, 0, 1, fake, None) == 1
    assert lib.hlf_sample(None, fake, 1, fake, None) == 1
    assert lib.hlf_get_status(None) == 1
    assert lib.hlf_destroy(None) == 0


def test_pack_rows_matches_oracle_packer():
    """The binding's host-side packing and the oracle's own packer agree."""
    from oracle.cpu import pack_rows as oracle_pack

    rng = np.random.default_rng(5)
    for n in (1, 9, 63, 64, 65, 130, 1024):
        A = (rng.random((7, n)) < 0.5).astype(np.uint8)
        assert np.array_equal(hlf.pack_rows(A), oracle_pack(A))
        assert np.array_equal(hlf.unpack_rows(hlf.pack_rows(A), n), A)


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    """No silent fallback: a missing libhlf.so is an error."""
    from paper_2103_00693_gb300 import hlf as mod

    monkeypatch.setattr(mod, "_LIB", None)
    monkeypatch.setattr(hbuild, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        mod.load()


def test_injected_allocation_failures_are_nomem(lib):
    """hlf_debug_fail_allocs makes the next allocating calls return
    HLF_ERR_NOMEM after their argument checks, with no GPU involved; argument
    errors still come first and do not consume an injected failure."""
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(0x1000)
    assert lib.hlf_debug_fail_allocs(-1) == 1
    assert lib.hlf_debug_fail_allocs(3) == 0
    assert lib.hlf_factor(fake, 0, None, ctypes.byref(h)) == 2      # size check first
    assert lib.hlf_factor(fake, 9, None, ctypes.byref(h)) == 6      # injected
    assert h.value is None
    m = ctypes.c_void_p()
    assert lib.hlf_many_create(16, ctypes.byref(m)) == 6
    b = ctypes.c_void_p()
    assert lib.hlf_batch_create(16, ctypes.byref(b)) == 6
    assert m.value is None and b.value is None
    assert lib.hlf_debug_fail_allocs(0) == 0


def test_release_library_is_not_the_debug_build(lib):
    """The release library reports that it is not the debug build and that
    no check failed, without touching a GPU; null pointers are HLF_ERR_ARG."""
    first, dbg = ctypes.c_uint64(7), ctypes.c_int32(7)
    assert lib.hlf_debug_violation(ctypes.byref(first), ctypes.byref(dbg)) == 0
    assert (first.value, dbg.value) == (0, 0)
    assert lib.hlf_debug_violation(None, ctypes.byref(dbg)) == 1
    assert lib.hlf_debug_violation(ctypes.byref(first), None) == 1


def test_package_reexports_every_entry_point():
    """Every C entry point has a same-named function in the package (the
    status-string and device-count helpers included)."""
    missing = [name for name in hlf.SIGNATURES if not hasattr(hlf, name)]
    assert not missing, missing


def test_batched_and_upto_argument_checks(lib):
    """The batched calls and the device-rank reduce check their arguments on
    the host before touching the GPU."""
    fake = ctypes.c_void_p(0x1000)
    assert lib.hlf_factor_batched(None, fake, fake, 4, fake, None) == 1
    assert lib.hlf_enumerate_batched(None, 16, fake, None, None, None) == 1
    assert lib.hlf_enumerate_reduce_upto(None, 16, fake, None) == 1
    assert lib.hlf_batch_set_tiles(None, 8, 0, 256) == 1
