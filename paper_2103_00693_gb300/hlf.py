"""Python binding of libhlf's C ABI (include/hlf.h), with the same names.

Argument marshalling only: tensors become device pointers, streams become
cudaStream_t handles, status codes become exceptions. Every step of the
solver runs in the library's CUDA kernels; there is no CPU fallback, and
loading fails loudly if libhlf.so has not been built.

Bit layout (as in hlf.h): an n-bit vector is W = ceil(n/64) uint64 words,
bit j in word j // 64 at position j % 64. Device buffers are torch.int64
tensors used as raw 64-bit storage.
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

MAX_N = 1024
MAX_W = 16
BATCH_MAX_N = 256
REDUCE_WORDS = 2 + MAX_W  # hlf_reduce: count, hsum, xor_fold[16]

STATUS = {
    0: "HLF_OK", 1: "HLF_ERR_ARG", 2: "HLF_ERR_SIZE", 3: "HLF_ERR_NOT_SYMMETRIC",
    4: "HLF_ERR_PADDING", 5: "HLF_ERR_RANGE", 6: "HLF_ERR_NOMEM", 7: "HLF_ERR_TIMEOUT",
    8: "HLF_ERR_CUDA", 9: "HLF_ERR_INTERNAL",
}

STATUS_CODES = {v: k for k, v in STATUS.items()}

# Every entry point of include/hlf.h, with its ctypes signature.
_vp = ctypes.c_void_p
_u64 = ctypes.c_uint64
_i32 = ctypes.c_int32
SIGNATURES = {
    "hlf_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "hlf_device_count": (_i32, []),
    "hlf_debug_fail_allocs": (ctypes.c_int, [_i32]),
    "hlf_debug_violation": (ctypes.c_int, [ctypes.POINTER(_u64), ctypes.POINTER(_i32)]),
    "hlf_debug_bounds_probe": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, _vp]),
    "hlf_factor": (ctypes.c_int, [_vp, _i32, _vp, ctypes.POINTER(_vp)]),
    "hlf_get_rank": (ctypes.c_int, [_vp, ctypes.POINTER(_i32)]),
    "hlf_get_factor": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "hlf_get_shape": (ctypes.c_int, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "hlf_set_order": (ctypes.c_int, [_vp, _i32]),
    "hlf_get_status": (ctypes.c_int, [_vp]),
    "hlf_enumerate_store": (ctypes.c_int, [_vp, _u64, _u64, _vp, _vp]),
    "hlf_enumerate_store_upto": (ctypes.c_int, [_vp, _u64, _vp, _vp]),
    "hlf_enumerate_reduce_upto": (ctypes.c_int, [_vp, _u64, _vp, _vp]),
    "hlf_enumerate_store_dense": (ctypes.c_int, [_vp, _u64, _u64, _vp, _vp]),
    "hlf_enumerate_reduce": (ctypes.c_int, [_vp, _u64, _u64, _vp, _vp]),
    "hlf_enumerate_reduce_chunks": (ctypes.c_int, [_vp, _u64, _u64, _u64, _vp, _vp]),
    "hlf_enumerate_histogram": (ctypes.c_int, [_vp, _u64, _u64, _i32, _i32, _vp, _vp]),
    "hlf_sample": (ctypes.c_int, [_vp, _vp, _u64, _vp, _vp]),
    "hlf_destroy": (ctypes.c_int, [_vp]),
    "hlf_many_create": (ctypes.c_int, [_i32, ctypes.POINTER(_vp)]),
    "hlf_enumerate_store_many": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _i32, _vp]),
    "hlf_many_destroy": (ctypes.c_int, [_vp]),
    "hlf_batch_create": (ctypes.c_int, [_i32, ctypes.POINTER(_vp)]),
    "hlf_batch_set_tiles": (ctypes.c_int, [_vp, _i32, _i32, _u64]),
    "hlf_factor_batched": (ctypes.c_int, [_vp, _vp, _vp, _i32, _vp, _vp]),
    "hlf_enumerate_batched": (ctypes.c_int, [_vp, _u64, _vp, _vp, _vp, _vp]),
    "hlf_batch_set_spin_limit": (ctypes.c_int, [_vp, ctypes.c_uint32]),
    "hlf_batch_factor_reduce": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i32, _u64, _vp, _vp, _vp]),
    "hlf_batch_set_debug": (ctypes.c_int, [_vp, ctypes.c_uint32]),
    "hlf_batch_get_status": (ctypes.c_int, [_vp]),
    "hlf_batch_destroy": (ctypes.c_int, [_vp]),
    "hlf_batch_factor_reduce_noalloc": (ctypes.c_int, [_vp, _vp, _vp, _i32, _u64, _vp, _vp, _vp]),
    "hlf_probe_smem_atomics": (ctypes.c_int, [ctypes.c_uint32, _vp, ctypes.POINTER(_u64), _vp]),
}


class HlfError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}")


_LIB = None


def debug_requested() -> bool:
    """HLF_DEBUG=1 selects the debug library (bounds-checked kernels)."""
    return os.environ.get("HLF_DEBUG", "") == "1"


def lib_path() -> str:
    return _build.LIB_DEBUG if debug_requested() else _build.LIB


def load(build_if_missing: bool = False):
    """Load libhlf.so (libhlf_debug.so under HLF_DEBUG=1). Raises if it is
    missing (unless build_if_missing)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"{os.path.basename(path)} is not built ({path}); run __graft_entry__.build()")
        _build.build(debug=debug_requested())
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _check(st: int, where: str):
    if st != 0:
        raise HlfError(st, where)


def _stream_ptr(stream) -> int | None:
    import torch

    if stream is None:
        # the raw pointer of the current stream, without building a Stream object
        raw = getattr(torch._C, "_cuda_getCurrentRawStream", None)
        dev = getattr(torch._C, "_cuda_getDevice", None)
        if raw is not None and dev is not None and torch.cuda.is_initialized():
            return raw(dev()) or None
        stream = torch.cuda.current_stream()
    return stream.cuda_stream or None


def _ptr(t) -> int:
    return t.data_ptr()


def words(n: int) -> int:
    return (n + 63) // 64


def pack_rows(A: np.ndarray) -> np.ndarray:
    """Pack a dense 0/1 matrix [rows, n] into uint64 words [rows, W] (host-side
    argument marshalling for hlf_factor)."""
    A = np.asarray(A, dtype=np.uint8)
    rows, n = A.shape
    W = words(n)
    b = np.packbits(A, axis=1, bitorder="little")  # [rows, ceil(n / 8)], bits past n are 0
    if b.shape[1] != W * 8:
        full = np.zeros((rows, W * 8), dtype=np.uint8)
        full[:, :b.shape[1]] = b
        b = full
    return np.ascontiguousarray(b).view("<u8").reshape(rows, W).astype(np.uint64)


def unpack_rows(words_: np.ndarray, n: int) -> np.ndarray:
    w = np.ascontiguousarray(np.asarray(words_, dtype=np.uint64))
    if w.ndim == 1:
        w = w[:, None]
    b = np.unpackbits(w.view(np.uint8).reshape(w.shape[0], -1), axis=1, bitorder="little")
    return b[:, :n]


@dataclass
class ReduceResult:
    count: int
    hsum: int
    xor_fold: np.ndarray  # uint64 [W]

    @staticmethod
    def from_words(r, W: int) -> "ReduceResult":
        r = np.asarray(r).astype(np.int64).view(np.uint64)
        return ReduceResult(int(r[0]), int(r[1]), r[2:2 + W].copy())


# ----------------------------------------------------------------- entry points

def hlf_status_string(status: int) -> str:
    return load().hlf_status_string(status).decode()


def hlf_device_count() -> int:
    return int(load().hlf_device_count())


def hlf_debug_fail_allocs(count: int):
    """Fault injection for tests: the next `count` allocating calls fail with
    HLF_ERR_NOMEM (host-side; no GPU involved)."""
    _check(load().hlf_debug_fail_allocs(count), "hlf_debug_fail_allocs")


def hlf_debug_violation() -> tuple[int, bool]:
    """(the first failed bounds check recorded since the last call, 0 if none,
    2^63 | site << 48 | index mod 2^48; whether the loaded library is the
    debug build). Synchronises the device and clears the record."""
    first, dbg = _u64(0), _i32(0)
    _check(load().hlf_debug_violation(ctypes.byref(first), ctypes.byref(dbg)), "hlf_debug_violation")
    return int(first.value), bool(dbg.value)


def hlf_debug_bounds_probe(i: int, n: int, stream=None):
    """One device thread checks index i against [0, n) (site 1), touching no
    memory: a failed check is recorded in the debug build."""
    _check(load().hlf_debug_bounds_probe(i, n, _stream_ptr(stream)), "hlf_debug_bounds_probe")


def hlf_factor(A_dev, n: int, stream=None) -> int:
    """Stage 1 (CLA module): A_dev is a CUDA int64 tensor [n, W]; returns the
    handle (an opaque pointer value)."""
    if not A_dev.is_cuda or A_dev.dtype.itemsize != 8 or not A_dev.is_contiguous():
        raise ValueError("A_dev must be a contiguous 64-bit CUDA tensor [n, W]")
    h = _vp()
    _check(load().hlf_factor(_ptr(A_dev), n, _stream_ptr(stream), ctypes.byref(h)), "hlf_factor")
    return h.value


def hlf_get_rank(h: int) -> int:
    r = _i32()
    _check(load().hlf_get_rank(h, ctypes.byref(r)), "hlf_get_rank")
    return r.value


ORDER_GRAY = 0
ORDER_PAPER = 1


def hlf_set_order(h: int, order: int):
    _check(load().hlf_set_order(h, order), "hlf_set_order")


def hlf_get_shape(h: int) -> tuple[int, int]:
    n, W = _i32(), _i32()
    _check(load().hlf_get_shape(h, ctypes.byref(n), ctypes.byref(W)), "hlf_get_shape")
    return n.value, W.value


def hlf_get_factor(h: int):
    """(piv int32[r], z0 uint64[W], basis uint64[r, W]) copied to the host."""
    r = hlf_get_rank(h)
    _, W = hlf_get_shape(h)
    piv = np.zeros(max(r, 1), dtype=np.int32)
    z0 = np.zeros(W, dtype=np.uint64)
    basis = np.zeros((max(r, 1), W), dtype=np.uint64)
    _check(load().hlf_get_factor(h, piv.ctypes.data, z0.ctypes.data, basis.ctypes.data), "hlf_get_factor")
    return piv[:r], z0, basis[:r]


def hlf_get_status(h: int) -> int:
    return int(load().hlf_get_status(h))


def hlf_enumerate_store(h: int, offset: int, count: int, out_dev, stream=None):
    _check(load().hlf_enumerate_store(h, offset, count, _ptr(out_dev) if out_dev is not None else None,
                                      _stream_ptr(stream)), "hlf_enumerate_store")


def hlf_enumerate_store_upto(h: int, cap: int, out_dev, stream=None):
    """Every solution z(i), i < min(2^r, cap), into out_dev [cap, W], with r
    read on the device: no host wait after hlf_factor."""
    _check(load().hlf_enumerate_store_upto(h, cap, _ptr(out_dev) if out_dev is not None else None,
                                           _stream_ptr(stream)), "hlf_enumerate_store_upto")


def hlf_enumerate_reduce_upto(h: int, cap: int, red_dev, stream=None):
    """Reduce of [0, min(2^r, cap)) into red_dev [18] with r read on the
    device: no host wait after hlf_factor."""
    _check(load().hlf_enumerate_reduce_upto(h, cap, _ptr(red_dev), _stream_ptr(stream)),
           "hlf_enumerate_reduce_upto")


def hlf_enumerate_store_dense(h: int, offset: int, count: int, out_dev, stream=None):
    _check(load().hlf_enumerate_store_dense(h, offset, count, _ptr(out_dev) if out_dev is not None else None,
                                            _stream_ptr(stream)), "hlf_enumerate_store_dense")


def dense_words(count: int, n: int) -> int:
    """Words of a dense stream of `count` solutions of n bits."""
    return (count * n + 63) // 64


def hlf_enumerate_reduce(h: int, offset: int, count: int, red_dev, stream=None):
    _check(load().hlf_enumerate_reduce(h, offset, count, _ptr(red_dev), _stream_ptr(stream)),
           "hlf_enumerate_reduce")


def hlf_enumerate_reduce_chunks(h: int, offset: int, chunk: int, n_chunks: int, red_dev, stream=None):
    _check(load().hlf_enumerate_reduce_chunks(h, offset, chunk, n_chunks,
                                              _ptr(red_dev) if red_dev is not None else None,
                                              _stream_ptr(stream)), "hlf_enumerate_reduce_chunks")


def hlf_enumerate_histogram(h: int, offset: int, count: int, bit_lo: int, nbits: int, hist_dev, stream=None):
    _check(load().hlf_enumerate_histogram(h, offset, count, bit_lo, nbits, _ptr(hist_dev), _stream_ptr(stream)),
           "hlf_enumerate_histogram")


def hlf_sample(h: int, idx_dev, m: int, out_dev, stream=None):
    _check(load().hlf_sample(h, _ptr(idx_dev) if idx_dev is not None else None, m,
                             _ptr(out_dev) if out_dev is not None else None, _stream_ptr(stream)),
           "hlf_sample")


def hlf_destroy(h: int):
    _check(load().hlf_destroy(h), "hlf_destroy")


def hlf_many_create(max_windows: int) -> int:
    m = _vp()
    _check(load().hlf_many_create(max_windows, ctypes.byref(m)), "hlf_many_create")
    return m.value


def hlf_enumerate_store_many(m: int, handles, offsets, counts, outs, stream=None):
    """handles: list of handle values; offsets/counts: lists of ints; outs:
    list of CUDA tensors (each [count_j, W_j] 64-bit)."""
    k = len(handles)
    hs = (_vp * max(k, 1))(*handles)
    offs = (_u64 * max(k, 1))(*offsets)
    cnts = (_u64 * max(k, 1))(*counts)
    outp = (_vp * max(k, 1))(*[o.data_ptr() for o in outs])
    _check(load().hlf_enumerate_store_many(m, hs, offs, cnts, outp, k, _stream_ptr(stream)),
           "hlf_enumerate_store_many")


def hlf_many_destroy(m: int):
    _check(load().hlf_many_destroy(m), "hlf_many_destroy")


def hlf_batch_create(max_instances: int) -> int:
    b = _vp()
    _check(load().hlf_batch_create(max_instances, ctypes.byref(b)), "hlf_batch_create")
    return b.value


def hlf_batch_set_tiles(b: int, warps_per_item: int, ctas_per_sm: int, chunk: int):
    _check(load().hlf_batch_set_tiles(b, warps_per_item, ctas_per_sm, chunk), "hlf_batch_set_tiles")


def hlf_factor_batched(b: int, A_dev, offsets_dev, count: int, r_dev, stream=None):
    """Stage 1 of `count` matrices packed back to back in A_dev, matrix b in
    words [offsets_dev[b], offsets_dev[b+1]) (offsets: int64 [count + 1])."""
    _check(load().hlf_factor_batched(b, _ptr(A_dev), _ptr(offsets_dev), count, _ptr(r_dev), _stream_ptr(stream)),
           "hlf_factor_batched")


def hlf_enumerate_batched(b: int, cap: int, red_dev=None, out_dev=None, out_offsets_dev=None, stream=None):
    """Stage 2 of the plan's factored matrices: reduce into red_dev [count,
    18], or store into out_dev at out_offsets_dev (int64 [count + 1])."""
    _check(load().hlf_enumerate_batched(b, cap, _ptr(red_dev) if red_dev is not None else None,
                                        _ptr(out_dev) if out_dev is not None else None,
                                        _ptr(out_offsets_dev) if out_offsets_dev is not None else None,
                                        _stream_ptr(stream)), "hlf_enumerate_batched")


def hlf_batch_set_spin_limit(b: int, polls: int):
    _check(load().hlf_batch_set_spin_limit(b, polls), "hlf_batch_set_spin_limit")


def hlf_batch_factor_reduce(b: int, A_dev, word_off_dev, n_dev, count: int, cap: int, r_dev, red_dev,
                            stream=None):
    _check(load().hlf_batch_factor_reduce(b, _ptr(A_dev), _ptr(word_off_dev), _ptr(n_dev), count, cap,
                                          _ptr(r_dev), _ptr(red_dev), _stream_ptr(stream)),
           "hlf_batch_factor_reduce")


def hlf_batch_set_debug(b: int, flags: int):
    _check(load().hlf_batch_set_debug(b, flags), "hlf_batch_set_debug")


def hlf_batch_get_status(b: int) -> int:
    return int(load().hlf_batch_get_status(b))


def hlf_batch_destroy(b: int):
    _check(load().hlf_batch_destroy(b), "hlf_batch_destroy")


BATCH_NOALLOC_MAX = 1024


def hlf_batch_factor_reduce_noalloc(A_dev, word_off_dev, n_dev, count: int, cap: int, r_dev, red_dev,
                                    stream=None):
    """hlf_batch_factor_reduce without a plan and without any allocation in
    the library: for callers that cannot allocate device memory when they
    call (see include/hlf.h). At most BATCH_NOALLOC_MAX matrices per call;
    calls must not overlap on the GPU. The first call on a device may load
    the library's device code and so allocate: warm up before a region that
    must not. A bounded wait that ran out shows only as red[b].count below
    min(2^r[b], cap): compare the two to detect it."""
    _check(load().hlf_batch_factor_reduce_noalloc(_ptr(A_dev), _ptr(word_off_dev), _ptr(n_dev), count, cap,
                                                  _ptr(r_dev), _ptr(red_dev), _stream_ptr(stream)),
           "hlf_batch_factor_reduce_noalloc")


# ------------------------------------------------------------ convenience layer

class Factorization:
    """Owns one hlf_handle: the stage-1 result of one matrix, resident on the
    device, from which any window of solutions can be enumerated."""

    def __init__(self, A_dev, n: int, stream=None):
        self.n = n
        self.W = words(n)
        self.h = hlf_factor(A_dev, n, stream)

    @classmethod
    def from_dense(cls, A: np.ndarray, device="cuda", stream=None) -> "Factorization":
        import torch

        packed = pack_rows(A)
        A_dev = torch.from_numpy(packed.view(np.int64)).to(device)
        f = cls(A_dev, A.shape[0], stream)
        f._keep = A_dev  # A must stay alive until the factor kernel has run
        return f

    @property
    def rank(self) -> int:
        return hlf_get_rank(self.h)

    def space_log2(self) -> int:
        return min(self.rank, 64)

    def factor_host(self):
        return hlf_get_factor(self.h)

    def store(self, offset: int, count: int, out=None, stream=None):
        import torch

        if out is None:
            out = torch.empty((count, self.W), dtype=torch.int64, device="cuda")
        hlf_enumerate_store(self.h, offset, count, out, stream)
        return out

    def store_upto(self, cap: int, out=None, stream=None):
        """Solutions [0, min(2^r, cap)) into out [cap, W] without a host wait
        for r; the first min(2^r, cap) rows are valid once the stream is done."""
        import torch

        if out is None:
            out = torch.empty((cap, self.W), dtype=torch.int64, device="cuda")
        hlf_enumerate_store_upto(self.h, cap, out, stream)
        return out

    def store_dense(self, offset: int, count: int, out=None, stream=None):
        import torch

        if out is None:
            out = torch.empty(max(dense_words(count, self.n), 1), dtype=torch.int64, device="cuda")
        hlf_enumerate_store_dense(self.h, offset, count, out, stream)
        return out

    def reduce(self, offset: int, count: int, red=None, stream=None):
        import torch

        if red is None:
            red = torch.empty(REDUCE_WORDS, dtype=torch.int64, device="cuda")
        hlf_enumerate_reduce(self.h, offset, count, red, stream)
        return red

    def reduce_chunks(self, offset: int, chunk: int, n_chunks: int, red=None, stream=None):
        import torch

        if red is None:
            red = torch.empty((n_chunks, REDUCE_WORDS), dtype=torch.int64, device="cuda")
        hlf_enumerate_reduce_chunks(self.h, offset, chunk, n_chunks, red, stream)
        return red

    def histogram(self, offset: int, count: int, bit_lo: int, nbits: int, out=None, stream=None):
        import torch

        if out is None:
            out = torch.empty(1 << nbits, dtype=torch.int64, device="cuda")
        hlf_enumerate_histogram(self.h, offset, count, bit_lo, nbits, out, stream)
        return out

    def sample(self, idx_dev, out=None, stream=None):
        import torch

        m = idx_dev.numel()
        if out is None:
            out = torch.empty((m, self.W), dtype=torch.int64, device="cuda")
        hlf_sample(self.h, idx_dev, m, out, stream)
        return out

    def status(self) -> int:
        return hlf_get_status(self.h)

    def set_order(self, order: int):
        """ORDER_GRAY (default) or ORDER_PAPER for the later stage-2 calls."""
        hlf_set_order(self.h, order)

    def close(self):
        if self.h:
            hlf_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hlf_probe_smem_atomics(iters: int, sum_dev, stream=None) -> int:
    """Launch the shared-memory atomic microbenchmark (a measurement helper,
    not part of the method); returns the number of atomics it performs, which
    sum_dev (one int64 on the device) also receives."""
    n = _u64()
    _check(load().hlf_probe_smem_atomics(iters, _ptr(sum_dev), ctypes.byref(n), _stream_ptr(stream)),
           "hlf_probe_smem_atomics")
    return n.value
