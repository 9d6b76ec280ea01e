"""ctypes wrapper of the C oracle (hlf_oracle.c): the method restated
step by step on the CPU.

Test infrastructure only. See the package docstring for what pins each
function.
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from .build import build_oracle

_u8p = ctypes.POINTER(ctypes.c_uint8)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u64p = ctypes.POINTER(ctypes.c_uint64)

_LIB = None

ERRORS = {-1: "bad argument", -3: "A is not symmetric", -5: "window outside the index space",
          -6: "out of memory", -9: "inconsistent system"}


class OracleError(RuntimeError):
    pass


def bind(path: str):
    """Load an oracle library from `path` and declare its signatures."""
    lib = ctypes.CDLL(path)
    lib.orc_version.restype = ctypes.c_int
    lib.orc_mix64.restype = ctypes.c_uint64
    lib.orc_mix64.argtypes = [ctypes.c_uint64]
    lib.orc_factor.restype = ctypes.c_int
    lib.orc_factor.argtypes = [_u8p, ctypes.c_int, _i32p, _u8p, _u8p, _i32p, _i32p, _u8p]
    for name in ("orc_window", "orc_window_gray"):
        f = getattr(lib, name)
        f.restype = ctypes.c_int
        f.argtypes = [_u8p, _u8p, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, _u64p]
    lib.orc_reduce.restype = ctypes.c_int
    lib.orc_reduce.argtypes = [_u8p, _u8p, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                               ctypes.c_uint64, ctypes.c_int, _u64p]
    lib.orc_paper_order.restype = ctypes.c_int
    lib.orc_paper_order.argtypes = [_u8p, _i32p, ctypes.c_int, _u8p, ctypes.c_int,
                                    ctypes.c_uint64, ctypes.c_uint64, _u64p]
    return lib


def _lib():
    global _LIB
    if _LIB is None:
        _LIB = bind(build_oracle())
    return _LIB


def _check(rc: int) -> int:
    if rc < 0:
        raise OracleError(ERRORS.get(rc, f"oracle error {rc}"))
    return rc


def _p(arr, typ):
    return arr.ctypes.data_as(typ)


@dataclass
class Factor:
    """Stage-1 result (§2, CLA steps (1)-(4)) as the oracle computes it."""

    A: np.ndarray          # [n, n] uint8, the input
    n: int
    r: int
    piv: np.ndarray        # [r] int32, pivot columns p_1 < ... < p_r (0-based)
    R: np.ndarray          # [n, n] uint8, RREF; rows < r are B_1..B_r
    X: np.ndarray          # [n - r, n] uint8, kernel basis x_f
    free: np.ndarray       # [n - r] int32, the free column f of each x_f
    q: np.ndarray          # [n - r] int32, q(x_f) mod 4
    z0: np.ndarray         # [n] uint8, the particular solution z^a

    @property
    def W(self) -> int:
        return (self.n + 63) // 64

    @property
    def basis(self) -> np.ndarray:
        return self.R[: self.r]

    def basis_words(self, limit: int | None = None) -> np.ndarray:
        k = self.r if limit is None else min(self.r, limit)
        return pack_rows(self.R[:k])

    def z0_words(self) -> np.ndarray:
        return pack_rows(self.z0[None, :])[0]

    def space_log2(self) -> int:
        """log2 of the addressable index space, min(r, 64)."""
        return min(self.r, 64)


def pack_rows(bits: np.ndarray) -> np.ndarray:
    """Pack 0/1 rows into uint64 words: bit j of row i goes to word j // 64,
    bit j % 64 (the oracle's own packer)."""
    bits = np.asarray(bits, dtype=np.uint8)
    rows, n = bits.shape
    W = (n + 63) // 64
    out = np.zeros((rows, W), dtype=np.uint64)
    for j in range(n):
        out[:, j // 64] |= bits[:, j].astype(np.uint64) << np.uint64(j % 64)
    return out


def unpack_rows(words: np.ndarray, n: int) -> np.ndarray:
    words = np.asarray(words, dtype=np.uint64)
    if words.ndim == 1:
        words = words[:, None]
    out = np.zeros((words.shape[0], n), dtype=np.uint8)
    for j in range(n):
        out[:, j] = ((words[:, j // 64] >> np.uint64(j % 64)) & np.uint64(1)).astype(np.uint8)
    return out


def mix64(x: int) -> int:
    return int(_lib().orc_mix64(ctypes.c_uint64(x)))


def factor(A: np.ndarray) -> Factor:
    A = np.ascontiguousarray(A, dtype=np.uint8)
    n = A.shape[0]
    piv = np.zeros(n, dtype=np.int32)
    R = np.zeros((n, n), dtype=np.uint8)
    X = np.zeros((n, n), dtype=np.uint8)
    free = np.zeros(n, dtype=np.int32)
    q = np.zeros(n, dtype=np.int32)
    z0 = np.zeros(n, dtype=np.uint8)
    r = _check(_lib().orc_factor(_p(A, _u8p), n, _p(piv, _i32p), _p(R, _u8p), _p(X, _u8p),
                                 _p(free, _i32p), _p(q, _i32p), _p(z0, _u8p)))
    return Factor(A=A, n=n, r=r, piv=piv[:r].copy(), R=R, X=X[: n - r].copy(),
                  free=free[: n - r].copy(), q=q[: n - r].copy(), z0=z0)


def window(F: Factor, offset: int, count: int) -> np.ndarray:
    """z(i) for i in [offset, offset+count), from the direct formula."""
    out = np.zeros((count, F.W), dtype=np.uint64)
    _check(_lib().orc_window(_p(F.R, _u8p), _p(F.z0, _u8p), F.n, F.r, offset, count, _p(out, _u64p)))
    return out


def window_gray(F: Factor, offset: int, count: int) -> np.ndarray:
    """The same window, by Gray stepping from a seed at `offset`."""
    out = np.zeros((count, F.W), dtype=np.uint64)
    _check(_lib().orc_window_gray(_p(F.R, _u8p), _p(F.z0, _u8p), F.n, F.r, offset, count, _p(out, _u64p)))
    return out


def reduce(F: Factor, offset: int, count: int, threads: int | None = None):
    """(count, hsum, xor_fold[W]) of the window [offset, offset+count)."""
    if threads is None:
        threads = os.cpu_count() or 1
    res = np.zeros(2 + F.W, dtype=np.uint64)
    _check(_lib().orc_reduce(_p(F.R, _u8p), _p(F.z0, _u8p), F.n, F.r, offset, count, threads,
                             _p(res, _u64p)))
    return int(res[0]), int(res[1]), res[2:].copy()


def paper_order(F: Factor, t0: int, count: int) -> np.ndarray:
    """Counter values t in [t0, t0+count) in the paper's order: R^(r) = t on
    the pivots, z = A R XOR z^a (Eq. 3)."""
    out = np.zeros((count, F.W), dtype=np.uint64)
    _check(_lib().orc_paper_order(_p(F.A, _u8p), _p(F.piv, _i32p), F.r, _p(F.z0, _u8p), F.n,
                                  t0, count, _p(out, _u64p)))
    return out


def dense_stream(rows_bits: np.ndarray) -> np.ndarray:
    """Solutions as one packed bit stream: solution t's bit j is stream bit
    t * n + j, and stream bit b is bit b % 64 of word b // 64 (LSB first).
    Bits past the last solution in the last word are 0."""
    rows_bits = np.asarray(rows_bits, dtype=np.uint8)
    count, n = rows_bits.shape
    total = count * n
    words = (total + 63) // 64
    flat = np.zeros(words * 64, dtype=np.uint8)
    flat[:total] = rows_bits.reshape(-1)
    out = np.zeros(words, dtype=np.uint64)
    for b in range(64):
        out |= flat[b::64].astype(np.uint64) << np.uint64(b)
    return out


def window_dense(F: Factor, offset: int, count: int) -> np.ndarray:
    """The window [offset, offset+count) as a dense bit stream of n bits per
    solution (see dense_stream)."""
    return dense_stream(unpack_rows(window(F, offset, count), F.n))


def histogram(F: Factor, offset: int, count: int, bit_lo: int, nbits: int, order: str = "gray") -> np.ndarray:
    """Counts over the window of the value of bits bit_lo .. bit_lo+nbits-1
    of each solution (bit bit_lo least significant), from the oracle's own
    window (`order` "gray" or "paper")."""
    rows = window(F, offset, count) if order == "gray" else paper_order(F, offset, count)
    bits = unpack_rows(rows, F.n)[:, bit_lo:bit_lo + nbits].astype(np.int64)
    vals = bits @ (np.int64(1) << np.arange(nbits, dtype=np.int64))
    return np.bincount(vals, minlength=1 << nbits).astype(np.uint64)
