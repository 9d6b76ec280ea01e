"""The HLF problem from its definition, for tiny n (<= 12).

Test infrastructure only. Nothing here follows the two-stage method:

* `kernel_bruteforce`, `q_definition`, `solutions_bruteforce`: the problem of
  §1 written out: Ker(A) by trying every x, q(x) = x^T A x mod 4 as an
  integer, and S = every z with q(x) = 2 z^T x (mod 4) for all x in Ker(A).
* `statevector_support`: the quantum circuit of App. A (Eqs. A1-A2) run gate
  by gate on a 2^n state vector; its measurement support is the solution set.
* `mix64`, `chain_hash`: the SplitMix64 finalizer (Steele, Lea and Flood,
  OOPSLA 2014) in Python integers, and its chaining over the words of one
  solution, used to sum hashes over a brute-force solution set.
"""

from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1


def all_vectors(n: int) -> np.ndarray:
    """Every x in {0,1}^n as rows; row t has x_{j+1} = bit j of t."""
    t = np.arange(1 << n, dtype=np.int64)
    return ((t[:, None] >> np.arange(n)[None, :]) & 1).astype(np.uint8)


def kernel_bruteforce(A: np.ndarray) -> np.ndarray:
    """Ker(A) = {x : A x = 0 mod 2}, by trying all 2^n vectors."""
    A = np.asarray(A, dtype=np.int64)
    V = all_vectors(A.shape[0]).astype(np.int64)
    keep = np.all((V @ A.T) % 2 == 0, axis=1)
    return V[keep].astype(np.uint8)


def q_definition(A: np.ndarray, x: np.ndarray) -> int:
    """q(x) = x^T A x mod 4, with integer arithmetic."""
    A = np.asarray(A, dtype=np.int64)
    x = np.asarray(x, dtype=np.int64)
    return int(x @ A @ x) % 4


def solutions_bruteforce(A: np.ndarray) -> np.ndarray:
    """All z in {0,1}^n with q(x) = 2 z^T x (mod 4) for every x in Ker(A)
    (§1), as rows, in increasing order of sum_j z_{j+1} 2^j."""
    A = np.asarray(A, dtype=np.uint8)
    n = A.shape[0]
    K = kernel_bruteforce(A).astype(np.int64)
    qv = np.array([q_definition(A, x) for x in K], dtype=np.int64)
    Z = all_vectors(n).astype(np.int64)
    ok = np.ones(Z.shape[0], dtype=bool)
    for lo in range(0, Z.shape[0], 1024):
        D = Z[lo:lo + 1024] @ K.T
        ok[lo:lo + 1024] = np.all((qv[None, :] - 2 * D) % 4 == 0, axis=1)
    return Z[ok].astype(np.uint8)


def statevector_support(A: np.ndarray):
    """Run App. A's circuit on |0...0>: H on every qubit, CZ on every edge
    (A_ij = 1, i < j), S on every qubit with A_ii = 1, H on every qubit
    (Eqs. A1-A2). Qubit i is bit i of the basis index. Returns (support rows,
    probabilities on the support)."""
    A = np.asarray(A, dtype=np.uint8)
    n = A.shape[0]
    dim = 1 << n
    idx = np.arange(dim, dtype=np.int64)
    psi = np.zeros(dim, dtype=np.complex128)
    psi[0] = 1.0
    s = 1.0 / np.sqrt(2.0)

    def hadamard(v, q):
        v = v.reshape(dim >> (q + 1), 2, 1 << q)
        a0 = v[:, 0, :].copy()
        a1 = v[:, 1, :].copy()
        v[:, 0, :] = s * (a0 + a1)
        v[:, 1, :] = s * (a0 - a1)
        return v.reshape(dim)

    for q in range(n):
        psi = hadamard(psi, q)
    for i in range(n):
        for j in range(i + 1, n):
            if A[i, j]:
                both = ((idx >> i) & 1) & ((idx >> j) & 1)
                psi = np.where(both == 1, -psi, psi)
    for i in range(n):
        if A[i, i]:
            psi = np.where(((idx >> i) & 1) == 1, 1j * psi, psi)
    for q in range(n):
        psi = hadamard(psi, q)
    prob = np.abs(psi) ** 2
    sup = np.nonzero(prob > 1e-9)[0]
    rows = ((sup[:, None] >> np.arange(n)[None, :]) & 1).astype(np.uint8)
    return rows, prob[sup]


def mix64(x: int) -> int:
    """SplitMix64 finalizer on a 64-bit integer."""
    x &= MASK64
    x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & MASK64
    return x ^ (x >> 31)


def splitmix64_stream(seed: int, count: int) -> list[int]:
    """The SplitMix64 generator: state += 0x9E3779B97F4A7C15, output
    mix64(state)."""
    out, s = [], seed & MASK64
    for _ in range(count):
        s = (s + 0x9E3779B97F4A7C15) & MASK64
        out.append(mix64(s))
    return out


def chain_hash(words) -> int:
    """Hash of one solution stored as words w_0..w_{W-1}: h = mix64(w_0),
    then h = mix64(h ^ w_j)."""
    words = [int(w) for w in words]
    h = mix64(words[0])
    for w in words[1:]:
        h = mix64(h ^ w)
    return h


def bits_to_words(rows: np.ndarray) -> list[tuple[int, ...]]:
    """0/1 rows to tuples of 64-bit words (bit j -> word j // 64, bit j % 64),
    with Python integers, independent of numpy packing."""
    rows = np.asarray(rows, dtype=np.uint8)
    n = rows.shape[1]
    W = (n + 63) // 64
    out = []
    for row in rows:
        ws = [0] * W
        for j in range(n):
            if row[j]:
                ws[j // 64] |= 1 << (j % 64)
        out.append(tuple(ws))
    return out


def string_of(row) -> str:
    """A solution as the paper writes it: z_1 z_2 ... z_n left to right."""
    return "".join("1" if v else "0" for v in row)
