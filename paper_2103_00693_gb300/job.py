"""Resumable reduce of one instance's index window.

Enumeration is stateless given (factorisation, offset): any window seeds on
its own. A long reduce of [offset, offset + count) therefore checkpoints as
(the matrix, the window, the next index, the partial (count, hash sum,
XOR-fold) of [offset, next)); the partials of disjoint windows combine by +,
+ (mod 2^64) and XOR, so a job stopped at any chunk boundary and resumed in
another process, after a restart, or on another GPU, ends with exactly the
reduce of the whole window. The matrix is kept in the checkpoint as packed
rows with a digest, so a resumed job refuses a checkpoint that does not match
its own rows. The factorisation is recomputed on resume (stage 1 takes
microseconds); the reduce itself runs in the library's kernels.
"""

from __future__ import annotations

import hashlib
import json
from dataclasses import dataclass, field

import numpy as np

from . import hlf
from .shard import combine_reduce


def _digest(words: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(words, dtype=np.uint64).tobytes()).hexdigest()[:32]


@dataclass
class ReduceJob:
    """State of a chunked reduce of [offset, offset + count)."""

    n: int
    rows: np.ndarray  # packed uint64 [n][W]
    offset: int
    count: int
    chunk: int
    next: int = 0  # first index not yet reduced
    part: tuple = field(default=None)  # (count, hsum, xor_fold[W]) of [offset, next)

    @classmethod
    def start(cls, A: np.ndarray, offset: int, count: int, chunk: int = 1 << 30) -> "ReduceJob":
        if chunk < 1 or count < 0 or offset < 0:
            raise ValueError("chunk >= 1, count >= 0 and offset >= 0 are required")
        rows = hlf.pack_rows(A)
        W = rows.shape[1]
        return cls(n=A.shape[0], rows=rows, offset=offset, count=count, chunk=chunk, next=offset,
                   part=(0, 0, np.zeros(W, dtype=np.uint64)))

    @property
    def W(self) -> int:
        return self.rows.shape[1]

    def done(self) -> bool:
        return self.next >= self.offset + self.count

    def advance(self, reduce_fn, max_chunks: int = 1) -> int:
        """Reduce up to max_chunks further chunks with reduce_fn(o, c) ->
        (count, hsum, fold) and fold them into the partial; returns the
        number of chunks reduced."""
        k = 0
        end = self.offset + self.count
        while k < max_chunks and self.next < end:
            c = min(self.chunk, end - self.next)
            self.part = combine_reduce([self.part, reduce_fn(self.next, c)])
            self.next += c
            k += 1
        return k

    def result(self) -> tuple[int, int, np.ndarray]:
        if not self.done():
            raise RuntimeError("the job has not reached the end of its window")
        return self.part

    # ------------------------------------------------------------ checkpoint

    def to_json(self) -> str:
        c, h, f = self.part
        return json.dumps({
            "version": 1, "n": self.n, "rows": [format(int(x), "016x") for x in self.rows.ravel()],
            "rows_digest": _digest(self.rows), "offset": self.offset, "count": self.count,
            "chunk": self.chunk, "next": self.next,
            "partial": {"count": int(c), "hsum": int(h), "xor_fold": [format(int(x), "016x") for x in f]},
        })

    @classmethod
    def from_json(cls, text: str) -> "ReduceJob":
        d = json.loads(text)
        if d.get("version") != 1:
            raise ValueError("unknown checkpoint version")
        n = int(d["n"])
        W = hlf.words(n)
        rows = np.array([int(x, 16) for x in d["rows"]], dtype=np.uint64).reshape(n, W)
        if _digest(rows) != d["rows_digest"]:
            raise ValueError("checkpoint rows do not match their digest")
        offset, count, nxt = int(d["offset"]), int(d["count"]), int(d["next"])
        if not offset <= nxt <= offset + count:
            raise ValueError("checkpoint's next index lies outside its window")
        p = d["partial"]
        fold = np.array([int(x, 16) for x in p["xor_fold"]], dtype=np.uint64)
        if len(fold) != W or int(p["count"]) != nxt - offset:
            raise ValueError("checkpoint's partial does not match its window")
        return cls(n=n, rows=rows, offset=offset, count=count, chunk=int(d["chunk"]), next=nxt,
                   part=(int(p["count"]), int(p["hsum"]), fold))


def gpu_reduce_fn(job: ReduceJob, stream=None):
    """Factor the job's matrix on the current GPU and return (reduce_fn,
    close): reduce_fn(o, c) runs hlf_enumerate_reduce over [o, o + c) and
    returns its (count, hsum, fold); close() frees the factorisation."""
    import torch

    A_dev = torch.from_numpy(job.rows.view(np.int64)).cuda()
    G = hlf.Factorization(A_dev, job.n, stream)
    red = torch.empty(hlf.REDUCE_WORDS, dtype=torch.int64, device="cuda")

    def reduce_fn(o: int, c: int, _rows=A_dev):  # keeps the matrix alive while the factor kernel may read it
        G.reduce(o, c, red, stream)
        r = hlf.ReduceResult.from_words(red.cpu().numpy(), job.W)
        return r.count, r.hsum, r.xor_fold

    return reduce_fn, G.close
