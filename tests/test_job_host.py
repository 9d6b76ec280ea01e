"""The resumable reduce job on the CPU, with the oracle as its reduce: a job
stopped after any number of chunks, written to a JSON checkpoint, read back
(as after a restart) and finished, ends with exactly the reduce of the whole
window; checkpoints that do not match their rows or window are refused."""

import json

import numpy as np
import pytest

import synth
from oracle import cpu as oc
from paper_2103_00693_gb300.job import ReduceJob


@pytest.mark.parametrize("N,p,seed,off,cnt,chunk", [(6, 0.5, 3, 100, 300001, 40000), (9, 0.5, 8, 7, 99999, 8191),
                                                     (4, 1.0, 1, 0, 4096, 1000)])
def test_job_resumes_exactly(N, p, seed, off, cnt, chunk):
    A = synth.grid_instance(N, p, seed)
    F = oc.factor(A)
    cnt = min(cnt, (1 << F.space_log2()) - off)
    want = oc.reduce(F, off, cnt, 1)
    for stop in (0, 1, 3):
        job = ReduceJob.start(A, off, cnt, chunk)
        job.advance(lambda o, c: oc.reduce(F, o, c, 1), stop)
        text = job.to_json()
        resumed = ReduceJob.from_json(text)
        assert resumed.next == job.next and not resumed.done() or stop * chunk >= cnt
        while not resumed.done():
            resumed.advance(lambda o, c: oc.reduce(F, o, c, 1), 2)
        c, h, f = resumed.result()
        assert (c, h) == want[:2] and np.array_equal(f, want[2])


def test_job_refuses_bad_checkpoints():
    A = synth.grid_instance(5, 0.5, 2)
    F = oc.factor(A)
    job = ReduceJob.start(A, 0, 5000, 1000)
    job.advance(lambda o, c: oc.reduce(F, o, c, 1), 2)
    d = json.loads(job.to_json())
    bad = dict(d, rows=list(d["rows"]))
    bad["rows"][0] = format(int(bad["rows"][0], 16) ^ 1, "016x")
    with pytest.raises(ValueError):
        ReduceJob.from_json(json.dumps(bad))
    with pytest.raises(ValueError):
        ReduceJob.from_json(json.dumps(dict(d, next=6000)))
    with pytest.raises(ValueError):
        ReduceJob.from_json(json.dumps(dict(d, partial=dict(d["partial"], count=1))))
    with pytest.raises(RuntimeError):
        job.result()
