"""The seeded generators: reproducible, symmetric, with the stated shapes."""

import numpy as np

import synth


def test_grid_shapes_and_symmetry():
    for N in (2, 3, 6, 8):
        A = synth.grid_instance(N, 0.5, 3)
        assert A.shape == (N * N, N * N) and A.dtype == np.uint8
        assert np.array_equal(A, A.T)
        off = A.copy()
        off[np.arange(N * N), np.arange(N * N)] = 0
        # only nearest-neighbour edges
        for i, j in zip(*np.nonzero(off)):
            ri, ci, rj, cj = i // N, i % N, j // N, j % N
            assert abs(ri - rj) + abs(ci - cj) == 1


def test_all_connected_edge_count():
    for N in (2, 5, 32):
        A = synth.all_connected(N, "0" * (N * N))
        assert int(A.sum()) == 2 * 2 * N * (N - 1)
        assert len(synth.grid_edges(N)) == 2 * N * (N - 1)


def test_seeded_reproducible():
    a = synth.grid_instance(8, 0.5, 42)
    b = synth.grid_instance(8, 0.5, 42)
    c = synth.grid_instance(8, 0.5, 43)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert synth.window_offset(9, 40, 1 << 20) == synth.window_offset(9, 40, 1 << 20)
    assert 0 <= synth.window_offset(9, 40, 1 << 20) <= (1 << 40) - (1 << 20)
    assert synth.window_offset(1, 64, 5) <= (1 << 64) - 5
    s = synth.sample_indices(5, 1000, 10, 1 << 40)
    assert s.dtype == np.uint64 and s.min() >= 10 and s.max() < (1 << 40)


def test_paper_b_strings():
    assert synth.paper_b_patterns(4) == ["0000", "0001", "0011"]
    assert synth.b_from_string("1011").tolist() == [1, 0, 1, 1]


def test_batch_and_stream_generators():
    insts = synth.batch_instances(16, 4, 16, 0.5, 1)
    assert len(insts) == 16 and all(4 * 4 <= a.shape[0] <= 16 * 16 for a in insts)
    reqs = synth.poisson_stream(20, 100.0, 3, 32, 0.5, 10, 24, 2)
    ts = [r["t_arrival"] for r in reqs]
    assert ts == sorted(ts) and ts[0] == 0.0
    assert all((1 << 10) <= r["want"] <= (1 << 24) for r in reqs)


def test_random_regular_graphs():
    for n, d in ((10, 3), (64, 4), (1024, 3), (500, 8)):
        A = synth.random_regular(n, d, 7)
        off = A.copy()
        off[np.arange(n), np.arange(n)] = 0
        assert np.array_equal(A, A.T)
        assert np.all(off.sum(axis=1) == d)
