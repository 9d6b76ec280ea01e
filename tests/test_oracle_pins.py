"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints, closed forms, brute force on tiny inputs, App. A's quantum
circuit, or the published SplitMix64 outputs.
"""

import numpy as np
import pytest

import synth
from oracle import cpu as oc
from oracle import definitional as od
from tests.conftest import expand_b, read_golden


def as_strings(rows):
    return sorted(od.string_of(r) for r in rows)


def full_set(F):
    """Every solution the oracle enumerates, as 0/1 rows."""
    return oc.unpack_rows(oc.window(F, 0, 1 << F.r), F.n)


# ---------------------------------------------------------------- paper values

@pytest.mark.parametrize("row", read_golden("paper_2x2_solutions.txt"), ids=lambda r: r[0])
def test_paper_2x2_solution_lists(row):
    """§4, Fig. 3(a)-(c): the printed solution lists of the 2x2 grid."""
    b, r = row[0], int(row[1])
    want = [f"{t:04b}" for t in range(16)] if row[2] == "ALL" else row[2:]
    A = synth.all_connected(2, b)
    F = oc.factor(A)
    assert F.r == r
    assert as_strings(full_set(F)) == sorted(want)
    assert as_strings(od.solutions_bruteforce(A)) == sorted(want)


@pytest.mark.parametrize("row", read_golden("paper_grid_ranks.txt"), ids=lambda r: f"{r[0]}-{r[1]}")
def test_paper_ranks_and_counts(row):
    """§4 Fig. 3 and App. C Figs. 6-7: ranks and solution counts."""
    N, b, r, k = int(row[0]), expand_b(row[1]), int(row[2]), int(row[3])
    F = oc.factor(synth.all_connected(N, b))
    assert F.r == r and (1 << F.r) == k
    if N <= 3:
        assert len(od.solutions_bruteforce(synth.all_connected(N, b))) == k


# ------------------------------------------------------------ App. B closed form

@pytest.mark.parametrize("N", list(range(2, 17)))
def test_appB_rank_all_connected_b0(N):
    """App. B: an all-connected N x N grid with b = 0 has rank exactly n - N."""
    F = oc.factor(synth.all_connected(N, "0" * (N * N)))
    assert F.r == N * N - N


@pytest.mark.parametrize("seed", range(12))
def test_appB_rank_bounds_any_b(seed):
    """App. B: for any diagonal, n - N <= r <= n on all-connected grids."""
    N = 2 + seed % 9
    A = synth.grid_instance(N, 1.0, seed)
    F = oc.factor(A)
    assert N * N - N <= F.r <= N * N


# -------------------------------------------------------------- brute force

def _tiny_cases():
    cases = []
    for seed in range(10):
        cases.append(("grid3", synth.grid_instance(3, 0.5, seed)))
    for seed in range(4):
        cases.append(("grid2", synth.grid_instance(2, 0.5, 100 + seed)))
    for n in range(1, 11):
        for d in (0.2, 0.5, 0.8):
            cases.append((f"sym{n}-{d}", synth.random_symmetric(n, d, 1000 * n + int(10 * d))))
    cases.append(("zero5", np.zeros((5, 5), dtype=np.uint8)))
    cases.append(("eye6", np.eye(6, dtype=np.uint8)))
    return cases


TINY = _tiny_cases()


@pytest.mark.parametrize("name,A", TINY, ids=[c[0] for c in TINY])
def test_factor_against_bruteforce(name, A):
    """The oracle's stage 1 + full enumeration equal the definition of §1."""
    F = oc.factor(A)
    S = od.solutions_bruteforce(A)
    K = od.kernel_bruteforce(A)
    n = A.shape[0]
    # |Ker(A)| = 2^(n-r) and |S| = 2^r (§2)
    assert len(K) == 1 << (n - F.r)
    assert len(S) == 1 << F.r
    # the oracle's kernel basis spans Ker(A), q(x_f) matches the definition
    for x, f, q in zip(F.X, F.free, F.q):
        assert not np.any((A.astype(int) @ x) % 2)
        assert x[f] == 1
        assert q == od.q_definition(A, x)
    # z^a is the unique solution that vanishes on P
    cands = [z for z in S if not np.any(z[F.piv])]
    assert len(cands) == 1 and np.array_equal(cands[0], F.z0)
    # the enumerated set is the solution set
    assert as_strings(full_set(F)) == as_strings(S)


@pytest.mark.parametrize("name,A", TINY[:20], ids=[c[0] for c in TINY[:20]])
def test_appA_statevector_support(name, A):
    """App. A (Eqs. A1-A2): the measurement support of the graph-state
    circuit is the solution set, with uniform probability 2^-r."""
    F = oc.factor(A)
    sup, prob = od.statevector_support(A)
    assert as_strings(sup) == as_strings(full_set(F))
    assert np.allclose(prob, 2.0 ** -F.r, rtol=1e-9, atol=0)


def test_full_rank_every_string():
    """§3: r = n means every n-bit string is a solution, and z^a = 0."""
    for A in (np.eye(7, dtype=np.uint8), synth.all_connected(2, "1111")):
        F = oc.factor(A)
        n = A.shape[0]
        assert F.r == n and not F.z0.any()
        assert len(set(as_strings(full_set(F)))) == 1 << n


def test_zero_matrix_single_solution():
    """A = 0: Ker(A) is everything, q = 0, the only solution is z = 0."""
    F = oc.factor(np.zeros((9, 9), dtype=np.uint8))
    assert F.r == 0 and not F.z0.any()
    assert oc.window(F, 0, 1).tolist() == [[0]]


def test_non_symmetric_rejected():
    A = synth.all_connected(3, "0" * 9)
    A[0, 4] = 1
    with pytest.raises(oc.OracleError):
        oc.factor(A)


# ------------------------------------------------------------- window routes

@pytest.mark.parametrize("seed", range(6))
def test_window_direct_equals_gray_stepping(seed):
    A = synth.grid_instance(8, 0.5, seed)
    F = oc.factor(A)
    space = 1 << F.space_log2()
    for off, cnt in ((0, 300), (space - 257, 257), (12345 % space, 1000)):
        cnt = min(cnt, space - off)
        assert np.array_equal(oc.window(F, off, cnt), oc.window_gray(F, off, cnt))


def _gray_inverse(g: int) -> int:
    i = 0
    while g:
        i ^= g
        g >>= 1
    return i


@pytest.mark.parametrize("seed", range(4))
def test_window_validity_and_index_recovery(seed):
    """Every z(i) satisfies z . x_f = q(x_f)/2 on the kernel basis, and the
    inverse Gray code of z restricted to P recovers i (so z(i) are distinct)."""
    A = synth.grid_instance(6, 0.5, 50 + seed)
    F = oc.factor(A)
    off = (7919 * (seed + 1)) % (1 << F.r)
    cnt = min(2048, (1 << F.r) - off)
    Z = oc.unpack_rows(oc.window(F, off, cnt), F.n).astype(np.int64)
    par = (Z @ F.X.T.astype(np.int64)) % 2
    assert np.array_equal(par, np.broadcast_to(F.q // 2, par.shape))
    for t, z in enumerate(Z):
        g = sum(int(z[p]) << k for k, p in enumerate(F.piv))
        assert _gray_inverse(g) == off + t


def test_window_range_checks():
    F = oc.factor(synth.all_connected(2, "0000"))  # r = 2
    oc.window(F, 0, 4)
    oc.window(F, 4, 0)
    with pytest.raises(oc.OracleError):
        oc.window(F, 1, 4)
    with pytest.raises(oc.OracleError):
        oc.reduce(F, 5, 0)


# ------------------------------------------------------------------- reduce


def test_mix64_published_vectors():
    """SplitMix64's published outputs (Steele, Lea and Flood 2014) pin the
    finalizer in both the Python and the C oracle."""
    rows = read_golden("splitmix64_vectors.txt")
    by_seed = {}
    for seed, idx, hx in rows:
        by_seed.setdefault(int(seed), {})[int(idx)] = int(hx, 16)
    gamma = 0x9E3779B97F4A7C15
    for seed, outs in by_seed.items():
        stream = od.splitmix64_stream(seed, max(outs) + 1)
        for idx, want in outs.items():
            assert stream[idx] == want
            state = (seed + (idx + 1) * gamma) % (1 << 64)
            assert oc.mix64(state) == want


@pytest.mark.parametrize("name,A", TINY[::3], ids=[c[0] for c in TINY[::3]])
def test_reduce_against_bruteforce_set(name, A):
    """Count, hash sum and XOR-fold of the full Gray-order enumeration equal
    the same quantities over the brute-force solution set taken in another
    order (sum and XOR do not depend on order)."""
    F = oc.factor(A)
    S = od.solutions_bruteforce(A)
    words = od.bits_to_words(S)
    hs = sum(od.chain_hash(w) for w in words) % (1 << 64)
    fold = [0] * F.W
    for w in words:
        for j in range(F.W):
            fold[j] ^= w[j]
    for threads in (1, 3):
        c, h, f = oc.reduce(F, 0, 1 << F.r, threads)
        assert c == len(S) and h == hs and [int(x) for x in f] == fold


@pytest.mark.parametrize("seed", range(5))
def test_reduce_xor_fold_closed_forms(seed):
    """XOR over an affine space of dimension >= 2 is 0; over a dimension-1
    space {z^a, z^a ^ B_1} it is B_1; over the single point z^a it is z^a."""
    A = synth.grid_instance(5, 0.5, 300 + seed)
    F = oc.factor(A)
    _, _, fold = oc.reduce(F, 0, 1 << F.r)
    assert not fold.any()
    # aligned blocks of 2^k, k >= 2, are affine subspaces of dimension k
    for k in (2, 5):
        blk = 1 << k
        start = (seed * 977 * blk) % (1 << F.r)
        start -= start % blk
        _, _, f = oc.reduce(F, start, blk)
        assert not f.any()
    # r = 1 and r = 0
    A1 = np.zeros((4, 4), dtype=np.uint8)
    A1[2, 2] = 1
    F1 = oc.factor(A1)
    assert F1.r == 1
    _, _, f1 = oc.reduce(F1, 0, 2)
    assert np.array_equal(f1, F1.basis_words()[0])
    F0 = oc.factor(np.zeros((3, 3), dtype=np.uint8))
    c0, h0, f0 = oc.reduce(F0, 0, 1)
    assert c0 == 1 and np.array_equal(f0, F0.z0_words()) and h0 == od.mix64(0)


def test_reduce_parts_combine():
    """A window's reduce is the +/+/XOR combination of its sub-windows."""
    F = oc.factor(synth.grid_instance(6, 0.5, 7))
    off, cnt = 1000, 50000
    c, h, f = oc.reduce(F, off, cnt)
    cuts = [off, off + 1, off + 777, off + 30000, off + cnt]
    C, H, Fx = 0, 0, np.zeros_like(f)
    for a, b in zip(cuts, cuts[1:]):
        ci, hi, fi = oc.reduce(F, a, b - a, 2)
        C, H, Fx = C + ci, (H + hi) % (1 << 64), Fx ^ fi
    assert (C, H) == (c, h) and np.array_equal(Fx, f)


# -------------------------------------------------------------- paper order

@pytest.mark.parametrize("name,A", TINY[:18], ids=[c[0] for c in TINY[:18]])
def test_paper_order_same_set(name, A):
    """§2 Eq. 3 with the counter of §4 (R over {0,1}^r on the pivots,
    z = A R ^ z^a) yields the same set as the Gray-order enumeration."""
    F = oc.factor(A)
    P = oc.unpack_rows(oc.paper_order(F, 0, 1 << F.r), F.n)
    assert as_strings(P) == as_strings(full_set(F))
    assert len(set(as_strings(P))) == 1 << F.r


def test_large_n_factor_consistency():
    """n = 1024 (32 x 32 grid): the kernel basis annihilates A, q is even,
    and z^a satisfies every kernel equation."""
    A = synth.grid_instance(32, 0.5, 11)
    F = oc.factor(A)
    assert 0 < F.r <= 1024
    Ai = A.astype(np.int64)
    X = F.X.astype(np.int64)
    assert not np.any((X @ Ai) % 2)
    assert np.all(F.q % 2 == 0)
    assert np.array_equal((X @ F.z0.astype(np.int64)) % 2, F.q // 2)
    assert not F.z0[F.piv].any()


def _leftmost_independent_columns(A: np.ndarray) -> list[int]:
    """P = L_ind of §2, by its definition: scan the columns left to right and
    keep each one that is not in the span of those kept (spans held as sets
    of Python-int bit masks; independent of the oracle's elimination)."""
    n = A.shape[0]
    basis: dict[int, int] = {}  # leading bit -> reduced vector
    keep = []
    for c in range(n):
        v = int("".join(str(int(b)) for b in A[::-1, c]), 2)
        while v:
            top = v.bit_length() - 1
            if top not in basis:
                basis[top] = v
                keep.append(c)
                break
            v ^= basis[top]
    return keep


def _counter_of(R_P: np.ndarray) -> int:
    """The §4 counter value of R^(r) = R_{p_1} .. R_{p_r} read as a binary
    numeral with R_{p_1} most significant."""
    r = len(R_P)
    return sum(int(R_P[j - 1]) << (r - j) for j in range(1, r + 1))


@pytest.mark.parametrize("name,A", [c for c in TINY if 0 < c[1].shape[0] <= 10][:24],
                         ids=[c[0] for c in TINY if 0 < c[1].shape[0] <= 10][:24])
def test_paper_order_counter_recovered(name, A):
    """§2 Eq. 3 with the counter of §4: every solution the paper-order
    enumeration emits at counter t gives t back. From z alone: z^a is the
    brute-force solution that vanishes on P, and R_P is the one choice among
    all 2^r with (A R)|_P = (z ^ z^a)|_P (A[P,P] is nonsingular), found by
    trying every choice; t is then R^(r) read most significant first."""
    F = oc.factor(A)
    P = _leftmost_independent_columns(A)
    r = len(P)
    assert r == F.r
    S = od.solutions_bruteforce(A)
    za = [z for z in S if not np.any(z[P])]
    assert len(za) == 1
    za = za[0].astype(np.int64)
    # all 2^r choices of R_P and the pivot rows of A R they give
    choices = od.all_vectors(r).astype(np.int64)  # [2^r][r]
    App = A[np.ix_(P, P)].astype(np.int64)
    images = (choices @ App.T) % 2
    key = {tuple(y): R for y, R in zip(images.tolist(), choices)}
    assert len(key) == 1 << r  # A[P,P] nonsingular: the choice is unique
    Z = oc.unpack_rows(oc.paper_order(F, 0, 1 << r), F.n).astype(np.int64)
    for t, z in enumerate(Z):
        R_P = key[tuple(((z ^ za)[P]).tolist())]
        assert _counter_of(R_P) == t, (t, R_P)


def _gf2_solve(M: np.ndarray, rhs: np.ndarray) -> np.ndarray:
    """x with M x = rhs over GF(2) for a square nonsingular 0/1 matrix M,
    by elimination on Python-int row masks (written here, independent of the
    oracle's byte-per-bit elimination)."""
    m = M.shape[0]
    rows = [(int("".join(str(int(b)) for b in M[i, ::-1]), 2), int(rhs[i])) for i in range(m)]
    for c in range(m):
        p = next(i for i in range(c, m) if (rows[i][0] >> c) & 1)
        rows[c], rows[p] = rows[p], rows[c]
        for i in range(m):
            if i != c and (rows[i][0] >> c) & 1:
                rows[i] = (rows[i][0] ^ rows[c][0], rows[i][1] ^ rows[c][1])
    return np.array([rows[i][1] for i in range(m)], dtype=np.int64)


def test_paper_order_beyond_64_pivots():
    """r > 64: the paper order's 64-bit counter reaches the first 2^64 values.
    Each emitted z is a valid solution, the z are distinct, and the counter is
    recovered from z: R_P solves A[P,P] R_P = (z ^ z^a)|_P (solved here by a
    separate GF(2) elimination), the leading r - 64 entries are 0, and the
    rest read as a binary numeral (R_{p_1} most significant) give t."""
    A = synth.grid_instance(20, 0.5, 1234)
    F = oc.factor(A)
    assert F.r > 64
    P = _leftmost_independent_columns(A)
    assert P == [int(p) for p in F.piv[:F.r]]
    App = A[np.ix_(P, P)]
    za = F.z0.astype(np.int64)
    top = 1 << 64
    for t0, cnt in ((0, 300), (top - 300, 300), ((1 << 63) - 5, 10)):
        Z = oc.unpack_rows(oc.paper_order(F, t0, cnt), F.n).astype(np.int64)
        par = (Z @ F.X.T.astype(np.int64)) % 2
        assert np.array_equal(par, np.broadcast_to(F.q // 2, par.shape))
        assert len({tuple(z) for z in Z}) == cnt
        for k in range(0, cnt, 7):
            R_P = _gf2_solve(App, (Z[k] ^ za)[P])
            assert not R_P[:F.r - 64].any()
            assert _counter_of(R_P) == t0 + k


def test_dense_stream_layout():
    """The dense layout, checked bit by bit from its definition."""
    rng = np.random.default_rng(2)
    for count, n in ((1, 1), (3, 9), (64, 36), (65, 36), (7, 64), (5, 65), (9, 130)):
        rows = (rng.random((count, n)) < 0.5).astype(np.uint8)
        s = oc.dense_stream(rows)
        assert len(s) == (count * n + 63) // 64
        for t in range(count):
            for j in range(n):
                b = t * n + j
                assert (int(s[b // 64]) >> (b % 64)) & 1 == rows[t, j]
        tail = count * n
        if tail % 64:
            assert int(s[-1]) >> (tail % 64) == 0


def _gf2_rank(rows: np.ndarray) -> int:
    """Rank over GF(2) of 0/1 rows, by brute force over subsets for tiny
    inputs (independent of the oracle's elimination)."""
    rows = [int("".join(map(str, r[::-1])), 2) for r in rows]
    span = {0}
    for v in rows:
        span |= {s ^ v for s in span}
    return len(span).bit_length() - 1


@pytest.mark.parametrize("seed", range(6))
def test_histogram_closed_form(seed):
    """Over the full solution set (an affine space of dimension r), the
    values of any bit field form an affine space of dimension d = rank of
    the basis restricted to those bits, each value hit exactly 2^(r-d)
    times (Sec. 2: the solutions are z^a + Col(A))."""
    A = synth.grid_instance(4, 0.5, 900 + seed)
    F = oc.factor(A)
    for lo, nb in ((0, 4), (3, 5), (F.n - 6, 6), (0, F.n)):
        h = oc.histogram(F, 0, 1 << F.r, lo, nb)
        d = _gf2_rank(F.basis[:, lo:lo + nb])
        nz = h[h > 0]
        assert len(nz) == 1 << d and np.all(nz == (1 << (F.r - d)))
        z0v = int(sum(int(F.z0[lo + j]) << j for j in range(nb)))
        assert h[z0v] > 0
    # paper order gives the same histogram over the full set
    assert np.array_equal(oc.histogram(F, 0, 1 << F.r, 2, 7), oc.histogram(F, 0, 1 << F.r, 2, 7, "paper"))
