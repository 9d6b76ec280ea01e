"""CPU oracle for the two-stage FS2D HLF scheme of arXiv 2103.00693.

TEST INFRASTRUCTURE. Only `tests/`, `__graft_entry__.smoke()` and the
`cpu_baseline` / `--impl reference` legs of `bench.py` may import, call or
link anything in this package. The CUDA path never does, and the two share no
code: only the seeded generators in `synth/` serve both.

Contents and what pins each part (tests in tests/test_oracle_*.py):

* `definitional` -- the problem from its definition (§1), for n <= 12, and
  App. A's quantum circuit as a state vector (Eqs. A1-A2). Pinned by the
  paper's printed 2x2 solution lists (§4, Fig. 3(a)-(c)) and by each other.
* `cpu.factor` -- CLA steps (1)-(4) of §2 (Fig. 1(b)): RREF, pivots, rank,
  kernel basis, q mod 4, z^a. Pinned by brute force (n <= 12), the paper's
  ranks and solution counts for 2x2..5x5 grids (§4, App. C), App. B's rank
  r = n - N for all-connected grids with b = 0 and n - N <= r <= n for any b,
  and r = n => every string is a solution and z^a = 0.
* `cpu.window`, `cpu.window_gray` -- solution z(i) of index i (§2 Eqs. 1-3
  with the Gray-order reading): the two routes agree, every z is valid by the
  definition, index i is recovered as the inverse Gray code of z on P, and
  the full index space is exactly the brute-force set.
* `cpu.reduce` -- (count, hash sum, XOR-fold): count = 2^r; the fold matches
  its closed forms (0 for r >= 2 and for aligned blocks of >= 4, B_1 for
  r = 1, z^a for r = 0); the hash sum equals the sum over the brute-force set
  in any order; the hash itself reproduces SplitMix64's published outputs.
* `cpu.paper_order` -- §2's own order (binary counter, y = A R): same set as
  the brute force and as the Gray-order windows.

Every function here has a pin; none is "parity unpinned".
"""
