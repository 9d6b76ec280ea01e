"""The pins have teeth: plant one plausible mistake at a time in a copy of
the C oracle (a dropped term, a wrong shift, a transposed operand, a wrong
index, OR for XOR) and check that at least one pin of
tests/test_oracle_pins.py then fails. The mistakes live only in temporary
copies built here on the CPU."""

import os
import subprocess

import pytest

from oracle import cpu as oc
from oracle.build import SRC
from tests import test_oracle_pins as pins
from tests.conftest import read_golden

MUTANTS = {
    "q_drops_diagonal": ("s += (long long)A[(size_t)a * n + b] * x[b];",
                         "if (a != b) s += (long long)A[(size_t)a * n + b] * x[b];"),
    "gray_code_wrong_shift": ("uint64_t g = i ^ (i >> 1);", "uint64_t g = i ^ (i >> 2);"),
    "mix_wrong_shift": ("x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;",
                        "x = (x ^ (x >> 26)) * 0x94D049BB133111EBULL;"),
    "kernel_transposed": ("for (int k = 0; k < r; ++k) x[piv[k]] = R[(size_t)k * n + f];",
                          "for (int k = 0; k < r; ++k) x[piv[k]] = R[(size_t)f * n + k];"),
    "za_not_canonical": ("for (int k = 0; k < r; ++k) M[(size_t)(nf + k) * (n + 1) + piv[k]] = 1;",
                         "for (int k = 1; k < r; ++k) M[(size_t)(nf + k) * (n + 1) + piv[k]] = 1;"),
    "gray_step_wrong_index": ("int k = ctz64(i);", "int k = ctz64(i) + (i > 8 ? 1 : 0);"),
    "fold_or_not_xor": ("t->fold[w] ^= z[w];", "t->fold[w] |= z[w];"),
    "paper_counter_bit": ("R[piv[j - 1]] = r - j < 64 ? (uint8_t)((t >> (r - j)) & 1) : 0;",
                          "R[piv[j - 1]] = r - j < 64 ? (uint8_t)((t >> (j - 1 + (j == r))) & 1) : 0;"),
    "paper_counter_reversed": ("R[piv[j - 1]] = r - j < 64 ? (uint8_t)((t >> (r - j)) & 1) : 0;",
                               "R[piv[j - 1]] = j - 1 < 64 ? (uint8_t)((t >> (j - 1)) & 1) : 0;"),
    "rref_skips_rows_above": ("if (i == rank || !M[(size_t)i * cols + c]) continue;",
                              "if (i <= rank || !M[(size_t)i * cols + c]) continue;"),
}


def _pins_hold() -> bool:
    checks = [
        *(lambda row=row: pins.test_paper_2x2_solution_lists(row)
          for row in read_golden("paper_2x2_solutions.txt")),
        *(lambda row=row: pins.test_paper_ranks_and_counts(row)
          for row in read_golden("paper_grid_ranks.txt")[:6]),
        *(lambda c=c: pins.test_factor_against_bruteforce(*c) for c in pins.TINY[::4]),
        lambda: pins.test_window_direct_equals_gray_stepping(0),
        lambda: pins.test_window_validity_and_index_recovery(0),
        lambda: pins.test_mix64_published_vectors(),
        *(lambda c=c: pins.test_reduce_against_bruteforce_set(*c) for c in pins.TINY[::6]),
        lambda: pins.test_reduce_xor_fold_closed_forms(0),
        *(lambda c=c: pins.test_paper_order_same_set(*c) for c in pins.TINY[:18:3]),
        *(lambda c=c: pins.test_paper_order_counter_recovered(*c) for c in pins.TINY[:18:3]),
    ]
    for chk in checks:
        try:
            chk()
        except (AssertionError, oc.OracleError):
            return False
    return True


def test_unmutated_oracle_passes_the_pins():
    assert _pins_hold()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path, monkeypatch):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site of {name} not found"
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", str(lib),
                    str(mutated)], check=True)
    monkeypatch.setattr(oc, "_LIB", oc.bind(str(lib)))
    assert not _pins_hold(), f"mutant {name} passed every pin"
    assert os.path.exists(lib)
