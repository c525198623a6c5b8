"""The oracle's pins catch plausible mistakes.

Each case copies ac_oracle.c, plants one mistake (a dropped term, a wrong
sign, a wrong index, a transposed operand, a reversed tie-break, swapped
random words, a broken logarithm step, a threshold rounded instead of
floored), compiles the mutant with gcc and runs the pin that should reject it
with the mutant loaded in place of the real oracle.  The mutants live in a temporary directory; the committed
oracle is never modified.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from tests import test_oracle_dynamics as dyn
from tests import test_oracle_exp_ticks as ext
from tests import test_oracle_philox as phx
from tests import test_oracle_thresholds as thr

SRC = os.path.join(os.path.dirname(oracle.__file__), "ac_oracle.c")

MUTANTS = {
    "dropped_field_term": ("double dE = 2.0 * s * (J * S + h);", "double dE = 2.0 * s * (J * S);",
                           lambda: thr.test_detailed_balance_pairs(1.0, 1.0, 0.05)),
    "wrong_sign_in_exp": ("1.0 / (1.0 + exp(beta * dE))", "1.0 / (1.0 + exp(-beta * dE))",
                          lambda: thr.test_detailed_balance_pairs(0.44, 1.0, 0.0)),
    "wrong_table_index": ("thr[up + 5 * (s[c] > 0)]", "thr[up + 5 * (s[c] < 0)]",
                          lambda: dyn.test_transient_law_matches_exp_QT(2, 3, 0.5, 1.0, -0.3, 2.0, 4000)),
    "rows_cols_transposed": ("nb[1] = (uint64_t)(((r + 1) % rows) * cols + q);",
                             "nb[1] = (uint64_t)(((r + 1) % cols) * cols + q);",
                             lambda: dyn.test_heap_equals_linear_scan(3, 2, 3, 0.3, -0.1, 6)),
    "tie_break_reversed": ("(t[a] == t[b] && a < b)", "(t[a] == t[b] && a > b)",
                           dyn.test_forced_tie_is_broken_by_index),
    "gap_and_uniform_swapped": ("if (b[1] < thr[up + 5 * (s[c] > 0)])", "if (b[0] < thr[up + 5 * (s[c] > 0)])",
                                lambda: dyn.test_heap_equals_linear_scan(4, 5, 5, 1.0, 0.05, 4)),
    "philox_words_swapped": ("uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;",
                             "uint32_t n0 = (uint32_t)(p1 >> 32) ^ c3 ^ k0;",
                             lambda: phx.test_philox_matches_triton(7)),
    "threshold_rounded": ("t = (uint32_t)floor(v);", "t = (uint32_t)floor(v + 0.5);",
                          thr.test_table_is_the_floor_of_the_exact_probability),
    "q_threshold_rounded": ("(uint32_t)floor(v) : 0xFFFFFFFFu", "(uint32_t)floor(v + 0.5) : 0xFFFFFFFFu",
                            lambda: thr.test_q_table_is_the_floor_of_the_exact_probability(2)),
    "log_bit_dropped": ("f |= 1ull;", "f |= 0ull;", ext.test_exp_ticks_error_bound_and_positivity),
    "first_gap_from_init_block": ("philox_block(seed, (uint32_t)c, 0u, 0u, b0);\n        if (init == 1)\n            s[c] = 1;\n        else if (init == 2)\n            s[c] = -1;\n        else {\n            philox_block(seed, (uint32_t)c, 0u, 1u, ib);\n            s[c] = (ib[0] & 1u)",
                                  "philox_block(seed, (uint32_t)c, 0u, 1u, b0);\n        if (init == 1)\n            s[c] = 1;\n        else if (init == 2)\n            s[c] = -1;\n        else {\n            philox_block(seed, (uint32_t)c, 0u, 1u, ib);\n            s[c] = (ib[0] & 1u)",
                                  lambda: dyn.test_heap_equals_linear_scan(2, 3, 2, 0.7, 0.2, 6)),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pin_rejects_mutant(name, tmp_path):
    old, new, pin = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique: {old}"
    path = tmp_path / "mut.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-std=gnu99", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                    str(path), "-o", str(so), "-lm"], check=True)
    saved = oracle._load()
    oracle._lib = oracle._bind(ctypes.CDLL(str(so)))
    try:
        with pytest.raises(AssertionError):
            pin()
    finally:
        oracle._lib = saved
