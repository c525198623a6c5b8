"""Pins of the oracle's asynchronous Life-like automaton (reading R12).

Deterministic outer-totalistic rules on the 8-cell Moore neighbourhood under the
same Poisson asynchrony as the Ising array (Sec. 3 uses Conway's Game of Life as
the example of a deterministic rule).  Pinned against a brute-force linear-scan
simulator, against the rule on hand-built neighbourhoods, against still lifes, and
against the fact that arrival times do not depend on the states.
"""
import numpy as np
import pytest

import oracle
from tests.test_oracle_dynamics import _spec_init

T32 = 1 << 32
B3, S23 = oracle.CONWAY_BIRTH, oracle.CONWAY_SURVIVE


def _brute_life(s, t, n, rows, cols, birth, survive, seed, t_end):
    s, t, n = s.copy(), t.copy(), n.copy().astype(np.int64)
    N = rows * cols
    idx = np.arange(N)
    while True:
        tmin = t.min()
        if tmin >= t_end:
            break
        c = int(idx[t == tmin].min())
        r, q = divmod(c, cols)
        k = sum(1 for dr in (-1, 0, 1) for dq in (-1, 0, 1) if (dr or dq)
                and s[((r + dr) % rows) * cols + (q + dq) % cols] > 0)
        mask = survive if s[c] > 0 else birth
        s[c] = 1 if (mask >> k) & 1 else -1
        b = oracle.philox_blocks(seed, [c], [n[c] + 1], 0)[0]
        t[c] += oracle.exp_ticks(int(b[0]))
        n[c] += 1
    return s, t, n.astype(np.uint32)


@pytest.mark.parametrize("rows,cols,seed,density,rule", [
    (3, 3, 1, 1 << 31, (B3, S23)), (4, 5, 2, 1 << 31, (B3, S23)), (7, 6, 3, 3 << 30, (B3, S23)),
    (8, 8, 4, 1 << 30, ((1 << 3) | (1 << 6), S23)),                 # HighLife B36/S23
    (5, 9, 5, 1 << 31, (1 << 2, 0)),                                  # B2/S (seeds)
    (6, 4, 6, 1 << 31, (0x1FF, 0x1FF)),                               # every count gives life
])
def test_life_equals_brute_force(rows, cols, seed, density, rule):
    birth, survive = rule
    st = oracle.life_init(rows, cols, 0, density, seed)
    s0, t0, n0 = st.s.copy(), st.t.copy(), st.n.copy()
    oracle.life_run(st, birth, survive, seed, 6 * T32)
    s, t, n = _brute_life(s0, t0, n0, rows, cols, birth, survive, seed, 6 * T32)
    assert np.array_equal(st.s, s) and np.array_equal(st.t, t) and np.array_equal(st.n, n)


def test_rule_on_hand_built_neighbourhoods():
    """Cell (2, 2) of a 5x5 torus with exactly k live Moore neighbours, made to arrive first."""
    ring = [(1, 1), (1, 2), (1, 3), (2, 1), (2, 3), (3, 1), (3, 2), (3, 3)]
    seed = 9
    for alive in (False, True):
        for k in range(9):
            st = oracle.life_init(5, 5, 2, 0, seed)                 # all dead
            for (r, q) in ring[:k]:
                st.s[r * 5 + q] = 1
            c = 2 * 5 + 2
            st.s[c] = 1 if alive else -1
            st.t[:] = 10 * T32
            st.t[c] = 5
            oracle.life_run(st, B3, S23, seed, 6)                   # exactly one arrival
            expect = (k in (2, 3)) if alive else (k == 3)
            assert (st.s[c] > 0) == expect, (alive, k)
            b = oracle.philox_blocks(seed, [c], [1], 0)[0]
            assert st.t[c] == 5 + oracle.exp_ticks(int(b[0])) and st.n[c] == 1
            assert (st.n.sum() == 1)


def test_still_life_and_empty_torus():
    for block_at in [(0, 0), (3, 5), (7, 7)]:                       # a 2x2 block, across the seams too
        st = oracle.life_init(8, 8, 2, 0, 11)
        r0, q0 = block_at
        cells = {((r0 + a) % 8) * 8 + (q0 + b) % 8 for a in (0, 1) for b in (0, 1)}
        for c in cells:
            st.s[c] = 1
        s0 = st.s.copy()
        ev = oracle.life_run(st, B3, S23, 11, 30 * T32)
        assert ev > 1000 and np.array_equal(st.s, s0)
    st = oracle.life_init(9, 7, 2, 0, 12)
    oracle.life_run(st, B3, S23, 12, 20 * T32)
    assert (st.s < 0).all()


def test_arrival_times_do_not_depend_on_the_rule():
    """Poisson asynchrony: ticks and counts equal those of the Ising run with the same seed."""
    rows, cols, seed, T = 12, 10, 13, 8
    st = oracle.life_init(rows, cols, 0, 1 << 31, seed)
    oracle.life_run(st, B3, S23, seed, T * T32)
    ising = oracle.init(rows, cols, 0, seed)
    oracle.run(ising, oracle.thresholds(0.44), seed, T * T32)
    assert np.array_equal(st.t, ising.t) and np.array_equal(st.n, ising.n)
    s, t, _ = _spec_init(rows, cols, 0, seed)
    assert np.array_equal(oracle.life_init(rows, cols, 0, 1 << 31, seed).t, t)


def test_initial_density():
    for density in (0, 1 << 30, 1 << 31, 3 << 30, (1 << 32) - 1):
        st = oracle.life_init(200, 200, 0, density, 17)
        p = density / 2**32
        assert abs((st.s > 0).mean() - p) < 5 * np.sqrt(max(p * (1 - p), 1e-9) / 40000) + 1e-9
    assert (oracle.life_init(5, 5, 1, 0, 1).s > 0).all()
