"""Pins of the oracle's Ising array on the q-th degree neighbourhood (Sec. 3, reading R14).

Every cell within Manhattan distance q is a neighbour (M = 2q(q+1) of them); the
heat-bath rule uses their spin sum and a cell waits for all of them.  Pinned
against: the plain oracle for q = 1; a brute-force linear-scan simulator; the
heat-bath identity of the table (flip up + flip down = 1 for the same neighbours,
1/2 at beta = 0); arrival times that do not depend on the model.
"""
import numpy as np
import pytest

import oracle
from tests.test_oracle_dynamics import _spec_init

T32 = 1 << 32


def test_q1_is_the_plain_model():
    assert np.array_equal(oracle.thresholds_q(0.44, 1.0, 0.1, 1), oracle.thresholds(0.44, 1.0, 0.1))
    a = oracle.init(9, 11, 0, 4)
    oracle.run_q(a, 1, oracle.thresholds_q(0.5, 1.0, 0.0, 1), 4, 5 * T32)
    b = oracle.init(9, 11, 0, 4)
    oracle.run(b, oracle.thresholds(0.5), 4, 5 * T32)
    assert np.array_equal(a.s, b.s) and np.array_equal(a.t, b.t) and np.array_equal(a.n, b.n)


@pytest.mark.parametrize("q", [2, 3])
def test_table_identities(q):
    M = 2 * q * (q + 1)
    for beta, J, h in [(0.3, 1.0, 0.0), (0.7, 0.5, 0.2), (1.2, -0.4, 0.05)]:
        thr = oracle.thresholds_q(beta, J, h, q).astype(np.int64)
        for j in range(M + 1):
            # same neighbourhood: p(up -> down) + p(down -> up) = 1 (heat bath), within the floors
            assert abs(thr[j + (M + 1)] + thr[j] - 2**32) <= 2
    assert (oracle.thresholds_q(0.0, 1.0, 0.3, q) == 2**31).all()


def _brute_q(rows, cols, q, seed, beta, h, t_end):
    M = 2 * q * (q + 1)
    s, t, n = _spec_init(rows, cols, 0, seed)
    thr = oracle.thresholds_q(beta, 1.0, h, q)
    idx = np.arange(rows * cols)
    offs = [(dr, dx) for dr in range(-q, q + 1) for dx in range(-q, q + 1) if 0 < abs(dr) + abs(dx) <= q]
    assert len(offs) == M
    while True:
        tmin = t.min()
        if tmin >= t_end:
            break
        c = int(idx[t == tmin].min())
        r, x = divmod(c, cols)
        j = sum(1 for dr, dx in offs if s[((r + dr) % rows) * cols + (x + dx) % cols] > 0)
        b = oracle.philox_blocks(seed, [c], [n[c] + 1], 0)[0]
        if b[1] < thr[j + (M + 1) * (1 if s[c] > 0 else 0)]:
            s[c] = -s[c]
        t[c] += oracle.exp_ticks(int(b[0]))
        n[c] += 1
    return s.astype(np.int8), t, n.astype(np.uint32)


@pytest.mark.parametrize("rows,cols,q,seed,beta,h", [(5, 5, 2, 1, 0.2, 0.0), (6, 9, 2, 2, 0.4, 0.1),
                                                     (7, 7, 3, 3, 0.1, 0.0), (8, 10, 3, 4, 0.3, -0.2)])
def test_q_run_equals_brute_force(rows, cols, q, seed, beta, h):
    st = oracle.init(rows, cols, 0, seed)
    oracle.run_q(st, q, oracle.thresholds_q(beta, 1.0, h, q), seed, 4 * T32)
    s, t, n = _brute_q(rows, cols, q, seed, beta, h, 4 * T32)
    assert np.array_equal(st.s, s) and np.array_equal(st.t, t) and np.array_equal(st.n, n)


def test_arrivals_do_not_depend_on_the_neighbourhood():
    a = oracle.init(20, 16, 0, 6)
    oracle.run_q(a, 3, oracle.thresholds_q(0.2, 1.0, 0.0, 3), 6, 7 * T32)
    b = oracle.init(20, 16, 0, 6)
    oracle.run(b, oracle.thresholds(0.44), 6, 7 * T32)
    assert np.array_equal(a.t, b.t) and np.array_equal(a.n, b.n)
