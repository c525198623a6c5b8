"""Pins of the oracle's per-cell rates (the general asynchrony law (A) of Sec. 2, reading R13).

A cell with rate p = 2^20 / m draws its gaps as max(1, floor(e m / 2^20)) from the
rate-1 gap e.  Pinned against: Python integer arithmetic for the scaling; the plain
oracle for m = 2^20; an exact time-scaling identity (all rates 1/2 double every gap,
so the run to 2T is the rate-1 run to T with doubled ticks); a brute-force linear-scan
simulator with random per-cell rates; Poisson(p T) event counts per rate class.
"""
import numpy as np
import pytest

import oracle
from tests.test_oracle_dynamics import _spec_init

T32 = 1 << 32
ONE = oracle.RATE_ONE


def test_rated_gap_arithmetic():
    rng = np.random.default_rng(2)
    for _ in range(3000):
        e = int(rng.integers(1, 2**37))
        m = int(rng.integers(1, 2**32))
        assert oracle.rated_gap(e, m) == max(1, (e * m) >> 20)
    assert oracle.rated_gap(5, ONE) == 5 and oracle.rated_gap(1, 1) == 1


def test_unit_rates_are_the_plain_process():
    rows, cols, seed = 20, 24, 3
    m = np.full(rows * cols, ONE, dtype=np.uint32)
    a = oracle.init_rated(rows, cols, 0, seed, m)
    oracle.run_rated(a, oracle.thresholds(0.44), seed, m, 6 * T32)
    b = oracle.init(rows, cols, 0, seed)
    oracle.run(b, oracle.thresholds(0.44), seed, 6 * T32)
    assert np.array_equal(a.s, b.s) and np.array_equal(a.t, b.t) and np.array_equal(a.n, b.n)


def test_half_rates_double_time_exactly():
    rows, cols, seed, T = 16, 18, 5, 4
    m = np.full(rows * cols, 2 * ONE, dtype=np.uint32)
    a = oracle.init_rated(rows, cols, 0, seed, m)
    oracle.run_rated(a, oracle.thresholds(0.5, 1.0, 0.1), seed, m, 2 * T * T32)
    b = oracle.init(rows, cols, 0, seed)
    oracle.run(b, oracle.thresholds(0.5, 1.0, 0.1), seed, T * T32)
    assert np.array_equal(a.s, b.s) and np.array_equal(a.n, b.n) and np.array_equal(a.t, 2 * b.t)


def _brute_rated(rows, cols, seed, beta, m, t_end):
    s, t, n = _spec_init(rows, cols, 0, seed)
    t = np.array([max(1, (int(v) * int(mm)) >> 20) for v, mm in zip(t, m)], dtype=np.int64)
    thr = oracle.thresholds(beta)
    idx = np.arange(rows * cols)
    while True:
        tmin = t.min()
        if tmin >= t_end:
            break
        c = int(idx[t == tmin].min())
        r, q = divmod(c, cols)
        nb = [((r - 1) % rows) * cols + q, ((r + 1) % rows) * cols + q,
              r * cols + (q - 1) % cols, r * cols + (q + 1) % cols]
        j = sum(1 for d in nb if s[d] > 0)
        b = oracle.philox_blocks(seed, [c], [n[c] + 1], 0)[0]
        if b[1] < thr[j + 5 * (1 if s[c] > 0 else 0)]:
            s[c] = -s[c]
        t[c] += max(1, (oracle.exp_ticks(int(b[0])) * int(m[c])) >> 20)
        n[c] += 1
    return s.astype(np.int8), t, n.astype(np.uint32)


@pytest.mark.parametrize("rows,cols,seed", [(2, 3, 1), (4, 5, 2), (7, 6, 3)])
def test_rated_run_equals_brute_force(rows, cols, seed):
    rng = np.random.default_rng(seed)
    m = rng.integers(ONE // 8, ONE * 8, rows * cols).astype(np.uint32)
    st = oracle.init_rated(rows, cols, 0, seed, m)
    oracle.run_rated(st, oracle.thresholds(0.44), seed, m, 4 * T32)
    s, t, n = _brute_rated(rows, cols, seed, 0.44, m, 4 * T32)
    assert np.array_equal(st.s, s) and np.array_equal(st.t, t) and np.array_equal(st.n, n)


def test_counts_are_poisson_with_the_cell_rate():
    rows, cols, seed, T = 100, 100, 9, 20
    m = np.where(np.arange(rows * cols) % 2 == 0, ONE, 4 * ONE).astype(np.uint32)     # rates 1 and 1/4
    st = oracle.init_rated(rows, cols, 0, seed, m)
    oracle.run_rated(st, oracle.thresholds(0.3), seed, m, T * T32)
    for rate, sel in ((1.0, m == ONE), (0.25, m == 4 * ONE)):
        k = st.n[sel].astype(np.float64)
        mean = rate * T
        assert abs(k.mean() - mean) < 5 * np.sqrt(mean / k.size)
        assert abs(k.var() / mean - 1) < 0.1
