"""Pin the time-only round model (Sec. 4) used to check the round kernel.

In each synchronous round of the one-cell-per-PE algorithm (Fig. 3.2) a cell
advances iff its key is below all four neighbours' keys.  For iid continuous
keys the first round's fraction is exactly 1/5 in expectation (the cell is
the minimum of five), and the paper reports the long-run efficiency of a
large n x n torus with Poisson asynchrony as about 0.121 (Sec. 4).
"""
import numpy as np

import oracle

T32 = 1 << 32


def test_first_round_fraction_is_one_fifth():
    st = oracle.init(512, 512, oracle.INIT_RANDOM, 17)
    en = oracle.time_rounds(st, 17, 1 * T32, max_rounds=1 << 12)
    f1 = en[0] / st.t.size
    assert abs(f1 - 0.2) < 0.004, f1


def test_long_run_fraction_near_0121():
    L = 256
    st = oracle.init(L, L, oracle.INIT_RANDOM, 23)
    en = oracle.time_rounds(st, 23, 60 * T32, max_rounds=1 << 14)
    f = en / (L * L)
    steady = f[200:450].mean()
    assert abs(steady - 0.121) < 0.003, steady
    # every committed arrival is counted once: sum over rounds = total events
    assert en.sum() == int(st.n.astype(np.int64).sum())
    assert np.all(st.t >= 60 * T32)


def test_rounds_reach_the_same_times_as_the_heap():
    """Times do not depend on spins: the round model and the heap agree on (t, n)."""
    a = oracle.init(40, 36, oracle.INIT_RANDOM, 5)
    b = a.copy()
    oracle.time_rounds(a, 5, 9 * T32)
    oracle.run(b, oracle.thresholds(0.44), 5, 9 * T32)
    assert np.array_equal(a.t, b.t) and np.array_equal(a.n, b.n)


def test_observables_and_checksum_by_brute_force():
    st = oracle.simulate(10, 14, 0.44, 1.0, 0.0, 3, 3)
    s = st.s.reshape(10, 14).astype(np.int64)
    m, b = oracle.observables(st)
    assert m == s.sum()
    assert b == int((s * np.roll(s, -1, axis=1)).sum() + (s * np.roll(s, -1, axis=0)).sum())

    def mix(z):
        z &= (1 << 64) - 1
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & ((1 << 64) - 1)
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & ((1 << 64) - 1)
        return z ^ (z >> 31)

    acc = 0
    for c in range(st.s.size):
        z = mix(c)
        z = mix(z ^ int(st.t[c]))
        z = mix(z ^ ((int(st.n[c]) << 1) | int(st.s[c] > 0)))
        acc = (acc + z) & ((1 << 64) - 1)
    assert oracle.checksum(st) == acc
