"""Helpers shared by the GPU tests: run the library and the oracle on one case."""
import numpy as np

import oracle

T32 = 1 << 32


def oracle_state(rows, cols, beta, J, h, seed, T, init=0):
    st = oracle.init(rows, cols, init, seed)
    oracle.run(st, oracle.thresholds(beta, J, h), seed, int(T * T32))
    return st


def lib_state(rows, cols, beta, J, h, seed, T, init=0, kernel=1, Lb=64, rounds=1, polls=8):
    import paper_cs_0502039_gb300 as ac
    with ac.Sim(rows, cols, beta, J, h, seed, init=init, kernel=kernel, Lb=Lb, rounds=rounds,
                polls=polls) as sim:
        sim.run_until_ticks(int(T * T32))
        s, t, n = sim.read_state()
        stats = sim.stats()
    return s, t, n, stats


def assert_same(st, s, t, n, what=""):
    bad_s = np.flatnonzero(st.s != s)
    bad_t = np.flatnonzero(st.t != t)
    bad_n = np.flatnonzero(st.n != n)
    assert bad_s.size == 0 and bad_t.size == 0 and bad_n.size == 0, (
        f"{what}: {bad_s.size} spins, {bad_t.size} ticks, {bad_n.size} counts differ; "
        f"first cells {bad_s[:5]} {bad_t[:5]} {bad_n[:5]}")
