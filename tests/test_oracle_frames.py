"""Pins of the oracle's snapshot frames (Sec. 3, "Generating the output", Fig. 3.7).

Frame K is every cell's spin after all of its arrivals with tick <= K dt: the
figure stores a subarray's image before it processes the first event later than
K dt.  The oracle computes a frame as the global state after its heap run to
K dt + 1.  The tests below read the same frames off a different object -- the
per-cell spin histories logged by the brute-force linear-scan simulator -- and
check the one place where the two readings of "the state at K dt" differ: an
arrival exactly at K dt.
"""
import numpy as np
import pytest

import oracle
from tests.test_oracle_dynamics import _spec_init

T32 = 1 << 32


def _histories(rows, cols, init_mode, seed, beta, h, t_end):
    """Brute-force run logging, per cell, the initial spin and (tick, new spin) of every arrival."""
    s, t, n = _spec_init(rows, cols, init_mode, seed)
    thr = oracle.thresholds(beta, 1.0, h)
    N = rows * cols
    idx = np.arange(N)
    hist = [[(-1, int(s[c]))] for c in range(N)]
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
        hist[c].append((int(tmin), int(s[c])))
        t[c] += oracle.exp_ticks(int(b[0]))
        n[c] += 1
    return hist


def _frame_from_histories(hist, T):
    """Each cell's spin after its last logged arrival with tick <= T."""
    out = np.zeros(len(hist), dtype=np.int8)
    for c, h in enumerate(hist):
        v = h[0][1]
        for tick, spin in h[1:]:
            if tick <= T:
                v = spin
            else:
                break
        out[c] = v
    return out


@pytest.mark.parametrize("rows,cols,seed,beta,h,dt,K0,count", [
    (4, 5, 11, 0.44, 0.0, T32 // 2, 0, 7),
    (6, 4, 12, 0.9, 0.1, T32 // 7, 3, 12),
    (5, 5, 13, 0.3, 0.0, 2 * T32 + 12345, 0, 2),
])
def test_frames_equal_history_lookup(rows, cols, seed, beta, h, dt, K0, count):
    for init_mode in (oracle.INIT_RANDOM, oracle.INIT_UP):
        st = oracle.init(rows, cols, init_mode, seed)
        fr = oracle.frames(st, oracle.thresholds(beta, 1.0, h), seed, dt, K0, count)
        hist = _histories(rows, cols, init_mode, seed, beta, h, (K0 + count) * dt + 1)
        for i in range(count):
            assert np.array_equal(fr[i], _frame_from_histories(hist, (K0 + i) * dt)), (init_mode, i)


def test_frame_includes_an_arrival_exactly_at_its_time():
    rows, cols, seed, beta = 4, 4, 21, 0.2
    hist = _histories(rows, cols, oracle.INIT_RANDOM, seed, beta, 0.0, 3 * T32)
    # a flipping arrival: the frame at exactly its tick must show the new spin
    flips = [(tick, c, spin) for c, h in enumerate(hist) for (tick, spin), (_, prev) in zip(h[1:], h[:-1])
             if spin != prev]
    assert flips
    tick, c, spin = flips[len(flips) // 2]
    thr = oracle.thresholds(beta)
    st = oracle.init(rows, cols, oracle.INIT_RANDOM, seed)
    fr = oracle.frames(st, thr, seed, tick, 1, 1)[0]
    assert fr[c] == spin
    # while the state strictly before that tick still has the old spin
    st2 = oracle.init(rows, cols, oracle.INIT_RANDOM, seed)
    oracle.run(st2, thr, seed, tick)
    assert st2.s[c] == -spin


def test_frame_zero_is_the_initial_state_and_frames_leave_the_trajectory_alone():
    rows, cols, seed, beta = 6, 6, 5, 0.44
    thr = oracle.thresholds(beta)
    st = oracle.init(rows, cols, oracle.INIT_RANDOM, seed)
    s0 = st.s.copy()
    fr = oracle.frames(st, thr, seed, T32 // 3, 0, 10)
    assert np.array_equal(fr[0], s0)            # first arrivals are > 0 (reading R3)
    oracle.run(st, thr, seed, 5 * T32)
    ref = oracle.init(rows, cols, oracle.INIT_RANDOM, seed)
    oracle.run(ref, thr, seed, 5 * T32)
    assert np.array_equal(st.s, ref.s) and np.array_equal(st.t, ref.t) and np.array_equal(st.n, ref.n)
