"""GPU parity of the Ising array on the q-th degree neighbourhood (Sec. 3, reading R14).

Every cell within Manhattan distance q is a neighbour; the temporal-blocked kernel
(the region losing q rings per round) must reproduce the oracle's heap run bit for
bit for q = 2 and 3, every rounds-per-launch setting, with frames, and with the same
arrival times as the nearest-neighbour array.
"""
import numpy as np
import pytest

import oracle
from tests.gpu_util import T32, assert_same

pytestmark = pytest.mark.gpu

ac = pytest.importorskip("paper_cs_0502039_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

# (rows, cols, q, beta, h, seed, T, init)
CASES = [
    (8, 8, 2, 0.2, 0.0, 1, 4, 0),
    (12, 12, 3, 0.1, 0.0, 2, 4, 0),
    (33, 47, 2, 0.3, 0.1, 3, 4, 0),
    (96, 130, 3, 0.15, -0.05, 4, 3, 1),
    (300, 250, 2, 0.25, 0.0, 5, 2, 0),
    (300, 260, 3, 0.2, 0.0, 6, 2, 0),       # q = 3 with interior (non-wrapping) regions
]


def _oracle(rows, cols, q, beta, h, seed, T, init):
    st = oracle.init(rows, cols, init, seed)
    oracle.run_q(st, q, oracle.thresholds_q(beta, 1.0, h, q), seed, int(T * T32))
    return st


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}_q{c[2]}")
def test_q_neighbourhood_matches_oracle(case):
    rows, cols, q, beta, h, seed, T, init = case
    ref = _oracle(*case)
    for rounds in (1, 2, 4, 6, 8):
        with ac.ising_q(rows, cols, beta, q, 1.0, h, seed, init, rounds) as sim:
            sim.run_until(T)
            s, t, n = sim.read_state()
            assert sim.stats()["events"] == int(ref.n.astype(np.int64).sum())
        assert_same(ref, s, t, n, f"q={q} rounds={rounds}")


def test_q_frames_and_arrivals():
    rows, cols, q, beta, seed, T = 64, 80, 2, 0.2, 7, 4
    dt = T32 // 2
    st = oracle.init(rows, cols, 0, seed)
    thr = oracle.thresholds_q(beta, 1.0, 0.0, q)
    ref = []
    for K in range(2 * T):
        oracle.run_q(st, q, thr, seed, K * dt + 1)
        ref.append(st.s.copy())
    with ac.ising_q(rows, cols, beta, q, seed=seed, rounds=3) as sim:
        sim.configure_frames(dt, 0, 3)
        got = sim.run_until_frames(T * T32)
        _, t1, n1 = sim.read_state()
    assert [k for k, _ in got] == list(range(2 * T))
    for k, f in got:
        assert np.array_equal(f, ref[k]), k
    with ac.Sim(rows, cols, 0.44, 1.0, 0.0, seed, kernel=ac.AC_KERNEL_ROUND, Lb=64, rounds=6) as plain:
        plain.run_until(T)
        _, t2, n2 = plain.read_state()
    assert np.array_equal(t1, t2) and np.array_equal(n1, n2)


def test_q_argument_checks():
    for args in [(16, 16, 0, 0.3, 1.0, 0.0, 1, 1), (16, 16, 0, 0.3, 1.0, 0.0, 4, 1), (11, 16, 0, 0.3, 1.0, 0.0, 3, 1)]:
        with pytest.raises(ac.ACError):
            ac.ac_create_q(*args)
    with ac.ising_q(16, 16, 0.3, 2) as sim:
        with pytest.raises(ac.ACError):
            sim.configure(ac.AC_KERNEL_BLOCKED, 32)
        with pytest.raises(ac.ACError):
            sim.set_rates(np.full(256, ac.AC_RATE_ONE, dtype=np.uint32))
        with pytest.raises(ac.ACError):
            ac.ac_batch_run_until([sim.handle], [T32])
