"""GPU parity of the asynchronous Life-like automaton and of massive tick ties.

Life (reading R12): a cell commits once its key is below all 8 Moore neighbours'
keys; the temporal-blocked kernel must reproduce the oracle's serial heap run bit
for bit (states, ticks, counts) for every rounds-per-launch setting, including
lattices whose small tiles make interior regions wrap across the torus seam.
Ties: states loaded with only a few distinct ticks make the (tick, index) order
decide almost every comparison, across seams too, for every kernel of both models.
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

B3, S23 = ac.AC_LIFE_CONWAY_BIRTH, ac.AC_LIFE_CONWAY_SURVIVE

# (rows, cols, density, birth, survive, seed, T, init)
CASES = [
    (4, 4, 1 << 31, B3, S23, 1, 6, 0),
    (5, 7, 1 << 31, B3, S23, 2, 6, 0),
    (24, 30, 3 << 30, B3, S23, 3, 5, 0),          # small tiles: interior regions wrap
    (64, 64, 1 << 31, B3, S23, 4, 6, 0),
    (100, 130, 1 << 30, (1 << 3) | (1 << 6), S23, 5, 4, 0),   # HighLife
    (300, 250, 1 << 31, B3, S23, 6, 3, 0),        # several tiles, seams both ways
    (96, 520, 1 << 31, 1 << 2, 0, 7, 3, 0),       # B2/S
    (40, 40, 0, B3, S23, 8, 3, 1),                # all alive at the start
]


def _oracle_life(rows, cols, density, birth, survive, seed, T, init):
    st = oracle.life_init(rows, cols, init, density, seed)
    oracle.life_run(st, birth, survive, seed, int(T * T32))
    return st


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}")
def test_life_matches_oracle(case):
    rows, cols, density, birth, survive, seed, T, init = case
    ref = _oracle_life(*case)
    for rounds in (1, 2, 4, 6, 8, 12, 16):
        with ac.life(rows, cols, seed, density / 2**32, birth, survive, init, rounds) as sim:
            sim.run_until(T)
            s, t, n = sim.read_state()
            st = sim.stats()
        assert_same(ref, s, t, n, f"life rounds={rounds}")
        assert st["events"] == int(ref.n.astype(np.int64).sum())


def test_life_ticks_equal_ising_ticks_and_frames():
    rows, cols, seed, T = 130, 100, 9, 4
    with ac.life(rows, cols, seed, 0.5) as lf, ac.Sim(rows, cols, 0.44, 1.0, 0.0, seed, kernel=ac.AC_KERNEL_ROUND,
                                                     Lb=64, rounds=6) as ising:
        lf.run_until(T)
        ising.run_until(T)
        _, t1, n1 = lf.read_state()
        _, t2, n2 = ising.read_state()
    assert np.array_equal(t1, t2) and np.array_equal(n1, n2)
    # snapshot frames of the automaton: frame K = state after all arrivals with tick <= K dt
    dt = T32 // 3
    count = (T * T32 - 1) // dt + 1              # frames with K dt < t_end
    st = oracle.life_init(rows, cols, 0, 1 << 31, seed)
    ref = []
    for K in range(count):
        oracle.life_run(st, B3, S23, seed, K * dt + 1)
        ref.append(st.s.copy())
    with ac.life(rows, cols, seed, 0.5, rounds=4) as lf:
        lf.configure_frames(dt, 0, 5)
        got = lf.run_until_frames(T * T32)
    assert [k for k, _ in got] == list(range(count))
    for k, f in got:
        assert np.array_equal(f, ref[k]), k


def _tied_state(rows, cols, seed):
    rng = np.random.default_rng(seed)
    s = np.where(rng.integers(0, 2, rows * cols) > 0, 1, -1).astype(np.int8)
    t = (1000 + rng.integers(0, 3, rows * cols)).astype(np.int64)     # three distinct ticks
    n = rng.integers(0, 5, rows * cols).astype(np.uint32)
    return s, t, n


@pytest.mark.parametrize("rows,cols", [(24, 30), (64, 96), (130, 250), (6, 7)])
def test_massive_ties_every_kernel(rows, cols):
    s0, t0, n0 = _tied_state(rows, cols, rows * cols)
    t_end = 3 * T32
    ref = oracle.State(rows, cols, s0.copy(), t0.copy(), n0.copy())
    oracle.run(ref, oracle.thresholds(0.5), 21, t_end)
    configs = [(ac.AC_KERNEL_ROUND, 32, 1, 0), (ac.AC_KERNEL_ROUND, 64, 2, 0), (ac.AC_KERNEL_ROUND, 64, 6, 0),
               (ac.AC_KERNEL_BLOCKED, 32, 1, 8), (ac.AC_KERNEL_BLOCKED, 64, 1, 2)]
    for kernel, Lb, rounds, polls in configs:
        with ac.Sim(rows, cols, 0.5, 1.0, 0.0, 21, kernel=kernel, Lb=Lb, rounds=rounds, polls=polls) as sim:
            sim.load_state(s0, t0, n0, 0)
            sim.run_until_ticks(t_end)
            s, t, n = sim.read_state()
        assert_same(ref, s, t, n, f"ising kernel={kernel} Lb={Lb} rounds={rounds}")
    if rows >= 4 and cols >= 4:
        ref = oracle.State(rows, cols, s0.copy(), t0.copy(), n0.copy())
        oracle.life_run(ref, B3, S23, 21, t_end)
        for rounds in (1, 3, 6):
            with ac.life(rows, cols, 21, rounds=rounds) as sim:
                sim.load_state(s0, t0, n0, 0)
                sim.run_until_ticks(t_end)
                s, t, n = sim.read_state()
            assert_same(ref, s, t, n, f"life rounds={rounds}")


def test_life_argument_checks():
    with pytest.raises(ac.ACError):
        ac.ac_create_life(3, 10, 0, 0, B3, S23, 1)             # rows < 4
    with pytest.raises(ac.ACError):
        ac.ac_create_life(10, 10, 0, 0, 1 << 9, S23, 1)        # 10-bit mask
    with ac.life(16, 16, 1) as sim:
        with pytest.raises(ac.ACError):
            sim.configure(ac.AC_KERNEL_BLOCKED, 32)
        with pytest.raises(ac.ACError):
            ac.ac_batch_run_until([sim.handle], [T32])
