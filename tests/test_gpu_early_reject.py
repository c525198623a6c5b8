"""Early commits of certain rejections (AC_OPT_EARLY_REJECT, the one-round kernel): the
trajectory must not change.  Every case is compared with the oracle bit for bit, at
temperatures where the rule commits many arrivals early (the low-temperature, positive-field,
all-up start of the 16384^2 configuration) and where it commits few, for a ferromagnet and
an antiferromagnet (the flip masks make no monotonicity assumption), with per-cell rates,
snapshot frames and runs split across calls."""
import numpy as np
import pytest

import oracle
from tests.gpu_util import T32, assert_same, oracle_state

pytestmark = pytest.mark.gpu

ac = pytest.importorskip("paper_cs_0502039_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from tests.test_gpu_parity import CASES  # noqa: E402


def _er_sim(rows, cols, beta, J, h, seed, init=0, Lb=32):
    sim = ac.Sim(rows, cols, beta, J, h, seed, init=init, kernel=ac.AC_KERNEL_ROUND, Lb=Lb, rounds=1)
    sim.set_option(ac.AC_OPT_EARLY_REJECT, 1)
    return sim


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}")
def test_early_rejection_matches_oracle(case):
    rows, cols, beta, J, h, seed, T, init = case
    ref = oracle_state(rows, cols, beta, J, h, seed, T, init)
    for Lb in (32, 64):
        with _er_sim(rows, cols, beta, J, h, seed, init, Lb) as sim:
            sim.run_until_ticks(int(T * T32))
            assert_same(ref, *sim.read_state(), f"early rejection Lb={Lb}")
            assert sim.stats()["events"] == int(ref.n.astype(np.int64).sum())


@pytest.mark.parametrize("beta,J,h,init", [(1.0, 1.0, 0.05, 1), (0.6, 1.0, 0.0, 0), (0.8, -1.0, 0.1, 0),
                                           (0.2, 1.0, 0.0, 0)])
def test_early_rejection_regimes(beta, J, h, init):
    rows, cols, seed, T = 128, 96, 3, 5
    ref = oracle_state(rows, cols, beta, J, h, seed, T, init)
    with _er_sim(rows, cols, beta, J, h, seed, init) as sim:
        sim.run_until_ticks(2 * T32 + 123)          # split across calls: masks refilled per call
        sim.run_until(T)
        assert_same(ref, *sim.read_state(), f"beta={beta} J={J} h={h}")
        st = sim.stats()
    if beta >= 0.6:
        # low temperature: many rejections go early, and fewer synchronous rounds are needed
        assert st["early_commits"] > 0.2 * st["events"]
        with ac.Sim(rows, cols, beta, J, h, seed, init=init, kernel=ac.AC_KERNEL_ROUND, Lb=32, rounds=1) as plain:
            plain.run_until_ticks(2 * T32 + 123)
            plain.run_until(T)
            base = plain.stats()
        assert st["launches"] < base["launches"]


def test_early_rejection_with_rates_and_frames():
    rows, cols, seed, beta = 48, 80, 1, 0.7
    m = (np.arange(rows * cols) % 7 + 1).astype(np.uint32) << 18
    rref = oracle.init_rated(rows, cols, 0, seed, m)
    oracle.run_rated(rref, oracle.thresholds(beta), seed, m, 4 << 32)
    with _er_sim(rows, cols, beta, 1.0, 0.0, seed) as sim:
        sim.set_rates(m)
        sim.run_until(4)
        assert_same(rref, *sim.read_state(), "rates")
    st = oracle.init(rows, cols, 0, seed)
    want = oracle.frames(st, oracle.thresholds(beta), seed, 1 << 31, 0, 8)
    with _er_sim(rows, cols, beta, 1.0, 0.0, seed) as sim:
        sim.configure_frames(1 << 31, 0, 3)
        got = sim.run_until_frames(4 << 32)
    assert [k for k, _ in got] == list(range(8))
    assert all(np.array_equal(f, want[k]) for k, f in got), "a frame differs"
