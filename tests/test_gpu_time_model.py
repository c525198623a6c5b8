"""GPU parity of the time-only round model (Sec. 4) against the oracle, bit-exact.

One circle, torus and cube per increment law (exponential, uniform, r^(1/8)): the
advancing-cell count of every round, the final times and the advance counts must
equal the oracle's.  The 2D exponential case is also the Ising round kernel's own
per-round history (the times do not depend on the spins).
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

ac = pytest.importorskip("paper_cs_0502039_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

T32 = 1 << 32


@pytest.mark.parametrize("dims,n", [(1, 2), (1, 3001), (2, 2), (2, 61), (3, 2), (3, 13)])
@pytest.mark.parametrize("law", [0, 1, 2])
def test_time_model_matches_oracle(dims, n, law):
    seed, t_end = 40 + dims + 3 * law, 5 * T32
    en_ref, t_ref, cnt_ref = oracle.time_model(dims, n, law, seed, t_end, 100_000)
    en, t, cnt, _ = ac.ac_time_model(dims, n, law, seed, t_end, 100_000, want_state=True)
    assert np.array_equal(en.astype(np.int64), en_ref), (dims, n, law)
    assert np.array_equal(t, t_ref) and np.array_equal(cnt, cnt_ref)


@pytest.mark.parametrize("dims,n,q", [(1, 2001, 2), (1, 999, 5), (2, 41, 2), (2, 33, 3), (3, 11, 2)])
def test_q_neighbourhood_matches_oracle(dims, n, q):
    for law in (0, 1):
        en_ref, t_ref, cnt_ref = oracle.time_model(dims, n, law, 77, 3 * T32, 100_000, q=q)
        en, t, cnt, _ = ac.ac_time_model(dims, n, law, 77, 3 * T32, 100_000, want_state=True, q=q)
        assert np.array_equal(en.astype(np.int64), en_ref), (dims, n, q, law)
        assert np.array_equal(t, t_ref) and np.array_equal(cnt, cnt_ref)


def test_round_cap_and_no_end():
    """max_rounds stops the run with the state after exactly that many rounds."""
    for dims, n in [(1, 500), (2, 30), (3, 9)]:
        en_ref, t_ref, cnt_ref = oracle.time_model(dims, n, 2, 3, 2**61, 37)
        en, t, cnt, _ = ac.ac_time_model(dims, n, 2, 3, 2**61, 37, want_state=True)
        assert len(en) == 37 and np.array_equal(en.astype(np.int64), en_ref)
        assert np.array_equal(t, t_ref) and np.array_equal(cnt, cnt_ref)


def test_2d_exponential_equals_the_ising_round_history():
    rows = cols = 64
    with ac.Sim(rows, cols, 0.44, 1.0, 0.0, 1, kernel=ac.AC_KERNEL_ROUND, Lb=32, rounds=1) as sim:
        sim.run_until(10)
        hist = sim.round_history()
    en, _, _, _ = ac.ac_time_model(2, 64, ac.AC_LAW_EXP, 1, 10 * T32, 100_000)
    assert np.array_equal(en, hist)


def test_time_model_argument_checks():
    for args in [(0, 10, 0), (4, 10, 0), (1, 1, 0), (1, 10, 3), (3, 1700, 0), (1, 10, -1)]:
        with pytest.raises(ac.ACError):
            ac.ac_time_model(*args, 1, T32, 10)
    with pytest.raises(ac.ACError):
        ac.ac_time_model(1, 10, 0, 1, -5, 10)
    with pytest.raises(ac.ACError):
        ac.ac_time_model(2, 6, 0, 1, T32, 10, q=3)          # n < 2q + 1
    with pytest.raises(ac.ACError):
        ac.ac_time_model(1, 100, 0, 1, T32, 10, q=9)
