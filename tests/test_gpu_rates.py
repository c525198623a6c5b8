"""GPU parity of per-cell rates (the general asynchrony law (A) of Sec. 2, reading R13).

Cells with rate 2^20 / m[c] draw their gaps as max(1, floor(e m / 2^20)); every kernel
and the batched paths must reproduce the oracle's heap run with the same rates bit for
bit.
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

ONE = ac.AC_RATE_ONE
ROUND, BLOCKED, EPOCH = ac.AC_KERNEL_ROUND, ac.AC_KERNEL_BLOCKED, ac.AC_KERNEL_EPOCH
# (the epoch kernel needs even cols and rows, cols >= 4 x its halo; a handle outside that
# runs the one-round kernel, which these cases then check as well)
CONFIGS = [(ROUND, 32, 1, 0), (ROUND, 64, 2, 0), (ROUND, 64, 6, 0), (BLOCKED, 32, 1, 8), (BLOCKED, 64, 1, 2),
           (EPOCH, 64, 4, 0), (EPOCH, 64, 6, 0)]


def _rates(N, seed, lo=ONE // 8, hi=ONE * 8):
    return np.random.default_rng(seed).integers(lo, hi, N).astype(np.uint32)


def _oracle(rows, cols, beta, h, seed, m, t_end):
    st = oracle.init_rated(rows, cols, 0, seed, m)
    oracle.run_rated(st, oracle.thresholds(beta, 1.0, h), seed, m, t_end)
    return st


@pytest.mark.parametrize("rows,cols,beta,h,seed,T", [(5, 7, 0.44, 0.0, 1, 5), (64, 64, 0.44, 0.0, 2, 4),
                                                     (100, 130, 0.6, 0.1, 3, 3), (300, 250, 0.3, 0.0, 4, 2)])
def test_rates_match_oracle(rows, cols, beta, h, seed, T):
    m = _rates(rows * cols, seed)
    ref = _oracle(rows, cols, beta, h, seed, m, T * T32)
    for kernel, Lb, rounds, polls in CONFIGS:
        with ac.Sim(rows, cols, beta, 1.0, h, seed, kernel=kernel, Lb=Lb, rounds=rounds, polls=polls) as sim:
            sim.set_rates(m)
            sim.run_until(T)
            s, t, n = sim.read_state()
            assert sim.stats()["events"] == int(ref.n.astype(np.int64).sum())
        assert_same(ref, s, t, n, f"rates kernel={kernel} Lb={Lb} rounds={rounds}")


def test_rates_in_batches_and_reset():
    dims = [(40, 50), (96, 96), (130, 70)]
    ms = [_rates(r * c, 10 + i) for i, (r, c) in enumerate(dims)]
    refs = [_oracle(r, c, 0.44, 0.0, 20 + i, m, 3 * T32) for i, ((r, c), m) in enumerate(zip(dims, ms))]
    for kernel, rounds in [(ROUND, 6), (BLOCKED, 1), (EPOCH, 4)]:
        handles = ac.ac_batch_create([(r, c, 0) for r, c in dims], [0.44] * 3, [1.0] * 3, [0.0] * 3, [20, 21, 22])
        sims = [ac.Sim(r, c, 0.44, 1.0, 0.0, 20 + i, handle=h) for i, ((r, c), h) in enumerate(zip(dims, handles))]
        try:
            for sim, m in zip(sims, ms):
                sim.configure(kernel, 32 if kernel == BLOCKED else 64, rounds, 8)
                sim.set_rates(m)
            ac.ac_batch_run_until([s.handle for s in sims], [3 * T32] * 3)
            for sim, ref in zip(sims, refs):
                s, t, n = sim.read_state()
                assert_same(ref, s, t, n, f"batched rates kernel={kernel}")
            sims[0].reset(20)                       # keeps the rates
            sims[0].run_until(3)
            s, t, n = sims[0].read_state()
            assert_same(refs[0], s, t, n, "rates after reset")
        finally:
            for sim in sims:
                sim.close()


def test_rate_argument_checks():
    with ac.Sim(16, 16, 0.44, 1.0, 0.0, 1, kernel=ROUND, Lb=32) as sim:
        with pytest.raises(ac.ACError):
            sim.set_rates(np.zeros(256, dtype=np.uint32))            # a zero multiplier
        sim.set_rates(np.full(256, 2 * ONE, dtype=np.uint32))
        sim.run_until(1)
        with pytest.raises(ac.ACError):
            sim.set_rates(None)                                      # after a run
        sim.reset(1)
        sim.set_rates(None)                                          # back to rate 1
        sim.run_until(2)
        ref = oracle.init(16, 16, 0, 1)
        oracle.run(ref, oracle.thresholds(0.44), 1, 2 * T32)
        s, t, n = sim.read_state()
        assert_same(ref, s, t, n, "rates cleared")
    with ac.life(16, 16, 1) as lf:
        with pytest.raises(ac.ACError):
            lf.set_rates(np.full(256, ONE, dtype=np.uint32))


def test_rates_with_frames_and_resume():
    """Per-cell rates with snapshot frames, and a checkpoint reloaded mid-run."""
    rows, cols, seed, beta, T = 96, 80, 8, 0.44, 4
    m = _rates(rows * cols, 31)
    dt = T32 // 2
    st = oracle.init_rated(rows, cols, 0, seed, m)
    thr = oracle.thresholds(beta)
    ref_frames = []
    for K in range(2 * T):
        oracle.run_rated(st, thr, seed, m, K * dt + 1)
        ref_frames.append(st.s.copy())
    oracle.run_rated(st, thr, seed, m, T * T32)
    with ac.Sim(rows, cols, beta, 1.0, 0.0, seed, kernel=ROUND, Lb=64, rounds=4) as sim:
        sim.set_rates(m)
        sim.configure_frames(dt, 0, 2)
        got = sim.run_until_frames(T * T32)
        s, t, n = sim.read_state()
    assert [k for k, _ in got] == list(range(2 * T))
    assert all(np.array_equal(f, ref_frames[k]) for k, f in got)
    assert_same(st, s, t, n, "rates with frames")
    # checkpoint at T = 2, reload into a fresh handle with the same rates, continue to T
    mid = oracle.init_rated(rows, cols, 0, seed, m)
    oracle.run_rated(mid, thr, seed, m, 2 * T32)
    with ac.Sim(rows, cols, beta, 1.0, 0.0, seed, kernel=BLOCKED, Lb=32, polls=8) as sim:
        sim.set_rates(m)
        sim.load_state(mid.s, mid.t, mid.n, 2 * T32)
        sim.run_until(T)
        s, t, n = sim.read_state()
    assert_same(st, s, t, n, "rates after a reload")


@pytest.mark.parametrize("kernel,rounds", [(ROUND, 6), (EPOCH, 4), (EPOCH, 6)])
def test_rates_on_some_lattices_of_a_batch(kernel, rounds):
    """A batch whose lattices mix per-cell rates and rate 1: the launch runs with rates, and
    a lattice without them keeps its plain trajectory."""
    dims = [(48, 64), (96, 96), (64, 130)]
    ms = [_rates(48 * 64, 31), None, _rates(64 * 130, 33)]
    refs = []
    for i, ((r, c), m) in enumerate(zip(dims, ms)):
        if m is None:
            st = oracle.init(r, c, 0, 40 + i)
            oracle.run(st, oracle.thresholds(0.44, 1.0, 0.0), 40 + i, 3 * T32)
        else:
            st = _oracle(r, c, 0.44, 0.0, 40 + i, m, 3 * T32)
        refs.append(st)
    handles = ac.ac_batch_create([(r, c, 0) for r, c in dims], [0.44] * 3, [1.0] * 3, [0.0] * 3, [40, 41, 42])
    sims = [ac.Sim(r, c, 0.44, 1.0, 0.0, 40 + i, handle=h) for i, ((r, c), h) in enumerate(zip(dims, handles))]
    try:
        for sim, m in zip(sims, ms):
            sim.configure(kernel, 64, rounds, 8)
            if m is not None:
                sim.set_rates(m)
        ac.ac_batch_run_until([s.handle for s in sims], [3 * T32] * 3)
        for sim, ref, m in zip(sims, refs, ms):
            s, t, n = sim.read_state()
            assert_same(ref, s, t, n, f"mixed batch kernel={kernel} rates={m is not None}")
    finally:
        for sim in sims:
            sim.close()
