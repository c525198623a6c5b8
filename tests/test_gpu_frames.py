"""GPU parity of snapshot frames (Sec. 3, "Generating the output", Fig. 3.7).

Frame K is every cell's spin after all of its arrivals with tick <= K dt.  The
kernels write frames from their commits while the run proceeds, inside a window of
B frame slots (the figure's lag bound); every frame must equal the oracle's state
at that time bit for bit, for every kernel and tuning, and the trajectory must be
the one without frames.
"""
import ctypes

import numpy as np
import pytest

import oracle
from tests.gpu_util import T32, assert_same, oracle_state

pytestmark = pytest.mark.gpu

ac = pytest.importorskip("paper_cs_0502039_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

ROUND, BLOCKED = ac.AC_KERNEL_ROUND, ac.AC_KERNEL_BLOCKED

CONFIGS = [(ROUND, 32, 1, 0), (ROUND, 64, 2, 0), (ROUND, 64, 6, 0), (ROUND, 64, 8, 0),
           (BLOCKED, 32, 1, 8), (BLOCKED, 64, 1, 2)]

# (rows, cols, beta, h, seed, T, init, dt_ticks, K0, B)
CASES = [
    (48, 80, 0.44, 0.0, 3, 4, 0, T32 // 2, 0, 1),           # one slot: a drain per frame
    (64, 64, 0.44, 0.0, 1, 5, 0, T32, 1, 4),
    (100, 130, 0.6, 0.1, 6, 3, 2, T32 // 9, 0, 8),           # several frames per mean gap
    (96, 96, 0.3, 0.0, 7, 3, 0, 3 * T32 // 4 + 77, 2, 3),    # frame ticks off the unit grid
    (33, 65, 0.9, -0.05, 5, 3, 1, T32 // 4, 0, 64),          # more slots than frames
]


def oracle_frames(rows, cols, beta, h, seed, init, dt, K0, count):
    st = oracle.init(rows, cols, init, seed)
    return oracle.frames(st, oracle.thresholds(beta, 1.0, h), seed, dt, K0, count)


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}_B{c[9]}")
def test_frames_match_oracle_every_kernel(case):
    rows, cols, beta, h, seed, T, init, dt, K0, B = case
    t_end = T * T32
    count = (t_end - 1) // dt - K0 + 1            # frames with K dt < t_end
    ref = oracle_frames(rows, cols, beta, h, seed, init, dt, K0, count)
    ref_state = oracle_state(rows, cols, beta, 1.0, h, seed, T, init)
    for kernel, Lb, rounds, polls in CONFIGS:
        what = f"kernel={kernel} Lb={Lb} rounds={rounds}"
        with ac.Sim(rows, cols, beta, 1.0, h, seed, init=init, kernel=kernel, Lb=Lb, rounds=rounds,
                    polls=polls) as sim:
            sim.configure_frames(dt, K0, B)
            got = sim.run_until_frames(t_end)
            assert [k for k, _ in got] == list(range(K0, K0 + count)), what
            for i, (k, fr) in enumerate(got):
                bad = np.flatnonzero(fr != ref[i])
                assert bad.size == 0, f"{what}: frame {k}: {bad.size} cells differ, first {bad[:5]}"
            s, t, n = sim.read_state()
            assert_same(ref_state, s, t, n, what)
            assert sim.frames_status() == (K0 + count, B, dt)


def test_frames_across_calls_and_at_an_arrival_tick():
    """Frames continue over several run calls (the window carries over), and a frame
    whose tick equals an arrival's tick includes that arrival."""
    rows, cols, beta, seed = 64, 96, 0.44, 9
    st0 = oracle.init(rows, cols, 0, seed)
    dt = int(np.sort(st0.t)[len(st0.t) // 2])      # a first-arrival tick of some cell
    count = 9
    ref = oracle_frames(rows, cols, beta, 0.0, seed, 0, dt, 0, count)
    for kernel, Lb, rounds, polls in [(ROUND, 64, 1, 0), (ROUND, 64, 4, 0), (BLOCKED, 32, 1, 8)]:
        with ac.Sim(rows, cols, beta, 1.0, 0.0, seed, kernel=kernel, Lb=Lb, rounds=rounds, polls=polls) as sim:
            sim.configure_frames(dt, 0, 3)
            got = []
            for stop in (dt // 3, 2 * dt, 2 * dt + 1, 5 * dt + 7, (count - 1) * dt + 1):
                got += sim.run_until_frames(stop)
            assert [k for k, _ in got] == list(range(count))
            for i, (_, fr) in enumerate(got):
                assert np.array_equal(fr, ref[i]), (kernel, rounds, i)
            # a plain run call with frames configured drops the frames it completes
            sim.run_until_ticks((count + 3) * dt + 1)
            assert sim.frames_status()[0] == count + 4
            ref_state = oracle_state(rows, cols, beta, 1.0, 0.0, seed, ((count + 3) * dt + 1) / T32)
            s, t, n = sim.read_state()
            assert_same(ref_state, s, t, n, f"kernel={kernel} rounds={rounds}")


class _DevArray:
    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "|i1", "data": (ptr, False), "version": 3}


def test_device_pointer_frames():
    rows, cols, beta, seed, dt = 80, 80, 0.5, 4, T32 // 2
    ref = oracle_frames(rows, cols, beta, 0.0, seed, 0, dt, 0, 8)
    got = {}

    def on_frame(K, ptr, n):
        t = torch.as_tensor(_DevArray(ptr, n), device="cuda")
        got[K] = t.clone().cpu().numpy()
        torch.cuda.synchronize()

    with ac.Sim(rows, cols, beta, 1.0, 0.0, seed, kernel=ROUND, Lb=64, rounds=4) as sim:
        sim.configure_frames(dt, 0, 2)
        ac.ac_run_until_frames(sim.handle, 4 * T32, on_frame, on_host=False)
    assert sorted(got) == list(range(8))
    for k in range(8):
        assert np.array_equal(got[k], ref[k]), k


def test_frames_argument_checks_and_reset():
    with ac.Sim(32, 32, 0.44, 1.0, 0.0, 1, kernel=ROUND, Lb=32, rounds=1) as sim:
        for dt, K0, B in [(0, 0, 4), (T32, 0, ac.AC_MAX_FRAMES + 1), (T32, -1, 4), (T32, 0, -1),
                          (1 << 60, 0, 4)]:
            with pytest.raises(ac.ACError):
                sim.configure_frames(dt, K0, B)
        with pytest.raises(ac.ACError):
            ac.ac_run_until_frames(sim.handle, T32)            # nothing configured
        sim.run_until(2)
        with pytest.raises(ac.ACError):
            sim.configure_frames(T32 // 2, 3, 4)               # frame 3 at t = 1.5 is past
        sim.configure_frames(T32 // 2, 4, 4)                   # frame 4 at t = 2 is fine (tick <= 2)
        assert sim.frames_status() == (4, 4, T32 // 2)
        with pytest.raises(ac.ACError):
            ac.ac_batch_run_until([sim.handle], [3 * T32])      # batch refuses frames
        sim.reset(1)
        assert sim.frames_status()[1] == 0                      # reset turns frames off
        sim.configure_frames(T32, 0, 2)
        sim.configure_frames(0, 0, 0)                           # B = 0: off
        assert sim.frames_status()[1] == 0
