"""Asynchronous state transfers: loads and reads enqueued on a copy stream, overlapping
other handles' runs, give exactly the synchronous results and the oracle's trajectory.

A checkpoint/resume through ac_load_state_async / ac_read_state_async must be the same
state as through the synchronous calls (the random streams are positioned by the counts,
so the resumed trajectory is the oracle's), and a pipeline of several handles -- load the
next lattice and read back the previous one while a lattice runs -- must leave every
lattice bit-identical to its lone run.  An invalid state loaded asynchronously is refused
at the handle's next call, with the state unchanged.
"""
import numpy as np
import pytest

import oracle
from tests.gpu_util import T32, assert_same, oracle_state

pytestmark = pytest.mark.gpu

ac = pytest.importorskip("paper_cs_0502039_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _pinned(N):
    return (torch.empty(N, dtype=torch.int8).pin_memory(), torch.empty(N, dtype=torch.int64).pin_memory(),
            torch.empty(N, dtype=torch.int32).pin_memory())


def _np(bufs):
    s, t, n = bufs
    return s.numpy(), t.numpy(), n.numpy().view(np.uint32)


@pytest.mark.parametrize("kernel,rounds", [(ac.AC_KERNEL_EPOCH, 8), (ac.AC_KERNEL_ROUND, 6),
                                           (ac.AC_KERNEL_BLOCKED, 1)])
def test_async_checkpoint_resume_matches_oracle(kernel, rounds):
    rows, cols, beta, seed = 96, 130, 0.44, 5
    ref = oracle_state(rows, cols, beta, 1.0, 0.0, seed, 5)
    copy = torch.cuda.Stream()
    N = rows * cols
    mid = _pinned(N)
    with ac.Sim(rows, cols, beta, 1.0, 0.0, seed, kernel=kernel, Lb=32, rounds=rounds) as a:
        a.run_until(2)
        ac.ac_read_state_async(a.handle, *_np(mid), copy.cuda_stream)
        a.run_until(3)                      # ordered after the read on the device
        copy.synchronize()
    want = oracle_state(rows, cols, beta, 1.0, 0.0, seed, 2)
    assert_same(want, *_np(mid), "asynchronous read at T = 2")
    out = _pinned(N)
    with ac.Sim(rows, cols, beta, 1.0, 0.0, seed, kernel=kernel, Lb=32, rounds=rounds) as b:
        ac.ac_load_state_async(b.handle, *_np(mid), 2 * T32, copy.cuda_stream)
        b.run_until(5)                      # waits for the load, then continues the trajectory
        ac.ac_read_state_async(b.handle, *_np(out), copy.cuda_stream)
        copy.synchronize()
        assert b.stats()["t_done"] == 5 * T32
    assert_same(ref, *_np(out), "asynchronous resume")


def test_pipeline_overlapping_lattices_equals_lone_runs():
    """Three lattices on one compute stream, their loads and reads on a copy stream, issued so
    that lattice i+1 loads and lattice i-1 is read back while lattice i runs."""
    cases = [(128, 96, 0.3, 1), (200, 160, 0.4407, 2), (64, 256, 0.6, 3)]
    compute, copy = torch.cuda.Stream(), torch.cuda.Stream()
    sims = [ac.Sim(r, c, b, 1.0, 0.0, sd, kernel=ac.AC_KERNEL_EPOCH, rounds=8) for r, c, b, sd in cases]
    try:
        init, outs = [], []
        for s in sims:
            buf = _pinned(s.rows * s.cols)
            ac.ac_read_state(s.handle, *_np(buf))
            init.append(buf)
            outs.append(_pinned(s.rows * s.cols))
            ac.ac_set_stream(s.handle, compute.cuda_stream)
        for _ in range(2):                  # twice: the second pass starts from handles at T = 4
            ac.ac_load_state_async(sims[0].handle, *_np(init[0]), 0, copy.cuda_stream)
            for i, s in enumerate(sims):
                if i + 1 < len(sims):
                    ac.ac_load_state_async(sims[i + 1].handle, *_np(init[i + 1]), 0, copy.cuda_stream)
                s.run_until(4)
                ac.ac_read_state_async(s.handle, *_np(outs[i]), copy.cuda_stream)
            copy.synchronize()
            for (r, c, b, sd), o in zip(cases, outs):
                assert_same(oracle_state(r, c, b, 1.0, 0.0, sd, 4), *_np(o), f"pipelined {r}x{c}")
    finally:
        for s in sims:
            s.close()


def test_invalid_async_load_is_refused_at_the_next_call():
    rows, cols, seed = 40, 48, 7
    copy = torch.cuda.Stream()
    with ac.Sim(rows, cols, 0.44, 1.0, 0.0, seed, kernel=ac.AC_KERNEL_EPOCH, rounds=4) as sim:
        sim.run_until(1)
        before = sim.read_state()
        s, t, n = (x.copy() for x in before)
        s[17] = 0                            # not a spin
        bufs = _pinned(rows * cols)
        for dst, src in zip(_np(bufs), (s, t, n)):
            dst[:] = src
        ac.ac_load_state_async(sim.handle, *_np(bufs), 1 * T32, copy.cuda_stream)
        with pytest.raises(ac.ACError) as ei:
            sim.run_until(2)
        assert ei.value.status == ac.ac.AC_ERR_ARG and "cell 17" in str(ei.value)
        after = sim.read_state()
        assert all(np.array_equal(a, b) for a, b in zip(before, after))
        sim.run_until(2)                     # the handle goes on from its own state
        ref = oracle_state(rows, cols, 0.44, 1.0, 0.0, seed, 2)
        assert_same(ref, *sim.read_state(), "after a refused load")
