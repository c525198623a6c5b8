"""Small parity cases for the bounds-checked library (run as a subprocess with AC_LIB_PATH
pointing at libac_check.so): every kernel family on degenerate, ragged and multi-tile tori,
snapshot frames, the Life automaton, the q-th degree neighbourhood, per-cell rates, batches,
asynchronous transfers and the allocation-free entry.  Each result must equal the oracle
bit for bit, and no call may report a bounds violation (AC_ERR_STATE).  Prints one line per
group and exits non-zero on the first difference."""
import sys

import numpy as np


def main() -> int:
    import torch
    import oracle
    import paper_cs_0502039_gb300 as ac
    from tests.gpu_util import T32, assert_same, lib_state, oracle_state
    assert "libac_check" in ac.ac.LIB_PATH, ac.ac.LIB_PATH
    R, B, E = ac.AC_KERNEL_ROUND, ac.AC_KERNEL_BLOCKED, ac.AC_KERNEL_EPOCH
    lattices = [(2, 2, 1), (5, 7, 2), (33, 65, 3), (64, 64, 4), (100, 130, 5), (300, 250, 6), (64, 520, 7)]
    configs = [(R, 32, 1, 0), (R, 64, 8, 0), (R, 64, 13, 0), (B, 32, 1, 8), (B, 64, 1, 8), (E, 64, 8, 0),
               (E, 64, 2, 0), (E, 128, 4, 0)]
    for rows, cols, seed in lattices:
        ref = oracle_state(rows, cols, 0.44, 1.0, 0.05, seed, 3)
        for kernel, Lb, rounds, polls in configs:
            s, t, n, _ = lib_state(rows, cols, 0.44, 1.0, 0.05, seed, 3, 0, kernel, Lb, rounds, polls)
            assert_same(ref, s, t, n, f"{rows}x{cols} kernel={kernel} Lb={Lb} rounds={rounds}")
    for rows, cols, seed in lattices[:5]:       # early commits of certain rejections (one-round kernel)
        ref = oracle_state(rows, cols, 0.9, 1.0, 0.05, seed, 3, 1)
        with ac.Sim(rows, cols, 0.9, 1.0, 0.05, seed, init=1, kernel=R, Lb=32, rounds=1) as sim:
            sim.set_option(ac.AC_OPT_EARLY_REJECT, 1)
            sim.run_until(3)
            assert_same(ref, *sim.read_state(), f"early rejection {rows}x{cols}")
    print("kernels ok", flush=True)
    rows, cols, seed = 48, 80, 1
    st = oracle.init(rows, cols, 0, seed)
    want = oracle.frames(st, oracle.thresholds(0.44), seed, 1 << 31, 0, 6)
    with ac.Sim(rows, cols, 0.44, 1.0, 0.0, seed, kernel=R, Lb=64, rounds=6) as sim:
        sim.configure_frames(1 << 31, 0, 2)
        got = sim.run_until_frames(3 << 32)
    assert [k for k, _ in got] == list(range(6)) and all(np.array_equal(f, want[k]) for k, f in got), "frames"
    print("frames ok", flush=True)
    lref = oracle.life_init(rows, cols, 0, 1 << 31, seed)
    oracle.life_run(lref, oracle.CONWAY_BIRTH, oracle.CONWAY_SURVIVE, seed, 3 << 32)
    with ac.life(rows, cols, seed, 0.5, rounds=4) as sim:
        sim.run_until(3)
        assert_same(lref, *sim.read_state(), "life")
    for q, rounds in ((2, 3), (3, 2)):
        qref = oracle.init(64, 72, 0, seed)
        oracle.run_q(qref, q, oracle.thresholds_q(0.2, 1.0, 0.0, q), seed, 3 << 32)
        with ac.ising_q(64, 72, 0.2, q, seed=seed, rounds=rounds) as sim:
            sim.run_until(3)
            assert_same(qref, *sim.read_state(), f"q = {q}")
    m = (np.arange(rows * cols) % 7 + 1).astype(np.uint32) << 18
    for kernel, rounds in ((R, 6), (E, 4), (B, 1)):
        rref = oracle.init_rated(rows, cols, 0, seed, m)
        oracle.run_rated(rref, oracle.thresholds(0.44), seed, m, 3 << 32)
        with ac.Sim(rows, cols, 0.44, 1.0, 0.0, seed, kernel=kernel, Lb=32, rounds=rounds) as sim:
            sim.set_rates(m)
            sim.run_until(3)
            assert_same(rref, *sim.read_state(), f"rates kernel {kernel}")
    print("models ok", flush=True)
    from paper_cs_0502039_gb300 import workloads
    ws = workloads.batch_workload(n=6, lmin=32, lmax=160, T=3)
    for kernel, rounds in ((E, 8), (R, 8), (B, 1)):
        hs = ac.ac_batch_create([(w["rows"], w["cols"], w["init"]) for w in ws], [w["beta"] for w in ws],
                                [w["J"] for w in ws], [w["h"] for w in ws], [w["seed"] for w in ws])
        sims = [ac.Sim(w["rows"], w["cols"], w["beta"], w["J"], w["h"], w["seed"], handle=h) for w, h in zip(ws, hs)]
        for s_ in sims:
            s_.configure(kernel, 32, rounds, 8)
        for _ in range(2):
            for w, s_ in zip(ws, sims):
                s_.reset(w["seed"], w["init"])
            ac.ac_batch_run_until([s_.handle for s_ in sims], [3 * T32] * len(sims))
        for w, s_ in zip(ws, sims):
            ref = oracle_state(w["rows"], w["cols"], w["beta"], w["J"], w["h"], w["seed"], 3)
            assert_same(ref, *s_.read_state(), f"batch kernel {kernel} {w['rows']}x{w['cols']}")
            s_.close()
    copy = torch.cuda.Stream()
    N = 96 * 130
    bufs = (torch.empty(N, dtype=torch.int8).pin_memory(), torch.empty(N, dtype=torch.int64).pin_memory(),
            torch.empty(N, dtype=torch.int32).pin_memory())
    views = (bufs[0].numpy(), bufs[1].numpy(), bufs[2].numpy().view(np.uint32))
    with ac.Sim(96, 130, 0.44, 1.0, 0.0, 5, kernel=E, rounds=8) as a:
        a.run_until(2)
        ac.ac_read_state_async(a.handle, *views, copy.cuda_stream)
        copy.synchronize()
    with ac.Sim(96, 130, 0.44, 1.0, 0.0, 5, kernel=E, rounds=8) as b:
        ac.ac_load_state_async(b.handle, *views, 2 * T32, copy.cuda_stream)
        b.run_until(4)
        assert_same(oracle_state(96, 130, 0.44, 1.0, 0.0, 5, 4), *b.read_state(), "asynchronous resume")
    with ac.Sim(64, 64, 0.6, 1.0, 0.1, 1, kernel=B, Lb=64) as ref:
        Nn = 64 * 64
        s_ = torch.empty(Nn, dtype=torch.int8, device="cuda")
        t_ = torch.empty(Nn, dtype=torch.int64, device="cuda")
        n_ = torch.empty(Nn, dtype=torch.int32, device="cuda")
        ac.ac_read_state_device(ref.handle, s_.data_ptr(), t_.data_ptr(), n_.data_ptr())
        key = t_ * 2 + (s_ > 0).to(torch.int64)
        ac.ac_run_blocked_static(64, 64, 0.6, 1.0, 0.1, 1, key.data_ptr(), n_.data_ptr(), 3 * T32)
        torch.cuda.synchronize()
        want = oracle_state(64, 64, 0.6, 1.0, 0.1, 1, 3)
        kk = key.cpu().numpy()
        assert np.array_equal((kk >> 1), want.t) and np.array_equal(np.where(kk & 1, 1, -1), want.s), "static entry"
    print("batch, transfers, static entry ok", flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
