"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, bit-exact.

The trajectory of the Poisson-asynchronous Glauber array is unique given the
per-cell random streams and the (tick, index) order (Sec. 3, uniqueness of the
one-cell-per-PE trajectory; invariance of the aggregated algorithm under
re-partitioning), so spins, next-arrival ticks and per-cell counts must agree
exactly -- tolerance 0 -- for every kernel, tile side and tuning.
"""
import numpy as np
import pytest

import oracle
from tests.gpu_util import T32, assert_same, lib_state, oracle_state

pytestmark = pytest.mark.gpu

ac = pytest.importorskip("paper_cs_0502039_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

ROUND, BLOCKED, EPOCH = ac.AC_KERNEL_ROUND, ac.AC_KERNEL_BLOCKED, ac.AC_KERNEL_EPOCH

# (rows, cols, beta, J, h, seed, T, init): degenerate tori, ragged tiles, several tiles
CASES = [
    (2, 2, 0.44, 1.0, 0.0, 1, 8, 0),
    (2, 3, 0.7, 1.0, 0.2, 2, 8, 0),
    (3, 2, 0.3, 1.0, -0.1, 3, 8, 1),
    (5, 7, 1.0, 1.0, 0.05, 4, 6, 0),
    (33, 65, 0.44, 1.0, 0.0, 5, 4, 0),
    (64, 64, 0.44, 1.0, 0.0, 1, 10, 0),        # 64x64, beta 0.44, seed 1, T = 10
    (100, 130, 0.6, 1.0, 0.1, 6, 3, 2),
    (130, 66, 0.2, 0.8, -0.3, 7, 3, 0),
    (2, 200, 0.5, 1.0, 0.0, 8, 4, 0),
    (257, 3, 0.5, 1.0, 0.0, 9, 4, 0),
    (300, 250, 0.44, 1.0, 0.0, 10, 3, 0),      # several temporal-blocked tiles, seams both ways
    (64, 520, 0.9, 1.0, -0.05, 12, 3, 1),
]

# rounds > 1 selects the temporal-blocked round kernel where rows, cols >= 4 * rounds; 12 is the
# deepest halo of the 96-wide region, 13 the shallowest of the 128-wide one
CONFIGS = [
    (ROUND, 32, 1, 0), (ROUND, 64, 1, 0), (ROUND, 32, 5, 0), (ROUND, 128, 3, 0), (ROUND, 64, 2, 0),
    (ROUND, 64, 8, 0), (ROUND, 64, 12, 0), (ROUND, 64, 13, 0), (ROUND, 64, 16, 0),
    (BLOCKED, 32, 1, 8), (BLOCKED, 64, 1, 8), (BLOCKED, 128, 1, 8), (BLOCKED, 32, 4, 0),
    # the epoch kernel (even halos; odd cols, small tori and the odd halo 5 take its round-kernel fallback)
    (EPOCH, 64, 2, 0), (EPOCH, 64, 6, 0), (EPOCH, 64, 8, 0), (EPOCH, 64, 12, 0), (EPOCH, 64, 14, 0),
    (EPOCH, 64, 16, 0), (EPOCH, 64, 5, 0),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}")
def test_all_kernels_match_oracle(case):
    rows, cols, beta, J, h, seed, T, init = case
    ref = oracle_state(rows, cols, beta, J, h, seed, T, init)
    for kernel, Lb, rounds, polls in CONFIGS:
        s, t, n, stats = lib_state(rows, cols, beta, J, h, seed, T, init, kernel, Lb, rounds, polls)
        assert_same(ref, s, t, n, f"kernel={kernel} Lb={Lb} rounds={rounds} polls={polls}")
        assert stats["events"] == int(ref.n.astype(np.int64).sum())


def test_round_history_equals_time_only_model():
    """Round kernel with one round per launch = Fig. 3.2: per-round enabled counts
    equal those of the oracle's time-only round model (Sec. 4) exactly."""
    rows, cols, seed, T = 64, 64, 1, 10
    st = oracle.init(rows, cols, 0, seed)
    en = oracle.time_rounds(st, seed, T * T32)
    with ac.Sim(rows, cols, 0.44, 1.0, 0.0, seed, kernel=ROUND, Lb=32, rounds=1) as sim:
        sim.run_until(T)
        hist = sim.round_history()
        stats = sim.stats()
    assert np.array_equal(hist.astype(np.int64), en)
    assert stats["global_rounds"] == len(en)
    assert abs(stats["enabled_frac_mean"] - en.mean() / (rows * cols)) < 1e-12


def test_stats_observables_and_checksum():
    rows, cols, beta, seed, T = 96, 80, 0.5, 11, 5
    ref = oracle_state(rows, cols, beta, 1.0, 0.2, seed, T)
    s, t, n, stats = lib_state(rows, cols, beta, 1.0, 0.2, seed, T)
    m, b = oracle.observables(ref)
    assert stats["sum_s"] == m and stats["sum_bonds"] == b
    assert stats["checksum"] == oracle.checksum(ref)
    assert stats["total_counts"] == int(ref.n.astype(np.int64).sum())


@pytest.mark.parametrize("case", [(300, 250, 8), (64, 64, 16), (130, 66, 4), (96, 200, 2)], ids=str)
def test_epoch_kernel_runs_its_own_path(case):
    """The epoch kernel is the path taken (one launch per run call, tile visits counted)
    and matches the oracle; several tiles, the torus seams in both directions."""
    rows, cols, rounds = case
    ref = oracle_state(rows, cols, 0.44, 1.0, 0.0, 3, 4)
    s, t, n, stats = lib_state(rows, cols, 0.44, 1.0, 0.0, 3, 4, 0, EPOCH, 64, rounds, 0)
    assert_same(ref, s, t, n, f"epoch kernel {rows}x{cols} rounds={rounds}")
    assert stats["kernel"] == EPOCH and stats["visits"] > 0 and stats["launches"] >= 1
    assert stats["rounds_per_launch"] == rounds


@pytest.mark.parametrize("kernel", [ROUND, BLOCKED, EPOCH])
def test_run_splitting_and_checkpoint_resume(kernel):
    rows, cols, beta, seed = 70, 90, 0.44, 13
    ref = oracle_state(rows, cols, beta, 1.0, 0.0, seed, 6)
    with ac.Sim(rows, cols, beta, 1.0, 0.0, seed, kernel=kernel, Lb=32, rounds=1 if kernel == BLOCKED else 4) as a:
        a.run_until_ticks(2 * T32 + 777)
        a.run_until(4)
        s, t, n = a.read_state()
    with ac.Sim(rows, cols, beta, 1.0, 0.0, 999, kernel=kernel, Lb=64) as b:
        b.load_state(s, t, n, 4 * T32)
        # the seed is part of the state's identity: restore it with reset + load
        b.reset(seed)
        b.load_state(s, t, n, 4 * T32)
        b.run_until(6)
        s2, t2, n2 = b.read_state()
    assert_same(ref, s2, t2, n2, "checkpoint/resume")


def test_reset_reproduces_create():
    with ac.Sim(40, 40, 0.44, 1.0, 0.0, 5) as a:
        a.run_until(3)
        a.reset(21, ac.AC_INIT_UP)
        a.run_until(2)
        s, t, n = a.read_state()
    ref = oracle_state(40, 40, 0.44, 1.0, 0.0, 21, 2, init=1)
    assert_same(ref, s, t, n, "reset")


def test_read_state_device_matches_host():
    with ac.Sim(50, 60, 0.44, 1.0, 0.0, 3) as sim:
        sim.run_until(2)
        s, t, n = sim.read_state()
        ds = torch.empty(3000, dtype=torch.int8, device="cuda")
        dt = torch.empty(3000, dtype=torch.int64, device="cuda")
        dn = torch.empty(3000, dtype=torch.int32, device="cuda")
        ac.ac_read_state_device(sim.handle, ds.data_ptr(), dt.data_ptr(), dn.data_ptr())
        assert np.array_equal(ds.cpu().numpy(), s)
        assert np.array_equal(dt.cpu().numpy(), t)
        assert np.array_equal(dn.cpu().numpy().view(np.uint32), n)


def test_watchdog_reports_stall_without_fault():
    """With edge publication suppressed a multi-tile lattice cannot finish: the
    bounded polls and the watchdog must end the run with AC_ERR_STALL, and the
    device must stay usable."""
    with ac.Sim(256, 256, 0.44, 1.0, 0.0, 1, kernel=BLOCKED, Lb=32, polls=2) as sim:
        sim.set_option(ac.AC_OPT_WATCHDOG_NS, 50_000_000)
        sim.set_option(ac.AC_OPT_DROP_PUBLISH, 1)
        with pytest.raises(ac.ACError) as ei:
            sim.run_until(20)
        assert ei.value.status == ac.ac.AC_ERR_STALL
    ref = oracle_state(64, 64, 0.44, 1.0, 0.0, 1, 2)
    s, t, n, _ = lib_state(64, 64, 0.44, 1.0, 0.0, 1, 2, kernel=BLOCKED, Lb=32)
    assert_same(ref, s, t, n, "after a stall")


def test_epoch_watchdog_reports_stall_without_fault():
    """The epoch kernel with its epoch words withheld: every tile of the second epoch
    waits on neighbours that never publish, so the bounded waits and the watchdog end
    the run with AC_ERR_STALL; the device stays usable."""
    with ac.Sim(256, 256, 0.44, 1.0, 0.0, 1, kernel=EPOCH, rounds=8) as sim:
        sim.set_option(ac.AC_OPT_WATCHDOG_NS, 50_000_000)
        sim.set_option(ac.AC_OPT_DROP_PUBLISH, 1)
        with pytest.raises(ac.ACError) as ei:
            sim.run_until(20)
        assert ei.value.status == ac.ac.AC_ERR_STALL
    ref = oracle_state(256, 256, 0.44, 1.0, 0.0, 1, 2)
    s, t, n, _ = lib_state(256, 256, 0.44, 1.0, 0.0, 1, 2, kernel=EPOCH, rounds=8)
    assert_same(ref, s, t, n, "after an epoch-kernel stall")


def test_invalid_arguments_are_rejected():
    with ac.Sim(16, 16, 0.44, 1.0, 0.0, 1) as sim:
        sim.run_until(2)
        with pytest.raises(ac.ACError):
            sim.run_until(1)                     # t_end decreasing
        with pytest.raises(ac.ACError):
            sim.configure(BLOCKED, 48)           # unsupported tile side
        bad_t = np.zeros(256, dtype=np.int64)
        with pytest.raises(ac.ACError):
            sim.load_state(np.ones(256, np.int8), bad_t, np.zeros(256, np.uint32), 0)


def test_temporal_blocking_with_uneven_loaded_counts():
    """Counts too far apart for the temporal-blocked kernel's 16-bit window: the run
    must finish through the 32-bit-count kernel and stay bit-exact."""
    rows, cols, seed = 200, 160, 21
    st = oracle.init(rows, cols, 0, seed)
    st.n[: rows * cols // 2] += 100000          # half the cells far ahead in their streams
    ref = st.copy()
    oracle.run(ref, oracle.thresholds(0.5, 1.0, 0.0), seed, 4 * T32)
    with ac.Sim(rows, cols, 0.5, 1.0, 0.0, seed, kernel=ROUND, rounds=8) as sim:
        sim.load_state(st.s, st.t, st.n, 0)
        sim.run_until(4)
        s, t, n = sim.read_state()
    assert_same(ref, s, t, n, "uneven counts")


def test_bkl_class_counts():
    """Cells per BKL class (spin, up neighbours) equal the oracle's count of its own state."""
    for rows, cols, seed, T, kernel, rounds in [(2, 3, 1, 4, ROUND, 1), (64, 64, 1, 10, ROUND, 6),
                                                (100, 130, 6, 3, BLOCKED, 1)]:
        ref = oracle_state(rows, cols, 0.44, 1.0, 0.0, seed, T)
        with ac.Sim(rows, cols, 0.44, 1.0, 0.0, seed, kernel=kernel, Lb=32, rounds=rounds) as sim:
            sim.run_until(T)
            got = sim.class_counts()
        assert np.array_equal(got.astype(np.int64), oracle.class_counts(ref)) and got.sum() == rows * cols
