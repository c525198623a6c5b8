"""Full-size parity: 4096 x 4096 (three temperatures and the Life automaton, T = 50) and 16384 x 16384.

The expected values in tests/golden/ were written by tests/golden/make_golden.py,
which calls only the CPU oracle: for each checkpoint the committed-event total,
the state fingerprint, the magnetisation and bond sums and (s, t, n) of 256 fixed
cells.  The GPU runs use the launch configurations the benchmark times.  The
16384 x 16384 run is checked against the oracle on its T = 1 prefix and, to
T = 20, across kernels (the trajectory is unique, Sec. 3), with properties that
hold at any size.
"""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ac = pytest.importorskip("paper_cs_0502039_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
T32 = 1 << 32


def _golden(name):
    with open(os.path.join(GOLDEN, name + ".json")) as f:
        return json.load(f)


def _device_samples(sim, cells):
    N = sim.rows * sim.cols
    s = torch.empty(N, dtype=torch.int8, device="cuda")
    t = torch.empty(N, dtype=torch.int64, device="cuda")
    n = torch.empty(N, dtype=torch.int32, device="cuda")
    ac.ac_read_state_device(sim.handle, s.data_ptr(), t.data_ptr(), n.data_ptr())
    idx = torch.tensor(cells, dtype=torch.int64, device="cuda")
    return (s[idx].cpu().numpy().astype(np.int64), t[idx].cpu().numpy(),
            n[idx].cpu().numpy().view(np.uint32).astype(np.int64))


def _check_checkpoint(sim, cp, what):
    st = sim.stats()
    assert st["checksum"] == int(cp["checksum"]), f"{what}: checksum"
    assert st["total_counts"] == cp["events"], f"{what}: events"
    assert st["sum_s"] == cp["sum_s"] and st["sum_bonds"] == cp["sum_bonds"], f"{what}: observables"
    cells = [c[0] for c in cp["samples"]]
    s, t, n = _device_samples(sim, cells)
    want = np.array([c[1:] for c in cp["samples"]], dtype=np.int64)
    assert np.array_equal(s, want[:, 0]) and np.array_equal(t, want[:, 1]) and np.array_equal(n, want[:, 2]), what


@pytest.mark.parametrize("beta", ["0.30", "0.4407", "0.60"])
@pytest.mark.parametrize("kernel,rounds", [(ac.AC_KERNEL_ROUND, 6), (ac.AC_KERNEL_ROUND, 8), (ac.AC_KERNEL_BLOCKED, 1),
                                           (ac.AC_KERNEL_EPOCH, 8), (ac.AC_KERNEL_EPOCH, 10)])
def test_4096_runs_match_oracle(beta, kernel, rounds):
    g = _golden("ising4096_b" + beta)
    with ac.Sim(g["rows"], g["cols"], g["beta"], g["J"], g["h"], g["seed"], init=g["init"], kernel=kernel,
                Lb=64, rounds=rounds) as sim:
        for cp in g["checkpoints"]:
            sim.run_until(cp["T"])
            _check_checkpoint(sim, cp, f"beta={beta} kernel={kernel} T={cp['T']}")


@pytest.mark.parametrize("rounds", [6, 8])
def test_4096_life_matches_oracle(rounds):
    """The asynchronous Conway automaton on the 4096^2 torus to T = 50 against the oracle's run."""
    g = _golden("life4096")
    with ac.life(g["rows"], g["cols"], g["seed"], g["density"] / 2**32, g["birth"], g["survive"], g["init"],
                 rounds) as sim:
        for cp in g["checkpoints"]:
            sim.run_until(cp["T"])
            _check_checkpoint(sim, cp, f"life rounds={rounds} T={cp['T']}")


@pytest.mark.parametrize("kernel,rounds", [(ac.AC_KERNEL_BLOCKED, 1), (ac.AC_KERNEL_ROUND, 6), (ac.AC_KERNEL_EPOCH, 8)])
def test_4096_batched_run_matches_oracle(kernel, rounds):
    """The three temperatures in one batched call: one graph-captured blocked launch, or one work
    list of all tiles for the temporal-blocked round kernel (replayed launch chunks)."""
    gs = [_golden("ising4096_b" + b) for b in ("0.30", "0.4407", "0.60")]
    sims = [ac.Sim(g["rows"], g["cols"], g["beta"], g["J"], g["h"], g["seed"], init=g["init"],
                   kernel=kernel, Lb=64, rounds=rounds) for g in gs]
    try:
        for T in (1, 50):
            ac.ac_batch_run_until([s.handle for s in sims], [T * T32] * 3)
            for g, s in zip(gs, sims):
                cp = [c for c in g["checkpoints"] if c["T"] == T][0]
                _check_checkpoint(s, cp, f"batched kernel={kernel} beta={g['beta']} T={T}")
    finally:
        for s in sims:
            s.close()


def test_16384_prefix_and_cross_kernel():
    g = _golden("ising16384_T1")
    cp = g["checkpoints"][0]
    results = {}
    for name, kernel, rounds in (("round", ac.AC_KERNEL_ROUND, 8), ("blocked", ac.AC_KERNEL_BLOCKED, 1),
                                 ("epoch", ac.AC_KERNEL_EPOCH, 8)):
        with ac.Sim(g["rows"], g["cols"], g["beta"], g["J"], g["h"], g["seed"], init=g["init"], kernel=kernel,
                    Lb=64, rounds=rounds) as sim:
            sim.run_until(1)
            _check_checkpoint(sim, cp, f"16384 {name} T=1")
            sim.run_until(20)
            st = sim.stats()
            results[name] = (st["checksum"], st["total_counts"], st["sum_s"], st["sum_bonds"])
            N = g["rows"] * g["cols"]
            # every cell's next arrival is past t_end; about 20 arrivals per cell (Poisson, rate 1)
            t = torch.empty(N, dtype=torch.int64, device="cuda")
            ac.ac_read_state_device(sim.handle, 0, t.data_ptr(), 0)
            assert int(t.min().item()) >= 20 * T32
            assert abs(st["total_counts"] / N - 20.0) < 0.01
            # low temperature, positive field, all-up start: the lattice stays almost all up
            assert st["sum_s"] / N > 0.99
    assert results["round"] == results["blocked"] == results["epoch"]
