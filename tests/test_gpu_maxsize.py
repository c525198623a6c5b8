"""The largest lattice the C ABI accepts, and runs of zero length.

rows * cols = 65535 * 65537 = 2^32 - 1 cells (51 GB of state, twice that with the
temporal-blocked kernel's second buffer): every 32-bit cell index of the Philox
counter is in use, and the kernels' index arithmetic must not wrap.  The oracle
cannot run this size, so sampled cells are checked one by one against properties
that hold at any size, computed from the oracle's pinned primitives:
  * a cell's arrivals are its own stream's (Sec. 3, per-cell streams; the times do
    not depend on the spins): count = the arrivals before t_end, tick = the next one;
  * a cell that has not arrived keeps its initial spin;
  * a cell whose committed arrivals all precede its four neighbours' first arrivals
    saw the neighbours' initial spins, so its spin follows from the heat-bath rule.
"""
import numpy as np
import pytest

import oracle
from tests.gpu_util import T32

pytestmark = pytest.mark.gpu

ac = pytest.importorskip("paper_cs_0502039_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _arrivals(seed, c, t_end):
    """Committed count and next tick of cell c from its own stream."""
    a = oracle.exp_ticks(int(oracle.philox_blocks(seed, [c], [0], 0)[0][0]))
    n, gaps = 0, []
    while a < t_end:
        n += 1
        b = oracle.philox_blocks(seed, [c], [n], 0)[0]
        gaps.append((a, b))
        a += oracle.exp_ticks(int(b[0]))
    return n, a, gaps


def _first_arrival(seed, c):
    return oracle.exp_ticks(int(oracle.philox_blocks(seed, [c], [0], 0)[0][0]))


def _init_spin(seed, c):
    return 1 if int(oracle.philox_blocks(seed, [c], [0], 1)[0][0]) & 1 else -1


@pytest.mark.skipif(torch.cuda.is_available() and torch.cuda.get_device_properties(0).total_memory < 200 * 2**30,
                    reason="needs about 170 GB of device memory")
def test_largest_lattice_sampled_cells():
    rows, cols, seed, beta = 65535, 65537, 5, 0.44
    N = rows * cols
    assert N == 2**32 - 1
    t_end = T32 // 50
    thr = oracle.thresholds(beta)
    rng = np.random.default_rng(1)
    sample = sorted(set([0, 1, cols - 1, cols, N // 2, N - cols, N - cols - 1, N - 2, N - 1] +
                        list(rng.integers(0, N, 3000))))
    idx = torch.tensor(sample, dtype=torch.int64, device="cuda")
    try:
        _largest_run(rows, cols, seed, beta, t_end, idx, sample, thr, N)
    except ac.ACError as e:
        if "AC_ERR_OOM" in str(e):
            pytest.skip(f"device memory: {e}")
        raise
    except torch.cuda.OutOfMemoryError as e:
        pytest.skip(f"device memory: {e}")


def _largest_run(rows, cols, seed, beta, t_end, idx, sample, thr, N):
    with ac.Sim(rows, cols, beta, 1.0, 0.0, seed, kernel=ac.AC_KERNEL_ROUND, Lb=64, rounds=6) as sim:
        sim.run_until_ticks(t_end)
        st = sim.stats()
        s = torch.empty(N, dtype=torch.int8, device="cuda")
        t = torch.empty(N, dtype=torch.int64, device="cuda")
        n = torch.empty(N, dtype=torch.int32, device="cuda")
        ac.ac_read_state_device(sim.handle, s.data_ptr(), t.data_ptr(), n.data_ptr())
        torch.cuda.synchronize()
        total = int(n.to(torch.int64).sum().item())
        ss, ts, ns = s[idx].cpu().numpy(), t[idx].cpu().numpy(), n[idx].cpu().numpy().astype(np.int64)
        lo, hi = int(t.min().item()), int(n.min().item())
        del s, t, n
    torch.cuda.empty_cache()
    assert total == st["events"] and lo >= t_end and hi >= 0
    assert abs(total - N * t_end / T32) < 6 * np.sqrt(N * t_end / T32)          # Poisson(N T)
    checked_rule = 0
    for j, c in enumerate(sample):
        c = int(c)
        cnt, nxt, gaps = _arrivals(seed, c, t_end)
        assert ns[j] == cnt and ts[j] == nxt, c
        s0 = _init_spin(seed, c)
        if cnt == 0:
            assert ss[j] == s0, c
            continue
        r, q = divmod(c, cols)
        nbrs = [((r - 1) % rows) * cols + q, ((r + 1) % rows) * cols + q,
                r * cols + (q - 1) % cols, r * cols + (q + 1) % cols]
        if min(_first_arrival(seed, d) for d in nbrs) > gaps[-1][0]:
            up = sum(1 for d in nbrs if _init_spin(seed, d) > 0)
            sp = s0
            for _, b in gaps:
                if int(b[1]) < int(thr[up + 5 * (1 if sp > 0 else 0)]):
                    sp = -sp
            assert ss[j] == sp, c
            checked_rule += 1
    assert checked_rule > 20


def test_zero_length_runs():
    rows, cols, seed = 64, 80, 3
    ref = oracle.init(rows, cols, 0, seed)
    for kernel, Lb, rounds in [(ac.AC_KERNEL_ROUND, 64, 1), (ac.AC_KERNEL_ROUND, 64, 6), (ac.AC_KERNEL_BLOCKED, 32, 1)]:
        with ac.Sim(rows, cols, 0.44, 1.0, 0.0, seed, kernel=kernel, Lb=Lb, rounds=rounds) as sim:
            sim.run_until(0)                         # t_end = 0: nothing before it
            sim.run_until_ticks(0)                   # the same t_end again
            s, t, n = sim.read_state()
            assert sim.stats()["events"] == 0
            assert np.array_equal(s, ref.s) and np.array_equal(t, ref.t) and (n == 0).all()
            first = int(ref.t.min())
            sim.run_until_ticks(first)               # strictly before the first arrival
            assert sim.stats()["events"] == 0
            sim.run_until_ticks(first + 1)           # exactly the first arrival
            assert sim.stats()["events"] == 1
