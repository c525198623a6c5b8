"""One lattice split into row slabs, on one GPU: each slab is a handle that steps its own
rows (R exact synchronous rounds per step) and exchanges its first and last R rows with
its neighbour slabs by device copies after every step.  The union of the slabs' own rows
must be the oracle's trajectory (the trajectory does not depend on the partition, the
remark after Fig. 3.6), on a ragged lattice and on the 4096^2 run to T = 50 whose
expected values the oracle wrote."""
import json
import os

import numpy as np
import pytest

from tests.gpu_util import T32, assert_same, oracle_state

pytestmark = pytest.mark.gpu

ac = pytest.importorskip("paper_cs_0502039_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_cs_0502039_gb300 import slabs  # noqa: E402


def _assemble(sims, plan, rows, cols):
    """The slabs' own rows, read back into one host state (s, t, n)."""
    s = np.empty(rows * cols, np.int8)
    t = np.empty(rows * cols, np.int64)
    n = np.empty(rows * cols, np.uint32)
    for sim, sl in zip(sims, plan):
        buf = torch.empty(sl.nrows * cols * 12, dtype=torch.uint8, device="cuda")
        ac.ac_slab_export(sim.handle, sl.row0, sl.nrows, buf.data_ptr())
        h = buf.cpu().numpy()
        key = h[:sl.nrows * cols * 8].view(np.uint64)
        cnt = h[sl.nrows * cols * 8:].view(np.uint32)
        lo, hi = sl.row0 * cols, (sl.row0 + sl.nrows) * cols
        s[lo:hi] = np.where(key & 1, 1, -1)
        t[lo:hi] = (key >> 1).astype(np.int64)
        n[lo:hi] = cnt
    return s, t, n


@pytest.mark.parametrize("rows,cols,nslabs,R,kernel", [(300, 260, 2, 4, ac.AC_KERNEL_ROUND),
                                                        (300, 260, 3, 8, ac.AC_KERNEL_EPOCH),
                                                        (97, 130, 2, 6, ac.AC_KERNEL_ROUND),
                                                        (64, 64, 4, 4, ac.AC_KERNEL_ROUND)])
def test_slabs_match_oracle(rows, cols, nslabs, R, kernel):
    beta, seed, T = 0.44, 11, 3
    ref = oracle_state(rows, cols, beta, 1.0, 0.05, seed, T)
    plan = slabs.plan(rows, nslabs, R)
    sims = [ac.Sim(rows, cols, beta, 1.0, 0.05, seed, kernel=kernel, Lb=64, rounds=R) for _ in plan]
    try:
        steps = slabs.run_on_one_gpu(ac, sims, plan, R, T * T32)
        assert steps > 1
        assert_same(ref, *_assemble(sims, plan, rows, cols), f"{nslabs} slabs R={R}")
        assert sum(s.stats()["events"] for s in sims) == int(ref.n.astype(np.int64).sum())
    finally:
        for s in sims:
            s.close()


def test_4096_split_in_two_slabs_matches_oracle():
    with open(os.path.join(os.path.dirname(__file__), "golden", "ising4096_b0.4407.json")) as f:
        g = json.load(f)
    R = 8
    plan = slabs.plan(g["rows"], 2, R)
    sims = [ac.Sim(g["rows"], g["cols"], g["beta"], g["J"], g["h"], g["seed"], init=g["init"],
                   kernel=ac.AC_KERNEL_ROUND, Lb=64, rounds=R) for _ in plan]
    try:
        slabs.run_on_one_gpu(ac, sims, plan, R, 50 * T32)
        # gather the own rows into the first handle and take its observables
        for sim, sl in zip(sims[1:], plan[1:]):
            buf = torch.empty(sl.nrows * g["cols"] * 12, dtype=torch.uint8, device="cuda")
            ac.ac_slab_export(sim.handle, sl.row0, sl.nrows, buf.data_ptr())
            ac.ac_slab_import(sims[0].handle, sl.row0, sl.nrows, buf.data_ptr())
        st = sims[0].stats()
        cp = [c for c in g["checkpoints"] if c["T"] == 50][0]
        assert st["checksum"] == int(cp["checksum"])
        assert st["total_counts"] == cp["events"]
        assert (st["sum_s"], st["sum_bonds"]) == (cp["sum_s"], cp["sum_bonds"])
    finally:
        for s in sims:
            s.close()
