"""The 512-lattice batch workload at its stated horizon: the 64 smallest lattices of the
workload (L = 32 .. 50, beta in [0.3, 0.6], seeds = their workload index) run in one
batched call to T = 100 and are compared, lattice by lattice and bit for bit, with the
oracle.  Both kernels that run batches on a shared work list are covered.  (The full
512-lattice batch is compared with 512 plain calls, fingerprint by fingerprint, in
bench.py's batch measurement.)"""
import numpy as np
import pytest

import oracle
from tests.gpu_util import T32, assert_same

pytestmark = pytest.mark.gpu

ac = pytest.importorskip("paper_cs_0502039_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_cs_0502039_gb300 import workloads  # noqa: E402


@pytest.fixture(scope="module")
def smallest():
    ws = workloads.batch_workload()
    ws = sorted(ws, key=lambda w: (w["rows"] * w["cols"], w["seed"]))[:64]
    refs = []
    for w in ws:
        st = oracle.init(w["rows"], w["cols"], w["init"], w["seed"])
        oracle.run(st, oracle.thresholds(w["beta"], w["J"], w["h"]), w["seed"], int(w["T"] * T32))
        refs.append(st)
    return ws, refs


@pytest.mark.parametrize("kernel,rounds", [(ac.AC_KERNEL_EPOCH, 8), (ac.AC_KERNEL_ROUND, 8)])
def test_64_smallest_c4_lattices_match_oracle_at_T100(smallest, kernel, rounds):
    ws, refs = smallest
    assert ws[0]["T"] == 100 and len(ws) == 64
    handles = ac.ac_batch_create([(w["rows"], w["cols"], w["init"]) for w in ws], [w["beta"] for w in ws],
                                 [w["J"] for w in ws], [w["h"] for w in ws], [w["seed"] for w in ws])
    sims = [ac.Sim(w["rows"], w["cols"], w["beta"], w["J"], w["h"], w["seed"], handle=h) for w, h in zip(ws, handles)]
    try:
        for s in sims:
            s.configure(kernel, 64, rounds, 0)
        ac.ac_batch_run_until([s.handle for s in sims], [int(w["T"] * T32) for w in ws])
        for w, s, ref in zip(ws, sims, refs):
            assert_same(ref, *s.read_state(), f"C4 lattice seed {w['seed']} ({w['rows']}x{w['cols']})")
            assert s.stats()["events"] == int(ref.n.astype(np.int64).sum())
    finally:
        for s in sims:
            s.close()
