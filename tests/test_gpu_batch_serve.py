"""Batched and served runs give each lattice exactly the result it has alone.

Lattices are independent and each trajectory is unique (Sec. 3), so a lattice run in
a batch -- one launch sequence over the tiles of many lattices, replayed from a CUDA
graph on repeated calls -- or inside the continuous-batching server must be
bit-identical to the same lattice run on its own, and to the CPU oracle.
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

from paper_cs_0502039_gb300 import serve as srv_mod  # noqa: E402
from paper_cs_0502039_gb300 import workloads  # noqa: E402


def _make(ws, kernel, rounds):
    handles = ac.ac_batch_create([(w["rows"], w["cols"], w["init"]) for w in ws], [w["beta"] for w in ws],
                                 [w["J"] for w in ws], [w["h"] for w in ws], [w["seed"] for w in ws])
    sims = [ac.Sim(w["rows"], w["cols"], w["beta"], w["J"], w["h"], w["seed"], handle=h) for w, h in zip(ws, handles)]
    for s in sims:
        s.configure(kernel, 64 if kernel == ac.AC_KERNEL_ROUND else 32, rounds, 8)
    return sims


@pytest.mark.parametrize("kernel,rounds", [(ac.AC_KERNEL_ROUND, 8), (ac.AC_KERNEL_ROUND, 4),
                                           (ac.AC_KERNEL_BLOCKED, 1), (ac.AC_KERNEL_EPOCH, 8),
                                           (ac.AC_KERNEL_EPOCH, 4)])
def test_batch_equals_oracle_and_alone(kernel, rounds):
    ws = workloads.batch_workload(n=10, lmin=32, lmax=200, T=3)
    sims = _make(ws, kernel, rounds)
    try:
        # two calls on the same handles: the second replays a captured graph
        ac.ac_batch_run_until([s.handle for s in sims], [2 * T32] * len(sims))
        ac.ac_batch_run_until([s.handle for s in sims], [int(w["T"] * T32) + 5 for w in ws])
        for w, s in zip(ws, sims):
            ref = oracle.init(w["rows"], w["cols"], w["init"], w["seed"])
            oracle.run(ref, oracle.thresholds(w["beta"], w["J"], w["h"]), w["seed"], int(w["T"] * T32) + 5)
            got = s.read_state()
            assert_same(ref, *got, f"batched L={w['rows']}")
            assert s.stats()["events"] == int(ref.n.astype(np.int64).sum())
    finally:
        for s in sims:
            s.close()


@pytest.mark.parametrize("kernel", [ac.AC_KERNEL_ROUND, ac.AC_KERNEL_EPOCH])
def test_batch_with_different_horizons_and_sizes(kernel):
    ws = workloads.batch_workload(n=6, lmin=40, lmax=300, T=4, seed=99)
    horizons = [int((1 + i) * T32) + 3 * i for i in range(len(ws))]
    sims = _make(ws, kernel, 8)
    try:
        ac.ac_batch_run_until([s.handle for s in sims], horizons)
        for w, s, te in zip(ws, sims, horizons):
            ref = oracle.init(w["rows"], w["cols"], w["init"], w["seed"])
            oracle.run(ref, oracle.thresholds(w["beta"], w["J"], w["h"]), w["seed"], te)
            assert_same(ref, *s.read_state(), f"horizon {te}")
    finally:
        for s in sims:
            s.close()


def test_served_jobs_equal_alone():
    reqs = workloads.serve_requests(rate=400.0, duration=0.06, lmin=64, lmax=320, tmin=2.0, tmax=9.0)
    assert len(reqs) >= 10
    results, wall, server = srv_mod.serve(reqs, budget_bytes=128 << 20, slice_T=2.0, realtime=False)
    assert len(results) == len(reqs)
    assert server.steps > 1
    for req, res in zip(sorted(reqs, key=lambda r: r["id"]), results):
        assert res.id == req["id"]
        with ac.Sim(req["rows"], req["cols"], req["beta"], 1.0, 0.0, req["seed"], kernel=ac.AC_KERNEL_BLOCKED,
                    Lb=32) as alone:
            alone.run_until_ticks(int(req["T"] * T32))
            st = alone.stats()
        assert (res.checksum, res.events, res.sum_s, res.sum_bonds) == (st["checksum"], st["events"], st["sum_s"],
                                                                      st["sum_bonds"]), req
        if req["rows"] <= 128:
            ref = oracle_state(req["rows"], req["cols"], req["beta"], 1.0, 0.0, req["seed"], req["T"])
            assert res.checksum == oracle.checksum(ref)


def test_batched_epoch_many_short_calls():
    """Many short batched epoch-kernel calls over a few small lattices (far fewer tiles than
    resident CTAs, so several epochs are claimed at once and every call ends on the stop
    epoch while claims are in flight): every call completes, and the states equal the
    oracle's.  A claim refused by the stop epoch must never leave an accepted item waiting
    on it (the stop epoch travels in the claim word)."""
    ws = workloads.batch_workload(n=6, lmin=48, lmax=128, T=1, seed=5)
    for w in ws:
        w["rows"] -= w["rows"] % 2
        w["cols"] -= w["cols"] % 2
    sims = _make(ws, ac.AC_KERNEL_EPOCH, 4)
    try:
        horizons = [0] * len(ws)
        for call in range(60):
            horizons = [h + T32 // 4 + 977 * (i + 1) * (call % 3) for i, h in enumerate(horizons)]
            ac.ac_batch_run_until([s.handle for s in sims], horizons)
        for w, s, te in zip(ws, sims, horizons):
            ref = oracle.init(w["rows"], w["cols"], w["init"], w["seed"])
            oracle.run(ref, oracle.thresholds(w["beta"], w["J"], w["h"]), w["seed"], te)
            assert_same(ref, *s.read_state(), f"{w['rows']}x{w['cols']} after 60 calls")
    finally:
        for s in sims:
            s.close()
