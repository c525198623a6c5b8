"""Continuous-batching server for simulation requests.

Each request asks for one lattice (side L, beta, J, h, seed, initial state) run to
time T.  The server keeps the lattices of admitted requests resident on the GPU and
advances all of them together: one step is a single ac_batch_run_until over every
resident handle, moving each to min(its T, its current time + slice).  Between steps
it retires finished requests (their fingerprint and observables are read, the handle
freed) and admits waiting ones while the resident footprint stays within the device
budget, so requests that arrive while others run join the next step.  Every result is
the request's exact trajectory: lattices are independent and their trajectories do not
depend on the schedule.

Footprint of a resident lattice (footprint_bytes): 12 bytes per cell of state, twice
(the round kernel's ping-pong buffers), the two sets of edge words of the tiling
(4 Lb words per tile each), the round history of one-round-per-launch runs, and a
2 MiB allowance for each of the handle's device allocations.  If a creation still
fails for lack of device memory, the request goes back to the head of the queue and
waits until resident lattices retire.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

from . import ac as _ac

TICKS = _ac.TICKS_PER_UNIT
_T0 = [time.perf_counter()]


def now_wall() -> float:
    """Seconds since the current serve() call started (the clock request arrivals use)."""
    return time.perf_counter() - _T0[0]


_ALLOC_SLACK = 2 << 20          # per device allocation of a handle
_ALLOCS = 10                    # key, cnt, key2, cnt2, edge words (2), counters, events, tile flags, reductions
_HISTORY = 1 << 19              # round history (512 KiB), only with one round per launch


def footprint_bytes(rows: int, cols: int, Lb: int = 64, rounds: int = 8) -> int:
    tiles = -(-rows // Lb) * -(-cols // Lb)
    edges = 2 * tiles * 4 * Lb * 8
    hist = _HISTORY if rounds == 1 else 0
    return 24 * rows * cols + edges + hist + _ALLOCS * _ALLOC_SLACK


@dataclass
class Result:
    id: int
    arrival: float
    admitted: float
    finished: float
    events: int
    checksum: int
    sum_s: int
    sum_bonds: int

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclass
class _Job:
    req: dict
    sim: _ac.Sim
    t_end: int
    admitted: float
    t_now: int = 0


@dataclass
class Server:
    budget_bytes: int = 64 << 30
    slice_T: float = 10.0
    kernel: int = _ac.AC_KERNEL_ROUND
    rounds: int = 8
    Lb: int = 64
    max_batch: int = 1024
    resident: list = field(default_factory=list)
    waiting: deque = field(default_factory=deque)
    results: list = field(default_factory=list)
    steps: int = 0
    events: int = 0

    def used(self) -> int:
        return sum(footprint_bytes(j.sim.rows, j.sim.cols, self.Lb, self.rounds) for j in self.resident)

    def submit(self, req: dict) -> None:
        self.waiting.append(req)

    def _admit(self, now: float) -> None:
        used = self.used()
        while self.waiting and len(self.resident) < self.max_batch:
            req = self.waiting[0]
            need = footprint_bytes(req["rows"], req["cols"], self.Lb, self.rounds)
            if self.resident and used + need > self.budget_bytes:
                break
            try:
                sim = _ac.Sim(req["rows"], req["cols"], req["beta"], req.get("J", 1.0), req.get("h", 0.0),
                              req["seed"], init=req.get("init", _ac.AC_INIT_RANDOM), kernel=self.kernel,
                              Lb=self.Lb, rounds=self.rounds)
            except _ac.ACError as e:
                if e.status != _ac.AC_ERR_OOM or not self.resident:
                    raise
                break                   # the request stays first in the queue until lattices retire
            self.waiting.popleft()
            self.resident.append(_Job(req, sim, int(req["T"] * TICKS), now))
            used += need

    def step(self, now: float) -> int:
        """Admit, advance every resident lattice by one slice, retire finished ones."""
        self._admit(now)
        if not self.resident:
            return 0
        slice_ticks = int(self.slice_T * TICKS)
        targets = [min(j.t_end, j.t_now + slice_ticks) for j in self.resident]
        _ac.ac_batch_run_until([j.sim.handle for j in self.resident], targets)
        self.steps += 1
        done_time = now_wall()
        keep = []
        for j, tgt in zip(self.resident, targets):
            j.t_now = tgt
            if tgt >= j.t_end:
                st = j.sim.stats()
                self.events += st["events"]
                self.results.append(Result(j.req["id"], j.req["arrival"], j.admitted, done_time, st["events"],
                                           st["checksum"], st["sum_s"], st["sum_bonds"]))
                j.sim.close()
            else:
                keep.append(j)
        self.resident = keep
        return len(targets)

    def drain(self, clock) -> None:
        while self.resident or self.waiting:
            self.step(clock())


def serve(requests, *, budget_bytes=64 << 30, slice_T=10.0, kernel=_ac.AC_KERNEL_ROUND, rounds=8, Lb=64,
          realtime=True):
    """Run a request stream.  With realtime=True, request i becomes visible at wall
    time start + arrival_i (the stream is replayed at its own pace); otherwise all are
    visible at once.  Returns (results sorted by id, wall seconds, server)."""
    srv = Server(budget_bytes=budget_bytes, slice_T=slice_T, kernel=kernel, rounds=rounds, Lb=Lb)
    pending = deque(sorted(requests, key=lambda r: r["arrival"]))
    _T0[0] = time.perf_counter()
    clock = now_wall

    while pending or srv.waiting or srv.resident:
        now = clock()
        while pending and (not realtime or pending[0]["arrival"] <= now):
            srv.submit(pending.popleft())
        if not srv.waiting and not srv.resident:
            if pending:
                time.sleep(max(0.0, min(pending[0]["arrival"] - now, 0.01)))
            continue
        srv.step(now)
    wall = clock()
    return sorted(srv.results, key=lambda r: r.id), wall, srv
