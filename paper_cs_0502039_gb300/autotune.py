"""Autotuner: pick the kernel and its tuning per lattice size class by timing them.

For a (rows, cols, beta) class -- each side rounded up to a power of two, beta put in
one of three buckets around the critical point -- every candidate configuration runs
the same trajectory (a lattice of the class's size, seed 1, the bucket's beta, about
5e8 arrivals by default) and the one with the highest committed-arrival rate (device
time of the run calls) wins.  The trajectory is the same for every candidate (Sec. 3:
it does not depend on the partition or the schedule), so the tuner changes speed
only; it also checks that every candidate ends in the same state fingerprint.
Results are cached in a JSON file keyed by GPU name and class.

Candidates: the round kernel with R in {4, 6, 8, 10, 12, 16} rounds per launch
(temporal blocking, where the lattice is large enough), R = 8 on the 128-wide region
(512 threads per CTA, one CTA per SM, instead of 384 threads and two CTAs), the epoch
kernel with R in {6, 8, 10, 12} and with R = 8, 10 on the 128-wide region, and the
blocked persistent kernel with tile side 32, 64 or 128 and 2 or 8 halo polls.

tune_batch() does the same for a batch of lattices (one ac_batch_run_until over all of
them) among the kernels that run batches on a shared work list: the round kernel
with temporal blocking and the epoch kernel.
"""
from __future__ import annotations

import json
import os

from . import ac as _ac

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "paper_cs_0502039_gb300", "autotune.json")

CANDIDATES = ([dict(kernel=_ac.AC_KERNEL_ROUND, Lb=64, rounds=r, polls=0) for r in (4, 6, 8, 10, 12, 16)] +
              [dict(kernel=_ac.AC_KERNEL_ROUND, Lb=128, rounds=8, polls=0)] +
              [dict(kernel=_ac.AC_KERNEL_EPOCH, Lb=64, rounds=r, polls=0) for r in (6, 8, 10, 12)] +
              [dict(kernel=_ac.AC_KERNEL_EPOCH, Lb=128, rounds=r, polls=0) for r in (8, 10)] +
              [dict(kernel=_ac.AC_KERNEL_BLOCKED, Lb=lb, rounds=1, polls=p) for lb in (32, 64, 128) for p in (2, 8)])

# batched = False: the lattices run one after another (one persistent launch each), which the
# epoch kernel's dynamic schedule can make faster than one shared work list
BATCH_CANDIDATES = ([dict(kernel=_ac.AC_KERNEL_ROUND, Lb=64, rounds=r, polls=0, batched=True) for r in (4, 6, 8, 10, 12)] +
                    [dict(kernel=_ac.AC_KERNEL_EPOCH, Lb=64, rounds=r, polls=0, batched=b)
                     for r in (6, 8, 10, 12) for b in (True, False)])

BETA_BUCKETS = ((0.35, 0.30), (0.50, 0.44), (float("inf"), 0.60))   # (upper bound, trial beta)


def beta_bucket(beta: float) -> float:
    """The trial temperature of beta's bucket: 0.30 (hot), 0.44 (near critical) or 0.60 (cold)."""
    for upper, trial in BETA_BUCKETS:
        if beta < upper:
            return trial
    return BETA_BUCKETS[-1][1]


def _bucket(n: int) -> int:
    b = 1
    while b < n:
        b *= 2
    return b


def _gpu_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name(0)
    except Exception:
        return "unknown"


def class_key(rows: int, cols: int, beta: float = 0.44) -> str:
    return f"{_gpu_name()}|{_bucket(rows)}x{_bucket(cols)}|b{beta_bucket(beta):.2f}"


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def measure(rows: int, cols: int, cfg: dict, T: float = 2.0, beta: float = 0.44) -> dict:
    with _ac.Sim(rows, cols, beta, 1.0, 0.0, 1, kernel=cfg["kernel"], Lb=cfg["Lb"], rounds=cfg["rounds"],
                 polls=cfg["polls"]) as sim:
        sim.run_until(T)                 # warm-up (module load, graph, allocation of the second buffer)
        sim.reset(1)
        sim.run_until(T)
        st = sim.stats()
    return dict(cfg, events=st["events"], device_ms=st["device_ms"],
                events_per_s=st["events"] / max(st["device_ms"], 1e-6) * 1e3, checksum=st["checksum"])


def horizon(rows: int, cols: int) -> float:
    """Trial length: about 5e8 arrivals (fixed per-call costs then weigh as in real runs), T in [2, 50]."""
    return min(50.0, max(2.0, 5e8 / (_bucket(rows) * _bucket(cols))))


def _store(path: str, key: str, entry: dict) -> None:
    cache = _load(path)
    cache[key] = entry
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, path)


def _entry(results: list) -> dict:
    keys = [k for k in ("kernel", "Lb", "rounds", "polls", "batched", "events_per_s") if k in results[0]]
    best = max(results, key=lambda r: r["events_per_s"])
    entry = {k: best[k] for k in keys}
    entry["measured"] = [{k: r[k] for k in keys} for r in results]
    return entry


def tune(rows: int, cols: int, T: float | None = None, cache_path: str | None = None, force: bool = False,
         beta: float = 0.44, candidates: list | None = None) -> dict:
    """Best configuration for the class of (rows, cols, beta); cached.  T: the trial run's length
    (default: horizon())."""
    path = cache_path or os.environ.get("AC_AUTOTUNE_CACHE", DEFAULT_CACHE)
    cache = _load(path)
    key = class_key(rows, cols, beta)
    if key in cache and not force:
        return cache[key]
    R, C = _bucket(rows), _bucket(cols)
    if T is None:
        T = horizon(rows, cols)
    results = [measure(R, C, cfg, T, beta_bucket(beta)) for cfg in (candidates or CANDIDATES)]
    sums = {r["checksum"] for r in results}
    if len(sums) != 1:
        raise RuntimeError(f"autotune: candidates disagree on the trajectory ({len(sums)} fingerprints)")
    entry = _entry(results)
    _store(path, key, entry)
    return entry


def batch_key(lats) -> str:
    """Class of a batch: its lattice count, the power-of-two bucket of its total cells and the beta
    bucket of its mean beta."""
    cells = sum(r * c for r, c, _ in lats)
    mean_beta = sum(b for _, _, b in lats) / max(1, len(lats))
    return f"{_gpu_name()}|batch{len(lats)}|{_bucket(cells)}|b{beta_bucket(mean_beta):.2f}"


def measure_batch(lats, cfg: dict, T: float) -> dict:
    """One batched run of lattices (rows, cols, beta) (seed i, random start) to T with `cfg`,
    after one untimed warm-up call; the device time of the batched call."""
    handles = _ac.ac_batch_create([(r, c, _ac.AC_INIT_RANDOM) for r, c, _ in lats], [b for _, _, b in lats],
                                  [1.0] * len(lats), [0.0] * len(lats), list(range(len(lats))))
    sims = [_ac.Sim(r, c, b, 1.0, 0.0, i, handle=h) for i, ((r, c, b), h) in enumerate(zip(lats, handles))]
    try:
        for s in sims:
            s.configure(cfg["kernel"], cfg["Lb"], cfg["rounds"], max(cfg["polls"], 0))
        hs = [s.handle for s in sims]
        t_end = [int(T * _ac.TICKS_PER_UNIT)] * len(sims)

        def run():
            if cfg.get("batched", True):
                _ac.ac_batch_run_until(hs, t_end)
            else:
                for h, te in zip(hs, t_end):
                    _ac.ac_run_until_ticks(h, te)
        run()
        for i, s in enumerate(sims):
            s.reset(i)
        run()
        st = [s.stats() for s in sims]
        # device time of the call: shared by the handles of a batch, summed when run one by one
        ms = st[0]["device_ms"] if cfg.get("batched", True) else sum(x["device_ms"] for x in st)
        events = sum(x["events"] for x in st)
        sums = tuple(x["checksum"] for x in st)
    finally:
        for s in sims:
            s.close()
    return dict(cfg, events=events, device_ms=ms, events_per_s=events / max(ms, 1e-6) * 1e3, checksum=sums)


def tune_batch(lats, T: float = 5.0, cache_path: str | None = None, force: bool = False,
               batched_only: bool = False) -> dict:
    """Best batch configuration for lattices [(rows, cols, beta)], timed on the batch itself to T;
    cached per batch class.  batched_only: among the candidates that run one batched call (for
    callers that always batch, e.g. the server)."""
    path = cache_path or os.environ.get("AC_AUTOTUNE_CACHE", DEFAULT_CACHE)
    cache = _load(path)
    key = batch_key(lats) + ("|batched" if batched_only else "")
    if key in cache and not force:
        return cache[key]
    cands = [c for c in BATCH_CANDIDATES if c["batched"] or not batched_only]
    results = [measure_batch(lats, cfg, T) for cfg in cands]
    if len({r["checksum"] for r in results}) != 1:
        raise RuntimeError("autotune: batch candidates disagree on the trajectories")
    entry = _entry(results)
    _store(path, key, entry)
    return entry


def apply(sim: "_ac.Sim", entry: dict) -> None:
    sim.configure(entry["kernel"], entry["Lb"], entry["rounds"], entry["polls"])
