"""Write stored expected values for the full-size parity tests.

Every value written here comes from the plain CPU oracle (``oracle/``) and
nothing else.  Each case runs one lattice configuration from its initial
state through a list of checkpoints T (t_end = T * 2^32 ticks) and records,
at each checkpoint, the committed-event total, the state fingerprint
(``oracle.checksum``), the magnetisation and bond sums, and (s, t, n) of a
fixed pseudo-random sample of cells.

Cases (the workloads of the parity tests):
  ising4096_b0.30 / b0.4407 / b0.60 -- 4096 x 4096 torus, random init from
      seed 7, J = 1, h = 0, run to T = 50 (checkpoints 1 and 50).
  ising16384_T1 -- 16384 x 16384 torus, all-up init, seed 3, beta = 1.0,
      J = 1, h = 0.05, T = 1 prefix of the T = 20 run.
  life4096 -- the asynchronous Life-like automaton (Conway, B3/S23) on a
      4096 x 4096 torus, half the cells alive at the start (density 2^31,
      seed 7), run to T = 50 (checkpoints 1 and 50).

Usage:  python tests/golden/make_golden.py <case> [<case> ...]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402

CASES = {
    "ising4096_b0.30": dict(rows=4096, cols=4096, init=0, seed=7, beta=0.30, J=1.0, h=0.0, Ts=[1, 50]),
    "ising4096_b0.4407": dict(rows=4096, cols=4096, init=0, seed=7, beta=0.4407, J=1.0, h=0.0, Ts=[1, 50]),
    "ising4096_b0.60": dict(rows=4096, cols=4096, init=0, seed=7, beta=0.60, J=1.0, h=0.0, Ts=[1, 50]),
    "ising16384_T1": dict(rows=16384, cols=16384, init=1, seed=3, beta=1.0, J=1.0, h=0.05, Ts=[1]),
    "life4096": dict(rows=4096, cols=4096, init=0, seed=7, density=1 << 31, birth=oracle.CONWAY_BIRTH,
                     survive=oracle.CONWAY_SURVIVE, Ts=[1, 50], model="life"),
}
NSAMPLE = 256


def sample_cells(N):
    """Fixed sample of cell indices (multiplicative hashing of 0..NSAMPLE-1)."""
    return sorted({(i * 2654435761 + 12345) % N for i in range(NSAMPLE)})


def run_case(name):
    cfg = CASES[name]
    life = cfg.get("model") == "life"
    if life:
        st = oracle.life_init(cfg["rows"], cfg["cols"], cfg["init"], cfg["density"], cfg["seed"])
        out = dict(case=name, source="oracle/ (plain serial heap simulator)", **cfg, checkpoints=[])
    else:
        st = oracle.init(cfg["rows"], cfg["cols"], cfg["init"], cfg["seed"])
        thr = oracle.thresholds(cfg["beta"], cfg["J"], cfg["h"])
        out = dict(case=name, source="oracle/ (plain serial heap simulator)", **cfg,
                   table=[int(v) for v in thr], checkpoints=[])
    cells = sample_cells(cfg["rows"] * cfg["cols"])
    events = 0
    for T in cfg["Ts"]:
        t0 = time.time()
        if life:
            events += oracle.life_run(st, cfg["birth"], cfg["survive"], cfg["seed"], T * oracle.TICKS_PER_UNIT)
        else:
            events += oracle.run(st, thr, cfg["seed"], T * oracle.TICKS_PER_UNIT)
        m, b = oracle.observables(st)
        out["checkpoints"].append(dict(
            T=T, events=events, checksum=str(oracle.checksum(st)), sum_s=m, sum_bonds=b,
            samples=[[c, int(st.s[c]), int(st.t[c]), int(st.n[c])] for c in cells],
            oracle_seconds=round(time.time() - t0, 1)))
        with open(os.path.join(HERE, name + ".json"), "w") as f:
            json.dump(out, f, indent=1)
        print(name, "T", T, "events", events, flush=True)


if __name__ == "__main__":
    for name in sys.argv[1:]:
        run_case(name)
