"""Seeded synthetic workloads (numpy draws only; none of the simulation's arithmetic).

batch_workload()  many independent lattices: side L log-uniform in [lmin, lmax]
                  (even), beta uniform, seed = index, all run to the same T.
serve_requests()  a Poisson stream of simulation requests: arrival times with
                  exponential gaps at `rate` per second, side L log-uniform in
                  [lmin, lmax] (even), beta and T uniform, seed = request id.
"""
from __future__ import annotations

import numpy as np

WORKLOAD_SEED = 0x5EED0502039


def _even_log_uniform(rng, lo, hi, n):
    return (2 * np.round(np.exp(rng.uniform(np.log(lo), np.log(hi), n)) / 2)).astype(np.int64).clip(lo, hi)


def batch_workload(n=512, lmin=32, lmax=1024, bmin=0.3, bmax=0.6, T=100.0, seed=WORKLOAD_SEED):
    rng = np.random.default_rng(seed)
    L = _even_log_uniform(rng, lmin, lmax, n)
    beta = rng.uniform(bmin, bmax, n)
    return [dict(rows=int(L[i]), cols=int(L[i]), beta=float(beta[i]), J=1.0, h=0.0, seed=i, init=0, T=float(T))
            for i in range(n)]


def serve_requests(rate=200.0, duration=60.0, lmin=64, lmax=2048, bmin=0.25, bmax=0.7, tmin=10.0, tmax=200.0,
                   seed=WORKLOAD_SEED + 1):
    rng = np.random.default_rng(seed)
    n = int(rate * duration * 1.5) + 16
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n))
    arrivals = arrivals[arrivals < duration]
    m = len(arrivals)
    L = _even_log_uniform(rng, lmin, lmax, m)
    beta = rng.uniform(bmin, bmax, m)
    T = rng.uniform(tmin, tmax, m)
    return [dict(id=i, arrival=float(arrivals[i]), rows=int(L[i]), cols=int(L[i]), beta=float(beta[i]), J=1.0,
                 h=0.0, seed=i, init=0, T=float(T[i])) for i in range(m)]
