"""Pin the integer exponential gap exp_ticks (stand-in for -ln r in Eq. (5)).

With 2^32 ticks per unit time and u = (2x+1)/2^33, the gap must be the tick
count of -ln u up to the fixed-point error of the repeated-squaring logarithm
(plus the +1 that keeps next_t > t, Eq. (2)).  The reference value is
computed in binary64 from math.log, whose error (< 1e-15 relative) is far
below one tick; the ln 2 constant is recomputed in exact decimal arithmetic.
"""
import math
from decimal import Decimal, getcontext

import numpy as np

import oracle


def _ref_ticks(x):
    u = (2.0 * np.asarray(x, dtype=np.float64) + 1.0) / 2.0**33
    return -np.log(u) * 2.0**32


def test_ln2_constant_is_floor_ln2_times_2_64():
    getcontext().prec = 80
    v = int(Decimal(2).ln() * (Decimal(2) ** 64))
    assert v == 0xB17217F7D1CF79AB


def test_exp_ticks_error_bound_and_positivity():
    rng = np.random.default_rng(3)
    xs = np.concatenate([
        np.arange(0, 1 << 16, dtype=np.uint64),
        np.arange((1 << 32) - (1 << 16), 1 << 32, dtype=np.uint64),
        rng.integers(0, 1 << 32, 1 << 20, dtype=np.uint64),
        np.array([(1 << k) + d for k in range(32) for d in (-1, 0, 1) if 0 <= (1 << k) + d < (1 << 32)],
                 dtype=np.uint64),
    ]).astype(np.uint32)
    got = oracle.exp_ticks_many(xs).astype(np.float64)
    ref = _ref_ticks(xs)
    err = got - ref
    assert err.max() <= 8.0 and err.min() >= -8.0, (err.min(), err.max())
    assert got.min() >= 1.0
    # floor + 1 adds ~0.5 tick and the truncated squaring underestimates the
    # logarithm by ~1 tick: the mean excess is a few ticks out of 2^32 per unit
    # time (relative rate error < 1e-9)
    assert 0.0 < err.mean() < 3.0


def test_exp_ticks_monotone_non_increasing():
    rng = np.random.default_rng(5)
    xs = np.unique(np.concatenate([
        rng.integers(0, 1 << 32, 1 << 20, dtype=np.uint64),
        np.arange(0, 1 << 14, dtype=np.uint64),
        np.arange((1 << 31) - (1 << 12), (1 << 31) + (1 << 12), dtype=np.uint64),
        np.arange((1 << 32) - (1 << 12), 1 << 32, dtype=np.uint64),
    ])).astype(np.uint32)
    g = oracle.exp_ticks_many(xs).astype(np.int64)
    assert np.all(np.diff(g) <= 0)


def test_exp_ticks_extremes():
    # x = 0: u = 2^-33, -ln u = 33 ln 2
    assert abs(oracle.exp_ticks(0) - 33 * math.log(2) * 2**32) < 8
    # x = 2^32 - 1: u = 1 - 2^-33, -ln u ~ 2^-33 -> 0.5 tick, floor + 1
    assert oracle.exp_ticks(2**32 - 1) in (1, 2)


def test_exp_ticks_distribution_is_exponential():
    """Uniform 32-bit words map to Exp(1) gaps: mean 1, P(gap > t) = e^-t."""
    rng = np.random.default_rng(11)
    xs = rng.integers(0, 1 << 32, 1 << 20, dtype=np.uint64).astype(np.uint32)
    g = oracle.exp_ticks_many(xs).astype(np.float64) / 2.0**32
    assert abs(g.mean() - 1.0) < 5 * 1.0 / math.sqrt(len(g))
    for t in (0.1, 0.5, 1.0, 2.0, 4.0):
        p = (g > t).mean()
        assert abs(p - math.exp(-t)) < 5 * math.sqrt(p * (1 - p) / len(g)) + 1e-6
