"""Pin the oracle's trajectory semantics against things other than itself.

* a brute-force O(N)-per-event linear-scan simulator (same spec, different
  algorithm: no heap) -- bit-exact on tiny tori;
* the exact finite-state chains of the 2x2, 2x3 and 3x3 tori: the Boltzmann
  law is stationary for the generator built from the table, and the oracle's
  state distribution at time T over many seeds matches P0 exp(Q T)
  (chi-square) -- this is Glauber's continuous-time chain of Sec. 1;
* per-cell arrival counts ~ Poisson(T) (Sec. 1, Poisson asynchrony), and
  counts/ticks independent of beta, J, h and the initial spins (the Ising
  law of Sec. 4: next_t does not depend on the states);
* beta = 0: P(s_T = s_0) = (1 + e^-T)/2 per cell;
* Onsager's energy and spontaneous magnetisation away from criticality.
"""
import itertools
import math

import numpy as np
import pytest
import scipy.linalg
import scipy.special
import scipy.stats

import oracle

T32 = 1 << 32


# ---------------------------------------------------------------- brute force
def _spec_init(rows, cols, init_mode, seed):
    """Initial state from the pinned primitives only (readings R3, R4)."""
    N = rows * cols
    cells = np.arange(N, dtype=np.uint32)
    b0 = oracle.philox_blocks(seed, cells, 0, 0)          # B(c, 0): first gap in .x
    ib = oracle.philox_blocks(seed, cells, 0, 1)          # I(c): initial spin from .x
    if init_mode == oracle.INIT_UP:
        s = np.ones(N, dtype=np.int64)
    elif init_mode == oracle.INIT_DOWN:
        s = -np.ones(N, dtype=np.int64)
    else:
        s = np.where(ib[:, 0] & 1, 1, -1).astype(np.int64)
    t = oracle.exp_ticks_many(b0[:, 0]).astype(np.int64)
    return s, t, np.zeros(N, dtype=np.int64)


def _brute_force(rows, cols, init_mode, seed, beta, J, h, t_end):
    s, t, n = _spec_init(rows, cols, init_mode, seed)
    thr = oracle.thresholds(beta, J, h)
    N = rows * cols
    idx = np.arange(N)
    while True:
        tmin = t.min()
        if tmin >= t_end:
            break
        c = int(idx[t == tmin].min())                  # smallest index among equal ticks
        r, q = divmod(c, cols)
        nb = [((r - 1) % rows) * cols + q, ((r + 1) % rows) * cols + q,
              r * cols + (q - 1) % cols, r * cols + (q + 1) % cols]
        j = sum(1 for d in nb if s[d] > 0)
        b = oracle.philox_blocks(seed, [c], [n[c] + 1], 0)[0]
        if b[1] < thr[j + 5 * (1 if s[c] > 0 else 0)]:
            s[c] = -s[c]
        t[c] += oracle.exp_ticks(int(b[0]))
        n[c] += 1
    return s.astype(np.int8), t, n.astype(np.uint32)


@pytest.mark.parametrize("rows,cols,seed,beta,h,T", [
    (2, 2, 1, 0.44, 0.0, 6), (2, 3, 2, 0.7, 0.2, 6), (3, 2, 3, 0.3, -0.1, 6),
    (3, 3, 4, 0.44, 0.0, 5), (4, 5, 5, 1.0, 0.05, 4), (5, 4, 6, 0.2, 0.0, 4),
    (8, 8, 7, 0.44, 0.0, 2), (2, 7, 8, 0.9, 0.3, 4), (6, 2, 9, 0.5, 0.0, 4)])
def test_heap_equals_linear_scan(rows, cols, seed, beta, h, T):
    for init_mode in (oracle.INIT_RANDOM, oracle.INIT_UP):
        st = oracle.init(rows, cols, init_mode, seed)
        oracle.run(st, oracle.thresholds(beta, 1.0, h), seed, T * T32)
        s, t, n = _brute_force(rows, cols, init_mode, seed, beta, 1.0, h, T * T32)
        assert np.array_equal(st.s, s)
        assert np.array_equal(st.t, t)
        assert np.array_equal(st.n, n)


def _tie_round(s0, rows, cols, seed, thr, order):
    s = s0.astype(np.int64).copy()
    for c in order:
        r, q = divmod(c, cols)
        nb = [((r - 1) % rows) * cols + q, ((r + 1) % rows) * cols + q,
              r * cols + (q - 1) % cols, r * cols + (q + 1) % cols]
        j = sum(1 for d in nb if s[d] > 0)
        b = oracle.philox_blocks(seed, [c], [1], 0)[0]
        if b[1] < thr[j + 5 * (s[c] > 0)]:
            s[c] = -s[c]
    return s.astype(np.int8)


def test_forced_tie_is_broken_by_index():
    """Equal ticks: the smaller row-major index commits first (reading R1)."""
    rows, cols = 4, 5
    thr = oracle.thresholds(1.2, 1.0, 0.0)
    distinguishing = 0
    for seed in range(40):
        st = oracle.init(rows, cols, oracle.INIT_RANDOM, seed)
        st.t[:] = 1000                       # every cell has an arrival at tick 1000
        a = st.copy()
        oracle.run(a, thr, seed, 1001)       # exactly one arrival per cell
        asc = _tie_round(st.s, rows, cols, seed, thr, range(rows * cols))
        desc = _tie_round(st.s, rows, cols, seed, thr, reversed(range(rows * cols)))
        assert np.array_equal(a.s, asc)
        assert np.all(a.n == 1)
        distinguishing += int(not np.array_equal(asc, desc))
    assert distinguishing >= 10              # the check has power against other orders


def test_run_splitting_is_exact():
    a = oracle.init(16, 12, oracle.INIT_RANDOM, 9)
    b = a.copy()
    thr = oracle.thresholds(0.44, 1.0, 0.0)
    oracle.run(a, thr, 9, 7 * T32)
    oracle.run(b, thr, 9, 3 * T32 + 12345)
    oracle.run(b, thr, 9, 7 * T32)
    assert np.array_equal(a.s, b.s) and np.array_equal(a.t, b.t) and np.array_equal(a.n, b.n)


# ---------------------------------------------------------- exact enumeration
def _states(N):
    return np.array(list(itertools.product([-1, 1], repeat=N)), dtype=np.int64)


def _nbrs(rows, cols):
    out = []
    for c in range(rows * cols):
        r, q = divmod(c, cols)
        out.append([((r - 1) % rows) * cols + q, ((r + 1) % rows) * cols + q,
                    r * cols + (q - 1) % cols, r * cols + (q + 1) % cols])
    return out


def _energy(sig, rows, cols, J, h):
    e = 0.0
    for c in range(rows * cols):
        r, q = divmod(c, cols)
        e -= J * sig[c] * sig[r * cols + (q + 1) % cols]
        e -= J * sig[c] * sig[((r + 1) % rows) * cols + q]
        e -= h * sig[c]
    return e


def _generator(rows, cols, thr):
    N = rows * cols
    S = _states(N)
    nb = _nbrs(rows, cols)
    index = {tuple(x): i for i, x in enumerate(S)}
    Q = np.zeros((len(S), len(S)))
    for i, sig in enumerate(S):
        for c in range(N):
            j = sum(1 for d in nb[c] if sig[d] > 0)
            rate = float(thr[j + 5 * (sig[c] > 0)]) / 2.0**32
            tgt = sig.copy()
            tgt[c] = -tgt[c]
            Q[i, index[tuple(tgt)]] += rate
        Q[i, i] = -Q[i].sum()
    return S, index, Q


@pytest.mark.parametrize("rows,cols,beta,J,h", [(2, 2, 0.44, 1.0, 0.0), (2, 3, 0.6, 1.0, 0.25),
                                                (3, 3, 0.44, 1.0, -0.15), (3, 3, 1.0, 0.5, 0.05)])
def test_boltzmann_is_stationary(rows, cols, beta, J, h):
    thr = oracle.thresholds(beta, J, h)
    S, _, Q = _generator(rows, cols, thr)
    w = np.array([math.exp(-beta * _energy(s, rows, cols, J, h)) for s in S])
    pi = w / w.sum()
    resid = pi @ Q
    assert np.abs(resid).max() <= 2 * rows * cols * 2.0**-32


@pytest.mark.parametrize("rows,cols,beta,J,h,T,nseeds", [
    (2, 2, 0.6, 1.0, 0.2, 1.5, 20000),
    (2, 3, 0.5, 1.0, -0.3, 2.0, 20000),
    (3, 3, 0.44, 1.0, 0.1, 1.0, 40000)])
def test_transient_law_matches_exp_QT(rows, cols, beta, J, h, T, nseeds):
    thr = oracle.thresholds(beta, J, h)
    S, index, Q = _generator(rows, cols, thr)
    p0 = np.full(len(S), 1.0 / len(S))                 # random init: iid fair spins
    pT = p0 @ scipy.linalg.expm(Q * T)
    counts = np.zeros(len(S))
    t_end = int(T * T32)
    for seed in range(nseeds):
        st = oracle.init(rows, cols, oracle.INIT_RANDOM, seed + 1000)
        oracle.run(st, thr, seed + 1000, t_end)
        counts[index[tuple(st.s.astype(np.int64))]] += 1
    exp = pT * nseeds
    chi2 = ((counts - exp) ** 2 / exp).sum()
    pval = scipy.stats.chi2.sf(chi2, len(S) - 1)
    assert pval > 1e-4, (chi2, pval)
    # the initial law alone must be rejected (the dynamics moved the state)
    chi0 = ((counts - p0 * nseeds) ** 2 / (p0 * nseeds)).sum()
    assert scipy.stats.chi2.sf(chi0, len(S) - 1) < 1e-6


# ------------------------------------------------------------ Poisson arrivals
def test_counts_are_poisson():
    T = 20
    st = oracle.simulate(64, 64, 0.44, 1.0, 0.0, 3, T)
    n = st.n.astype(np.float64)
    N = n.size
    assert abs(n.mean() - T) < 5 * math.sqrt(T / N)
    assert abs(n.var() - T) < 5 * T * math.sqrt(2.0 / N) + 0.5
    ks = np.arange(0, 45)
    hist = np.bincount(st.n.astype(np.int64), minlength=45)[:45].astype(np.float64)
    pmf = scipy.stats.poisson.pmf(ks, T) * N
    keep = pmf > 5
    chi2 = ((hist[keep] - pmf[keep]) ** 2 / pmf[keep]).sum()
    assert scipy.stats.chi2.sf(chi2, keep.sum() - 1) > 1e-4


def test_times_do_not_depend_on_spins_or_parameters():
    """Sec. 4: for the Ising law next_t is independent of the states."""
    ref = oracle.simulate(24, 20, 0.44, 1.0, 0.0, 77, 6)
    for beta, J, h, mode in [(0.0, 1.0, 0.0, 0), (1.5, 1.0, 0.3, 1), (0.3, -0.5, -0.2, 2)]:
        o = oracle.simulate(24, 20, beta, J, h, 77, 6, init_mode=mode)
        assert np.array_equal(o.t, ref.t) and np.array_equal(o.n, ref.n)


def test_beta_zero_closed_form():
    T = 1.0
    st0 = oracle.init(256, 256, oracle.INIT_RANDOM, 5)
    st = st0.copy()
    oracle.run(st, oracle.thresholds(0.0), 5, int(T * T32))
    frac = float((st.s == st0.s).mean())
    p = (1 + math.exp(-T)) / 2
    assert abs(frac - p) < 5 * math.sqrt(p * (1 - p) / st.s.size)


# ------------------------------------------------------------------- Onsager
def _onsager_energy(beta, J=1.0):
    K = 2 * beta * J
    k = 2 * math.sinh(K) / math.cosh(K) ** 2
    Kk = scipy.special.ellipk(k * k)
    return -J / math.tanh(K) * (1 + (2 / math.pi) * (2 * math.tanh(K) ** 2 - 1) * Kk)


def _onsager_m(beta, J=1.0):
    bc = 0.5 * math.log(1 + math.sqrt(2))
    return 0.0 if beta <= bc else (1 - math.sinh(2 * beta * J) ** -4) ** 0.125


def test_onsager_reference_values():
    assert abs(_onsager_energy(0.30) - (-0.70450)) < 5e-5
    assert abs(_onsager_energy(0.60) - (-1.90909)) < 5e-5
    assert abs(_onsager_m(0.60) - 0.97361) < 5e-5


@pytest.mark.parametrize("beta,init_mode,L,t_burn,t_meas", [
    (0.30, oracle.INIT_RANDOM, 192, 10, 40),
    (0.60, oracle.INIT_UP, 96, 10, 40)])
def test_equilibrium_matches_onsager(beta, init_mode, L, t_burn, t_meas):
    seed = 2024
    thr = oracle.thresholds(beta, 1.0, 0.0)
    st = oracle.init(L, L, init_mode, seed)
    es, ms = [], []
    for T in range(t_burn, t_burn + t_meas):
        oracle.run(st, thr, seed, T * T32)
        if T >= t_burn:
            msum, bonds = oracle.observables(st)
            es.append(-bonds / st.s.size)
            ms.append(abs(msum) / st.s.size)
    es, ms = np.array(es), np.array(ms)
    # samples one time unit apart; block them in pairs for a conservative error
    se_e = es.reshape(-1, 2).mean(1).std(ddof=1) / math.sqrt(len(es) / 2)
    assert abs(es.mean() - _onsager_energy(beta)) < 5 * se_e + 2e-3, (es.mean(), se_e)
    se_m = ms.reshape(-1, 2).mean(1).std(ddof=1) / math.sqrt(len(ms) / 2)
    assert abs(ms.mean() - _onsager_m(beta)) < 5 * se_m + (2e-3 if beta > 0.5 else 0.03), (ms.mean(), se_m)
