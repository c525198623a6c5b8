"""Pins of the oracle's time-only round model in 1, 2 and 3 dimensions (Sec. 4).

The model: every cell carries only its local time; in a round a cell advances iff
(t, index) is below the keys of all its neighbours on the circle / torus / cube and
t < t_end, then draws its next increment (exponential, uniform on (0, 1], or
r^(1/8), reading R11).  Pinned against a brute-force Python implementation built
from the separately pinned primitives, against the closed forms of the laws, against
the first-round fraction 1 / (2 dims + 1) of independent continuous times, and
against the limiting efficiencies the paper reports for large arrays.
"""
import numpy as np
import pytest

import oracle

T32 = 1 << 32


def test_laws():
    rng = np.random.default_rng(3)
    xs = np.concatenate([[0, 1, 2, 3, 2**31 - 1, 2**31, 2**32 - 2, 2**32 - 1],
                         rng.integers(0, 2**32, 4000)]).astype(np.uint64)
    for x in xs:
        x = int(x)
        assert oracle.gap(oracle.LAW_EXP, x) == oracle.exp_ticks(x)
        assert oracle.gap(oracle.LAW_UNIFORM, x) == x + 1
        r = (2 * x + 1) / 2**33
        g = oracle.gap(oracle.LAW_ROOT8, x)
        assert abs(g - T32 * r ** 0.125) <= 1e-5 * T32 * r ** 0.125, x
        assert g >= 2**27
    g = [oracle.gap(oracle.LAW_ROOT8, int(x)) for x in np.sort(xs)]
    assert all(a <= b for a, b in zip(g, g[1:]))                 # non-decreasing in x


def _isqrt_big(v):
    s = int(np.sqrt(float(v)))
    while s * s > v:
        s -= 1
    while (s + 1) * (s + 1) <= v:
        s += 1
    return s


def test_root8_steps_by_python_integers():
    for x in [0, 1, 5, 12345, 2**20, 2**31 + 7, 2**32 - 1]:
        s1 = _isqrt_big((2 * x + 1) << 31)
        s2 = _isqrt_big(s1 << 32)
        assert oracle.gap(oracle.LAW_ROOT8, x) == _isqrt_big(s2 << 32)


def _brute(dims, n, law, seed, t_end, max_rounds, q=1):
    N = n ** dims
    idx = np.arange(N)
    coords = [(idx // n ** a) % n for a in range(dims)]
    nbrs = []
    import itertools
    for off in itertools.product(range(-q, q + 1), repeat=dims):
        if not 0 < sum(abs(o) for o in off) <= q:
            continue
        nb = idx.copy()
        for a, o in enumerate(off):
            nb = nb - coords[a] * n ** a + ((coords[a] + o) % n) * n ** a
        nbrs.append(nb)
    t = np.array([oracle.gap(law, int(b[0])) for b in oracle.philox_blocks(seed, idx, np.zeros(N, np.uint32), 0)],
                 dtype=np.int64)
    cnt = np.zeros(N, dtype=np.int64)
    hist = []
    for _ in range(max_rounds):
        en = t < t_end
        for nb in nbrs:
            en &= (t < t[nb]) | ((t == t[nb]) & (idx < nb)) | (nb == idx)
        if not en.any():
            break
        hist.append(int(en.sum()))
        for c in np.flatnonzero(en):
            b = oracle.philox_blocks(seed, [c], [cnt[c] + 1], 0)[0]
            t[c] += oracle.gap(law, int(b[0]))
            cnt[c] += 1
    return np.array(hist, dtype=np.int64), t, cnt.astype(np.uint32)


@pytest.mark.parametrize("dims,n", [(1, 2), (1, 9), (2, 2), (2, 5), (3, 2), (3, 3), (3, 4)])
@pytest.mark.parametrize("law", [0, 1, 2])
def test_model_equals_brute_force(dims, n, law):
    seed, t_end = 17 + dims, 3 * T32
    en, t, cnt = oracle.time_model(dims, n, law, seed, t_end, 10_000)
    en_b, t_b, cnt_b = _brute(dims, n, law, seed, t_end, 10_000)
    assert np.array_equal(en, en_b)
    assert np.array_equal(t, t_b) and np.array_equal(cnt, cnt_b)
    assert (t >= t_end).all()


@pytest.mark.parametrize("dims,n,q", [(1, 9, 2), (1, 13, 4), (2, 5, 2), (2, 7, 3), (3, 5, 2)])
def test_q_neighbourhood_equals_brute_force(dims, n, q):
    """The q-th degree neighbourhood of Sec. 3: every cell within Manhattan distance q."""
    for law in (0, 2):
        en, t, cnt = oracle.time_model(dims, n, law, 31, 2 * T32, 10_000, q=q)
        en_b, t_b, cnt_b = _brute(dims, n, law, 31, 2 * T32, 10_000, q=q)
        assert np.array_equal(en, en_b)
        assert np.array_equal(t, t_b) and np.array_equal(cnt, cnt_b)


@pytest.mark.parametrize("q", [2, 3])
def test_q_first_round_fraction(q):
    """A cell is the strict minimum of itself and its 2q(q+1) neighbours (2D) w.p. 1/(2q(q+1)+1)."""
    n = 300
    en, _, _ = oracle.time_model(2, n, 0, 5, 2**61, 1, q=q)
    p = 1 / (2 * q * (q + 1) + 1)
    assert abs(en[0] / n**2 - p) < 5 * np.sqrt(p * (1 - p) / n**2) * 2


def test_2d_exponential_equals_the_ising_round_model():
    st = oracle.init(24, 24, 0, 5)
    en_ref = oracle.time_rounds(st, 5, 6 * T32)
    en, t, cnt = oracle.time_model(2, 24, 0, 5, 6 * T32, 10_000)
    assert np.array_equal(en, en_ref)
    assert np.array_equal(t, st.t) and np.array_equal(cnt, st.n)


@pytest.mark.parametrize("dims,n", [(1, 60000), (2, 250), (3, 40)])
def test_first_round_fraction(dims, n):
    """Independent continuous times: a cell is the strict minimum of itself and its 2 dims
    neighbours with probability 1 / (2 dims + 1)."""
    N = n ** dims
    for law in (0, 1):
        en, _, _ = oracle.time_model(dims, n, law, 99, 2**61, 1)
        p = 1 / (2 * dims + 1)
        assert abs(en[0] / N - p) < 5 * np.sqrt(p * (1 - p) / N) * 2, (dims, law, en[0] / N)


@pytest.mark.parametrize("dims,n,law,paper", [
    (1, 100_000, 0, 0.247), (1, 100_000, 1, 0.271), (1, 100_000, 2, 0.3388),
    (2, 256, 0, 0.121), (2, 256, 1, 0.132)])
def test_long_run_efficiency_matches_the_paper(dims, n, law, paper):
    """Sec. 4: large-array limits of the fraction of cells advancing per round.  Measured
    over rounds 200..400 (the fraction still drifts down slowly, hence the tolerance)."""
    en, _, _ = oracle.time_model(dims, n, law, 7, 2**61, 400)
    eff = en[200:400].mean() / n ** dims
    assert abs(eff - paper) < 0.004, eff
