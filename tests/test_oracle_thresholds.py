"""Pin the flip-threshold table (appendix flip probabilities, heat-bath rule).

thr[j + 5*(s>0)] / 2^32 is the probability that an arrival flips spin s with
j up-neighbours (neighbour sum S = 2j - 4).  Detailed balance with respect to
exp(-beta E), E = -J sum s s' - h sum s, fixes each pair of reverse moves.
"""
import math

import numpy as np
import pytest

import oracle


def _dE(s, j, J, h):
    S = 2 * j - 4
    return 2.0 * s * (J * S + h)


@pytest.mark.parametrize("beta,J,h", [(0.44, 1.0, 0.0), (0.3, 1.0, 0.0), (1.0, 1.0, 0.05),
                                      (0.6, 0.7, -0.2), (0.25, -1.0, 0.4)])
def test_detailed_balance_pairs(beta, J, h):
    thr = oracle.thresholds(beta, J, h).astype(np.float64) / 2.0**32
    for j in range(5):
        # flipping s=-1 with j up-nbrs, and flipping back s=+1 with the same nbrs
        p_up = thr[j + 0]
        p_dn = thr[j + 5]
        dE = _dE(-1, j, J, h)                    # energy change of the -1 -> +1 move
        q = 2.0**-32
        # p(-1->+1)/p(+1->-1) = exp(-beta dE) up to the 2^-32 quantisation
        lhs = p_up
        rhs = p_dn * math.exp(-beta * dE)
        assert abs(lhs - rhs) <= 2 * q * (1 + math.exp(-beta * dE)) + 1e-15
        # heat-bath: the two probabilities sum to 1 (up to quantisation)
        assert abs(p_up + p_dn - 1.0) <= 2 * q


def test_beta_zero_is_one_half():
    assert np.all(oracle.thresholds(0.0, 1.0, 0.3) == 2**31)


def test_spin_flip_symmetry_at_zero_field():
    thr = oracle.thresholds(0.4407, 1.0, 0.0)
    assert np.array_equal(thr[0:5], thr[5:10][::-1])


def test_appendix_form_agrees_within_one_unit():
    """The appendix computes x/(1+x) with x = exp(-dE/T), T = 1/beta."""
    for beta, J, h in [(0.44, 1.0, 0.0), (1.0, 1.0, 0.05), (0.3, 1.0, 0.1)]:
        thr = oracle.thresholds(beta, J, h)
        for sp in (0, 1):
            s = 2 * sp - 1
            for j in range(5):
                x = math.exp(-_dE(s, j, J, h) * beta)
                p = x / (1.0 + x)
                assert abs(int(thr[j + 5 * sp]) - math.floor(p * 2**32)) <= 1


def test_saturation():
    thr = oracle.thresholds(50.0, 1.0, 0.0)
    assert thr[0] == 0 and thr[9] == 0          # strongly uphill: never flips
    assert thr[4] == 2**32 - 1 and thr[5] == 2**32 - 1   # downhill: always (but u = 2^32-1)


def test_class_counts_by_brute_force():
    """BKL classes (Sec. 3): cells counted by (spin, up neighbours), index j + 5 (s > 0)."""
    import oracle as _o
    for rows, cols, seed, T in [(2, 2, 1, 0), (3, 5, 2, 3), (16, 12, 3, 5)]:
        st = _o.init(rows, cols, 0, seed)
        if T:
            _o.run(st, _o.thresholds(0.44), seed, T << 32)
        want = np.zeros(10, dtype=np.int64)
        for c in range(rows * cols):
            r, q = divmod(c, cols)
            nb = [((r - 1) % rows) * cols + q, ((r + 1) % rows) * cols + q,
                  r * cols + (q - 1) % cols, r * cols + (q + 1) % cols]
            j = sum(1 for d in nb if st.s[d] > 0)
            want[j + 5 * (1 if st.s[c] > 0 else 0)] += 1
        assert np.array_equal(_o.class_counts(st), want)


# ---- the quantisation step against the exact heat-bath probability ----------
#
# The table is thr = min(floor(p 2^32), 2^32 - 1) with p = 1 / (1 + exp(beta dE))
# (appendix flip probability, Sec. 2 Eq. (1) heat-bath rule).  The decimal module
# evaluates p at 60 significant digits from the exact binary values of beta, J
# and h, so floor(p 2^32) is known exactly wherever p 2^32 is not within the
# binary64 evaluation error (a few 1e-6 ticks) of an integer.  A rounding or
# ceiling quantisation fails on about half of the entries.

def _exact_table(beta, J, h, M):
    from decimal import Decimal, getcontext
    getcontext().prec = 60
    b, j_, h_ = Decimal(beta), Decimal(J), Decimal(h)
    two32 = Decimal(2) ** 32
    out = []
    for sp in (0, 1):
        s = 1 if sp else -1
        for j in range(M + 1):
            S = 2 * j - M
            p = 1 / (1 + (b * 2 * s * (j_ * S + h_)).exp())
            out.append(p * two32)
    return out


GRID = [(0.44, 1.0, 0.0), (0.4407, 1.0, 0.0), (0.3, 1.0, 0.0), (0.6, 1.0, 0.0), (1.0, 1.0, 0.05),
        (0.25, -1.0, 0.4), (0.6, 0.7, -0.2), (0.37, 1.3, 0.11), (0.05, 1.0, -0.9), (2.0, 0.5, 0.01)]


def _check_against_exact(thr, exact):
    checked = above_half = 0
    for got, v in zip(thr.tolist(), exact):
        fl = int(v)                                      # v > 0: int() is floor
        frac = float(v - fl)
        if frac < 1e-5 or frac > 1 - 1e-5:              # binary64 may land on either side
            assert got in (fl - 1, fl, fl + 1)
            continue
        assert got == min(fl, 2**32 - 1), (got, v)
        checked += 1
        above_half += frac > 0.5
    return checked, above_half


def test_table_is_the_floor_of_the_exact_probability():
    checked = above_half = 0
    for beta, J, h in GRID:
        c, a = _check_against_exact(oracle.thresholds(beta, J, h), _exact_table(beta, J, h, 4))
        checked += c
        above_half += a
    assert checked >= 80 and above_half >= 10      # the grid does exercise the quantisation


def test_beta_044_table_printed_values():
    """beta = 0.44, J = 1, h = 0, spin -1 with j up neighbours: floor(2^32 p) for
    p = 1 / (1 + exp(-0.88 S)), S = 2j - 4, evaluated at 60 digits; spin +1 mirrors it."""
    want = [123473849, 630459708, 2147483648, 3664507587, 4171493446]
    thr = oracle.thresholds(0.44, 1.0, 0.0)
    assert thr[0:5].tolist() == want and thr[5:10].tolist() == want[::-1]
    assert oracle.thresholds_q(0.44, 1.0, 0.0, 1).tolist() == thr.tolist()
    exact = _exact_table(0.44, 1.0, 0.0, 4)
    assert [int(v) for v in exact[:5]] == want


@pytest.mark.parametrize("q", [1, 2, 3])
def test_q_table_is_the_floor_of_the_exact_probability(q):
    M = 2 * q * (q + 1)
    checked = above_half = 0
    for beta, J, h in GRID[:6]:
        c, a = _check_against_exact(oracle.thresholds_q(beta, J, h, q), _exact_table(beta, J, h, M))
        checked += c
        above_half += a
    assert checked >= 0.8 * 6 * 2 * (M + 1) and above_half >= 5
