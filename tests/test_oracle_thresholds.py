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
