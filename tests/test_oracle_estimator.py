"""Pins of the oracle's Monte Carlo estimator (Section 2.1.3, Eq. MCestimator)
against exact rational arithmetic and closed forms."""
from fractions import Fraction

import numpy as np
import pytest


def _exact(v, w, Q):
    """sum_p W^p (v^p)^q in exact rationals (W^p = 1/n without weights)."""
    n = len(v)
    out = []
    for q in range(1, Q + 1):
        if w is None:
            out.append(sum(Fraction(float(x)) ** q for x in v) / n)
        else:
            out.append(sum(Fraction(float(wp)) * Fraction(float(x)) ** q for x, wp in zip(v, w)))
    return out


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("n", [1, 2, 7, 50])
def test_exact_on_dyadic_inputs(orc, weighted, n):
    """Dyadic values a/64 (|a| <= 256) and weights k/1024: every term and
    partial sum is exact in binary64 and the division by a power of two is
    exact too, so the estimator must equal the rational value exactly."""
    rng = np.random.default_rng(n)
    for n_slices in (1, 3):
        v = rng.integers(-256, 257, size=(n_slices, n)) / 64.0
        w = rng.integers(0, 1025, size=(n_slices, n)) / 1024.0 if weighted else None
        got = orc.moments(v, 4, w)
        for s in range(n_slices):
            if not weighted and n & (n - 1):
                # division by a non-power of two rounds once
                ex = [float(e) for e in _exact(v[s], None, 4)]
                np.testing.assert_allclose(got[s], ex, rtol=2.3e-16, atol=0)
            else:
                ex = _exact(v[s], None if w is None else w[s], 4)
                assert [Fraction(g) for g in got[s]] == ex, (s, got[s], ex)


@pytest.mark.parametrize("k", [0, 3, 6])
def test_faulhaber_closed_forms(orc, k):
    """x_p = p / 2^k, p = 0..n-1 with n = 2^k: (1/n) sum_p x_p^q from the
    closed forms of sum_p p^q (Faulhaber), exact."""
    n = 1 << k
    v = np.arange(n, dtype=np.float64) / n
    m = n - 1
    sums = [Fraction(m * (m + 1), 2), Fraction(m * (m + 1) * (2 * m + 1), 6), Fraction(m * (m + 1), 2) ** 2,
            Fraction(m * (m + 1) * (2 * m + 1) * (3 * m * m + 3 * m - 1), 30)]
    got = orc.moments(v, 4)[0]
    for q in range(1, 5):
        assert Fraction(got[q - 1]) == sums[q - 1] / Fraction(n) ** (q + 1), (q, got[q - 1])


def test_uniform_weights_equal_the_unweighted_estimator_of_powers_of_two(orc):
    """W^p = 1/n given explicitly equals the unweighted form when n is a power
    of two (1/n exact), and a weight vector concentrated on one particle
    gives that particle's powers."""
    rng = np.random.default_rng(3)
    v = rng.standard_normal((2, 256))
    w = np.full((2, 256), 1.0 / 256)
    np.testing.assert_allclose(orc.moments(v, 3, w), orc.moments(v, 3), rtol=1e-15, atol=1e-16)
    w1 = np.zeros((2, 256))
    w1[:, 17] = 1.0
    got = orc.moments(v, 4, w1)
    for s in range(2):
        x, t = float(v[s, 17]), 1.0
        for q in range(1, 5):
            t = t * x
            assert got[s, q - 1] == t, (s, q)
