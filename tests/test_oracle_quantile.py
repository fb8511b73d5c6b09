"""Pins of the oracle's iterators (Section 4), above all the quantile
iterator J_q of Section 4.4, and of the W1 distance used for tolerances."""
import numpy as np
import pytest


def _random_cdf(rng, bins, empty_frac=0.3):
    m = rng.gamma(0.7, 1.0, bins)
    m[rng.random(bins) < empty_frac] = 0.0
    m[rng.integers(0, bins)] += 0.5
    counts = np.round(m / m.sum() * 4096).astype(np.int64)
    if counts.sum() == 0:
        counts[0] = 1
    c = np.concatenate([[0], np.cumsum(counts)]) / counts.sum()
    c[-1] = 1.0
    return c


def _gauss_cdf(g, mu, s):
    from scipy.stats import norm
    c = norm.cdf(g.edges(), mu, s)
    c = (c - c[0]) / (c[-1] - c[0])
    c[0], c[-1] = 0.0, 1.0
    return c


@pytest.mark.parametrize("seed", range(6))
def test_iterator_property_exact(orc, seed):
    """J(a, b, a) = b bit for bit in two-sided mode (Eq. iterator_property)."""
    rng = np.random.default_rng(seed)
    bins = int(rng.integers(3, 200))
    g = orc.Grid(bins, -4.0, 4.0)
    a = _random_cdf(rng, bins)
    b = _random_cdf(rng, bins)
    out = orc.iterate(g, a, b, a, orc.ITER_QUANTILE, orc.QMODE_TWO_SIDED)
    assert np.array_equal(out, b)


def test_midpoint_mode_breaks_property_on_empty_bin(orc):
    """The paper's midpoint rule for flat levels maps [1/2, 0, 1/2] to
    [1/3, 1/3, 1/3] when a = c (hand computation: knots (0,0), (1.5,1/2), (3,1))."""
    g = orc.Grid(3, 0.0, 3.0)
    b = np.array([0.0, 0.5, 0.5, 1.0])
    mid = orc.iterate(g, b, b, b, orc.ITER_QUANTILE, orc.QMODE_MIDPOINT)
    np.testing.assert_allclose(mid, [0.0, 1 / 3, 2 / 3, 1.0], rtol=0, atol=1e-15)
    two = orc.iterate(g, b, b, b, orc.ITER_QUANTILE, orc.QMODE_TWO_SIDED)
    assert np.array_equal(two, b)


@pytest.mark.parametrize("mode", [0, 1])
def test_positive_unit_mass(orc, mode):
    rng = np.random.default_rng(10 + mode)
    for _ in range(20):
        bins = int(rng.integers(3, 100))
        g = orc.Grid(bins, -2.0, 3.0)
        a, b, c = (_random_cdf(rng, bins) for _ in range(3))
        out = orc.iterate(g, a, b, c, orc.ITER_QUANTILE, mode)
        assert out[0] == 0.0 and out[-1] == 1.0
        assert np.all(np.diff(out) >= 0.0)


def test_gaussian_quantile_arithmetic(orc):
    """q of N(mu, s) is mu + s Phi^{-1}(p), so J_q of three Gaussians is
    N(mu_a + mu_b - mu_c, s_a + s_b - s_c) up to the O(h) binning error."""
    g = orc.Grid(600, -6.0, 6.0)
    a = _gauss_cdf(g, 0.4, 0.9)
    b = _gauss_cdf(g, -0.3, 0.7)
    c = _gauss_cdf(g, 0.1, 0.8)
    out = orc.iterate(g, a, b, c)
    expect = _gauss_cdf(g, 0.4 - 0.3 - 0.1, 0.9 + 0.7 - 0.8)
    assert orc.w1(g, out, expect) < 2e-3
    # a transposed operand (b and c swapped) lands far away
    wrong = orc.iterate(g, a, c, b)
    assert orc.w1(g, wrong, expect) > 0.1


def test_pure_advection_is_corrected(orc):
    """a(x) = c(x - s) with s a multiple of h shifts b by s (Section 6.3)."""
    g = orc.Grid(128, -4.0, 4.0)
    k = 10
    c = _gauss_cdf(g, -0.5, 0.5)
    a = np.concatenate([np.zeros(k), c[:-k]])
    b = _gauss_cdf(g, -0.8, 0.4)
    out = orc.iterate(g, a, b, c)
    expect = np.concatenate([np.zeros(k), b[:-k]])
    np.testing.assert_allclose(out[:-1], expect[:-1], rtol=0, atol=1e-12)


def test_monotone_fix_hand_computed(orc):
    """Grid [0,4] with 4 bins, all mass in bins 1-2:
    a = [0,0,.5,1,1], b = [0,0,.9,1,1], c = [0,0,.1,1,1].  Levels {0,.1,.5,.9,1}.
    Two-sided knots (q~ = qb + (qa - qc)):
      p=0 : q+ = 1 for all              -> (1, 0)
      p=.1: 1+.1/.9 + (1.2 - 2)         -> (0.3111.., .1) twice
      p=.5: 1+.5/.9 + (2 - (2+.4/.9))   -> (1.1111.., .5) twice
      p=.9: 2 + (2.8 - (2+.8/.9))       -> (1.9111.., .9) twice
      p=1 : q- = 3 for all              -> (3, 1)
    Pool-adjacent-violators pools the first three knots at (1 + 2*0.3111..)/3;
    the PL CDF through the knots is then read at the edges 1, 2, 3."""
    g = orc.Grid(4, 0.0, 4.0)
    a = np.array([0.0, 0.0, 0.5, 1.0, 1.0])
    b = np.array([0.0, 0.0, 0.9, 1.0, 1.0])
    c = np.array([0.0, 0.0, 0.1, 1.0, 1.0])
    out = orc.iterate(g, a, b, c)
    q1 = 1.0 + 0.1 / 0.9 + (1.2 - 2.0)
    q5 = 1.0 + 0.5 / 0.9 + (2.0 - (2.0 + 0.4 / 0.9))
    q9 = 2.0 + (2.8 - (2.0 + 0.8 / 0.9))
    pooled = (1.0 + 2.0 * q1) / 3.0
    at1 = 0.1 + (1.0 - pooled) / (q5 - pooled) * 0.4
    at2 = 0.9 + (2.0 - q9) / (3.0 - q9) * 0.1
    np.testing.assert_allclose(out, [0.0, at1, at2, 1.0, 1.0], rtol=0, atol=1e-14)


@pytest.mark.parametrize("it", [1, 2, 3])
def test_other_iterators(orc, it):
    rng = np.random.default_rng(it)
    g = orc.Grid(40, 0.0, 1.0)
    # a has full support, so that b is supported by a (needed by J_mult)
    a = 0.5 * (_random_cdf(rng, 40, 0.0) + np.linspace(0.0, 1.0, 41))
    b = _random_cdf(rng, 40, 0.1)
    out = orc.iterate(g, a, b, a, it)
    np.testing.assert_allclose(out, b, rtol=0, atol=1e-13)
    c = _random_cdf(rng, 40, 0.0)
    out = orc.iterate(g, a, b, c, it)
    assert out[0] == 0.0 and out[-1] == 1.0 and np.all(np.diff(out) >= 0)


def test_additive_hand_computed(orc):
    g = orc.Grid(3, 0.0, 3.0)
    cdf = lambda m: np.concatenate([[0.0], np.cumsum(m)])
    a, b, c = cdf([0.2, 0.3, 0.5]), cdf([0.5, 0.5, 0.0]), cdf([0.1, 0.1, 0.8])
    # a + b - c = [0.6, 0.7, -0.3] -> [0.6, 0.7, 0] / 1.3
    out = orc.iterate(g, a, b, c, orc.ITER_ADD)
    np.testing.assert_allclose(out, [0, 0.6 / 1.3, 1.0, 1.0], atol=1e-15)
    # a b / c = [1.0, 1.5, 0] / 2.5
    out = orc.iterate(g, a, b, c, orc.ITER_MULT)
    np.testing.assert_allclose(out, [0, 0.4, 1.0, 1.0], atol=1e-15)


def test_multiplicative_without_common_support_keeps_b(orc):
    """a b / c vanishes on every bin when b's mass sits where a or c has
    none: there is no mass to rescale and the update keeps b (the
    correction is dropped), bit for bit."""
    g = orc.Grid(4, 0.0, 4.0)
    cdf = lambda m: np.concatenate([[0.0], np.cumsum(m)])
    a, b, c = cdf([0.5, 0.5, 0.0, 0.0]), cdf([0.0, 0.0, 0.25, 0.75]), cdf([0.25, 0.25, 0.25, 0.25])
    np.testing.assert_array_equal(orc.iterate(g, a, b, c, orc.ITER_MULT), b)
    # a single common bin is enough to normalise: all mass goes there
    b2 = cdf([0.0, 0.5, 0.5, 0.0])
    np.testing.assert_allclose(orc.iterate(g, a, b2, c, orc.ITER_MULT), cdf([0.0, 1.0, 0.0, 0.0]), atol=0)


def test_rotation_is_a_rotation(orc):
    """sqrt of the result has unit L2 norm and the map sends sqrt(c) to sqrt(a)
    (Section 4.3): the inner product with sqrt(a) equals that of b with c."""
    rng = np.random.default_rng(5)
    g = orc.Grid(30, 0.0, 1.0)
    # a close to c and b of full support keep the rotated sqrt(b) non-negative,
    # so that squaring does not fold any component
    lin = np.linspace(0.0, 1.0, 31)
    c = 0.5 * (_random_cdf(rng, 30, 0.0) + lin)
    a = 0.9 * c + 0.1 * lin
    b = 0.5 * (_random_cdf(rng, 30, 0.0) + lin)
    out = orc.iterate(g, a, b, c, orc.ITER_ROT)
    ma, mb, mc, mo = (np.diff(v) for v in (a, b, c, out))
    assert abs(mo.sum() - 1.0) < 1e-14
    # a rotation preserves the inner product: <sqrt(out), sqrt(a)> = <sqrt(b), sqrt(c)>
    np.testing.assert_allclose(np.sqrt(mo) @ np.sqrt(ma), np.sqrt(mb) @ np.sqrt(mc), atol=1e-12)


def test_w1_pins(orc):
    g = orc.Grid(50, -2.0, 3.0)
    rng = np.random.default_rng(9)
    c1 = _random_cdf(rng, 50, 0.0)
    assert orc.w1(g, c1, c1) == 0.0
    # translation of a distribution that stays inside the domain moves W1 by the shift
    m = np.zeros(50)
    m[10:20] = rng.random(10)
    m /= m.sum()
    c_a = np.concatenate([[0.0], np.cumsum(m)])
    c_b = np.concatenate([[0.0] * 7, c_a[:-7]])
    assert abs(orc.w1(g, c_a, c_b) - 7 * g.h) < 1e-13
    # against a fine quadrature of |C1 - C2| for crossing CDFs
    c2 = _random_cdf(rng, 50, 0.0)
    xs = np.linspace(g.lo, g.hi, 2_000_001)
    e = g.edges()
    quad = np.trapezoid(np.abs(np.interp(xs, e, c1) - np.interp(xs, e, c2)), xs)
    assert abs(orc.w1(g, c1, c2) - quad) < 1e-9
