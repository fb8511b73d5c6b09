"""Pins of the oracle's restriction (Eq. binning, Eq. discr_cdf) and of the
matching by quantile transport (Section 5.1, Eq. transformation)."""
from fractions import Fraction

import numpy as np
import pytest


def test_edges_exact_on_dyadic_grid(orc):
    g = orc.Grid(512, -3.0, 3.0)
    e = g.edges()
    for i in range(513):
        assert Fraction(e[i]) == Fraction(-3) + Fraction(i) * Fraction(6, 512)


@pytest.mark.parametrize("bins,lo,hi", [(256, -4.0, 4.0), (7, -1.0, 2.5), (512, -3.0, 3.0)])
def test_restrict_bruteforce(orc, bins, lo, hi):
    g = orc.Grid(bins, lo, hi)
    rng = np.random.default_rng(bins)
    e = g.edges()
    x = np.concatenate([rng.normal(0.3, 1.5, 3000), e[rng.integers(0, bins + 1, 200)],
                        [lo - 10, hi + 10, lo, hi, np.nextafter(hi, 0), np.nextafter(lo, -9)]])
    counts, cdf = orc.restrict(x[None], g)
    ref = np.clip(np.searchsorted(e, x, side="right") - 1, 0, bins - 1)
    np.testing.assert_array_equal(counts[0], np.bincount(ref, minlength=bins))
    assert counts.sum() == x.size
    # the PL CDF is exact at the edges: C_i = #{x < e_i} / N (Section 4.4)
    xs = np.sort(x)
    for i in range(1, bins):
        assert cdf[0, i] == np.searchsorted(xs, e[i], side="left") / x.size
    assert cdf[0, 0] == 0.0 and cdf[0, bins] == 1.0


def test_edge_point_goes_right(orc):
    g = orc.Grid(4, 0.0, 4.0)
    assert orc.bin_index(1.0, g) == 1
    assert orc.bin_index(np.nextafter(1.0, 0.0), g) == 0
    assert orc.bin_index(4.0, g) == 3
    assert orc.bin_index(-1e300, g) == 0


def test_match_hand_computed(orc):
    g = orc.Grid(2, 0.0, 2.0)
    prior = np.array([[0.0, 0.5, 1.0]])
    target = np.array([[0.0, 0.25, 1.0]])
    x = np.array([[0.5, 1.5, -1.0, 3.0]])
    out = orc.match(x, g, prior, target)
    np.testing.assert_allclose(out[0], [1.0, 1.0 + 2.0 / 3.0, -1.0, 3.0], rtol=0, atol=1e-15)
    empty_first = np.array([[0.0, 0.0, 1.0]])
    out = orc.match(np.array([[0.5, -1.0]]), g, prior, empty_first)
    np.testing.assert_allclose(out[0], [1.25, 0.0], rtol=0, atol=1e-15)


def test_strong_projection_exact(orc):
    """M(R X, X) = X bit for bit (Eq. projection)."""
    g = orc.Grid(64, -2.0, 2.0)
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.normal(0, 0.7, (3, 5000)), rng.uniform(-4, 4, (3, 50))], axis=1)
    _, cdf = orc.restrict(x, g)
    out = orc.match(x, g, cdf, cdf)
    assert np.array_equal(out, x)


def test_match_monotone_and_consistent(orc):
    g = orc.Grid(100, -4.0, 4.0)
    rng = np.random.default_rng(4)
    N = 20000
    xbar = rng.normal(-0.5, 0.9, N)
    _, cp = orc.restrict(xbar[None], g)
    target_samples = rng.gamma(3.0, 0.5, 50000) - 1.0
    _, ct = orc.restrict(target_samples[None], g)
    out = orc.match(xbar[None], g, cp, ct)[0]
    order = np.argsort(xbar)
    assert np.all(np.diff(out[order]) >= 0)
    _, cnew = orc.restrict(out[None], g)
    rho_bar = np.diff(cp[0])
    bound = (g.hi - g.lo) * (rho_bar.max() + 1.0 / N)
    w = orc.w1(g, cnew[0], ct[0])
    assert w <= bound
    assert np.max(np.abs(cnew[0] - ct[0])) <= rho_bar.max() + 1.0 / N


def test_match_gaussian_affine(orc):
    """Gaussian prior to Gaussian target is the affine map mu + s (x - mubar)/sbar."""
    from scipy.stats import norm
    g = orc.Grid(400, -5.0, 5.0)
    rng = np.random.default_rng(8)
    xbar = rng.normal(0.0, 1.0, 200000)
    _, cp = orc.restrict(xbar[None], g)
    e = g.edges()
    ct = norm.cdf(e, 0.5, 0.8)
    ct = (ct - ct[0]) / (ct[-1] - ct[0])
    ct[0], ct[-1] = 0.0, 1.0
    out = orc.match(xbar[None], g, cp, ct[None])[0]
    sel = np.abs(xbar) < 2.5
    err = np.abs(out[sel] - (0.5 + 0.8 * xbar[sel]))
    assert err.max() < 0.03
    assert err.mean() < 0.005
