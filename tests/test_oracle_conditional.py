"""Pins of the oracle's matching that preserves the conditional distribution
(Section 5.2): reweighting with the relocation of unsupported target mass,
stratified resampling (Eq. stratified) and its deterministic variant, the
weighted restriction, and the parareal driver with these matchings.

Pinned against hand-computed cases (dyadic masses, exact in binary64), the
counting bounds that stratification fixes, brute-force weighted histograms,
an independent floating-point route (numpy cumsum + searchsorted), sample
means over many independent strata, and the exactness theorem."""
import numpy as np
import pytest


def _cdf(masses):
    return np.concatenate([[0.0], np.cumsum(np.asarray(masses, dtype=np.float64))])


@pytest.mark.parametrize("prior,target,expect", [
    # unsupported bin 1 splits 1/8 + 1/8 between bins 0 and 2; bin 4 has no
    # supported bin on its right, so all its mass goes to bin 3
    ([0.25, 0.0, 0.25, 0.5, 0.0], [0.5, 0.25, 0.0, 0.125, 0.125], [2.5, 0.0, 0.5, 0.5, 0.0]),
    # unsupported first bin: all of it to the right
    ([0.0, 0.5, 0.5], [0.5, 0.25, 0.25], [0.0, 1.5, 0.5]),
    # a run of unsupported bins, each split between the two ends of the run
    ([0.5, 0.0, 0.0, 0.5], [0.25, 0.25, 0.25, 0.25], [1.0, 0.0, 0.0, 1.0]),
    # target lighter than prior everywhere supported, nothing to move
    ([0.5, 0.25, 0.25], [0.25, 0.25, 0.5], [0.5, 1.0, 2.0]),
])
def test_reweight_factors_hand_computed(orc, prior, target, expect):
    g = orc.Grid(len(prior), 0.0, float(len(prior)))
    r = orc.reweight_factors(g, _cdf(prior), _cdf(target))
    np.testing.assert_array_equal(r, np.array(expect))


def _rand_ensemble_and_target(orc, g, rng, n):
    x = rng.normal(0.3, 0.6, n)
    _, cp = orc.restrict(x[None], g)
    m = rng.gamma(2.0, 1.0, g.bins) * (rng.random(g.bins) < 0.8)
    m /= m.sum()
    return x, cp[0], _cdf(m)


def test_reweighted_ensemble_restricts_to_the_relocated_target(orc):
    g = orc.Grid(40, -3.0, 3.0)
    rng = np.random.default_rng(1)
    n = 5000
    x, cp, ct = _rand_ensemble_and_target(orc, g, rng, n)
    w = orc.reweight(x[None], g, cp[None], ct[None])[0]
    # brute-force weighted histogram
    bins = np.array([orc.lib().or_bin(v, g.bins, g.lo, g.hi) for v in x])
    hist = np.bincount(bins, weights=w, minlength=g.bins)
    rb = np.diff(cp)
    rt = np.diff(ct)
    r = orc.reweight_factors(g, cp, ct)
    rho_new = r * rb
    np.testing.assert_allclose(hist, rho_new, rtol=0, atol=1e-13)
    # mass is conserved and lands only where the prior has particles
    assert abs(w.sum() - 1.0) < 1e-12
    assert abs(rho_new.sum() - rt.sum()) < 1e-13
    assert np.all(rho_new[rb == 0] == 0)
    # supported bins keep their own target mass at least
    assert np.all(rho_new[rb > 0] >= rt[rb > 0] - 1e-15)


def test_strong_projection_reweight(orc):
    g = orc.Grid(32, -2.0, 2.0)
    rng = np.random.default_rng(2)
    x = rng.normal(0.0, 0.7, 3001)
    _, cp = orc.restrict(x[None], g)
    w = orc.reweight(x[None], g, cp, cp)[0]
    assert np.all(w == 1.0 / 3001)
    wbar = rng.random(3001)
    w2 = orc.reweight(x[None], g, cp, cp, wbar[None])[0]
    np.testing.assert_array_equal(w2, wbar)


@pytest.mark.parametrize("n", [1, 2, 7, 1000, 4099])
@pytest.mark.parametrize("mode", [0, 1])
def test_resample_equal_weights_is_the_identity(orc, n, mode):
    w = np.full((3, n), 1.0 / n)
    idx = orc.resample(w, mode, seed=5, slice_begin=11)
    for s in range(3):
        np.testing.assert_array_equal(idx[s], np.arange(n))


def _lengths(orc, w):
    W = np.array([orc.weight_fixed(v) for v in w], dtype=object)
    T = sum(W)
    return np.array([float(v) * len(w) / float(T) for v in W])


def test_deterministic_counts_are_floor_or_ceil(orc):
    rng = np.random.default_rng(3)
    for n in (5, 64, 999):
        w = rng.gamma(0.7, 1.0, n) * (rng.random(n) < 0.7)
        w /= w.sum()
        idx = orc.resample(w[None], 1, seed=0, slice_begin=0)[0]
        assert np.all(np.diff(idx.astype(np.int64)) >= 0)
        counts = np.bincount(idx, minlength=n)
        assert counts.sum() == n
        ell = _lengths(orc, w)
        # equally spaced points, one per stratum: an interval of length l holds
        # floor(l) or ceil(l) of them
        assert np.all(counts >= np.floor(ell - 1e-9)) and np.all(counts <= np.ceil(ell + 1e-9))
        assert np.all(counts[w == 0] == 0)


def test_stratified_counts_bounds_and_unbiased(orc):
    rng = np.random.default_rng(4)
    n = 50
    w = rng.gamma(0.8, 1.0, n)
    w /= w.sum()
    ell = _lengths(orc, w)
    reps = 400
    idx = orc.resample(np.tile(w, (reps, 1)), 0, seed=9, slice_begin=100)
    counts = np.stack([np.bincount(idx[s], minlength=n) for s in range(reps)])
    assert np.all(counts.sum(axis=1) == n)
    # one point per stratum: an interval of length l holds between floor(l) - 1
    # and ceil(l) + 1 of them
    assert np.all(counts >= np.floor(ell) - 1) and np.all(counts <= np.ceil(ell) + 1)
    # unbiased: E[n_p] = N W_p / T; the count of a point of a stratum is Bernoulli
    mean = counts.mean(axis=0)
    assert np.all(np.abs(mean - ell) <= 5 * 0.5 / np.sqrt(reps) + 1e-9)
    # different slices draw different points
    assert len({tuple(c) for c in counts}) > 10


def test_resample_agrees_with_a_floating_point_route(orc):
    rng = np.random.default_rng(6)
    n = 20000
    w = rng.random(n) ** 3
    w /= w.sum()
    idx = orc.resample(w[None], 1, seed=0, slice_begin=0)[0]
    C = np.cumsum(w)
    u = (np.arange(n) + 0.5) / n * C[-1]
    ref = np.searchsorted(C, u, side="right")
    # the routes differ only where a point falls within rounding of a boundary
    diff = idx.astype(np.int64) != ref
    if diff.any():
        close = np.min(np.abs(C[np.minimum(ref[diff], n - 1)] - u[diff]))
        assert close < 1e-12
    assert diff.mean() < 1e-3


def test_restrict_weighted_brute_force(orc):
    g = orc.Grid(25, -1.0, 1.5)
    rng = np.random.default_rng(7)
    x = rng.normal(0.2, 0.5, (2, 3000))
    x[0, :5] = [-9.0, 9.0, -1.0, 1.5, 0.1]
    w = rng.random((2, 3000))
    w /= w.sum(axis=1, keepdims=True)      # probability weights (the fixed point holds totals < 8)
    cdf = orc.restrict_weighted(x, w, g)
    for s in range(2):
        bins = np.array([orc.lib().or_bin(v, g.bins, g.lo, g.hi) for v in x[s]])
        h = np.bincount(bins, weights=w[s], minlength=g.bins)
        ref = np.concatenate([[0.0], np.cumsum(h) / h.sum()])
        np.testing.assert_allclose(cdf[s], ref, rtol=0, atol=1e-14)
        assert cdf[s][0] == 0.0 and cdf[s][-1] == 1.0
    # uniform weights: the counting CDF up to rounding
    u = np.full_like(w, 1.0 / 3000)
    _, c2 = orc.restrict(x, g)
    np.testing.assert_allclose(orc.restrict_weighted(x, u, g), c2, rtol=0, atol=1e-15)


@pytest.mark.parametrize("matching", ["resample", "resample_det", "reweight"])
def test_exactness_theorem_conditional_matchings(orc, matching):
    model = orc.Model(kind=1, lam=0.5, beta=3.0, eps=0.05)
    grid = orc.Grid(48, -3.0, 3.0)
    rng = np.random.default_rng(8)
    N, K, S, dt = 600, 5, 7, 2e-3
    x0 = rng.normal(-0.5, 0.3, N)
    y0 = x0[None] + rng.normal(0, 0.5, (1, N))
    res = orc.parareal(model, grid, 0, x0, y0, K, S, dt, iters=K, matching=matching)
    xs, ys = orc.serial_fine(model, 0, x0, y0, K, S, dt)
    for k in range(K + 1):
        for n in range(k + 1):
            assert np.array_equal(res.x[k][n], xs[n]), (k, n)
            assert np.array_equal(res.y[k][n], ys[n]), (k, n)
            assert np.all(res.w[k][n] == 1.0 / N), (k, n)


@pytest.mark.parametrize("matching", ["resample", "resample_det"])
def test_resampled_pairs_are_prior_pairs(orc, matching):
    """The matching moves no particle: every output (x, y) is a prior pair,
    so the conditional law of y given x is the prior's; the restriction of the
    output follows the target up to the sampling error."""
    g = orc.Grid(30, -3.0, 3.0)
    rng = np.random.default_rng(10)
    n = 20000
    x = rng.normal(-0.2, 0.7, n)
    y = (2.0 * x + rng.normal(0, 0.1, n))[None]
    _, cp = orc.restrict(x[None], g)
    _, ct = orc.restrict(rng.normal(0.3, 0.6, n)[None], g)
    xs, ys, w = orc._conditional_match(g, x[None], y[None], cp, ct, matching, 3, 0, 1)
    assert w is None
    pairs = set(zip(x.tolist(), y[0].tolist()))
    assert all(p in pairs for p in zip(xs[0].tolist(), ys[0][0].tolist()))
    _, c_out = orc.restrict(xs, g)
    r = orc.reweight_factors(g, cp[0], ct[0])
    target = np.concatenate([[0.0], np.cumsum(r * np.diff(cp[0]))])
    assert orc.w1(g, c_out[0], target) < 2e-3
    # the conditional slope of y on x is the prior's 2.0, not the one a move of x alone would give
    slope = np.polyfit(xs[0], ys[0][0], 1)[0]
    assert abs(slope - 2.0) < 0.02


def test_target_outside_the_prior_support(orc):
    """All target mass left of the prior's support lands in the prior's first
    supported bin, all of it right of the support in its last: the factors are
    then 1/rhobar there and 0 elsewhere (dyadic masses, exact)."""
    g = orc.Grid(8, 0.0, 8.0)
    prior = [0.0, 0.0, 0.0, 0.25, 0.5, 0.25, 0.0, 0.0]
    left = [0.5, 0.25, 0.25, 0.0, 0.0, 0.0, 0.0, 0.0]
    right = [0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.5, 0.5]
    np.testing.assert_array_equal(orc.reweight_factors(g, _cdf(prior), _cdf(left)),
                                  [0, 0, 0, 4.0, 0, 0, 0, 0])
    np.testing.assert_array_equal(orc.reweight_factors(g, _cdf(prior), _cdf(right)),
                                  [0, 0, 0, 0, 0, 4.0, 0, 0])
    # the reweighted ensemble puts all its weight into that one bin
    x = np.array([3.5] * 4 + [4.5] * 8 + [5.5] * 4)
    w = orc.reweight(x[None], g, _cdf(prior)[None], _cdf(left)[None])[0]
    np.testing.assert_array_equal(w, [0.25] * 4 + [0.0] * 12)


@pytest.mark.parametrize("mode", [0, 1])
def test_resample_without_weight_is_the_identity(orc, mode):
    """A slice whose weights are all zero (T = 0) keeps its particles; the
    other slices are unaffected."""
    rng = np.random.default_rng(8)
    w = rng.random((3, 257))
    w /= w.sum(axis=1, keepdims=True)
    w[1] = 0.0
    idx = orc.resample(w, mode, seed=3, slice_begin=2)
    np.testing.assert_array_equal(idx[1], np.arange(257))
    ref = orc.resample(w[[0, 2]], mode, seed=3, slice_begin=2)
    np.testing.assert_array_equal(idx[0], ref[0])


def test_weight_fixed_rounds_to_nearest_even(orc):
    """The fixed point against exact rational arithmetic (ties to even)."""
    from _fixed_point import crafted_weights, fixed_exact
    for w in list(crafted_weights()) + [1.0, 0.5, 0.75, 1.0 / 3.0, 2.0 ** -61, 3.9]:
        assert orc.weight_fixed(w) == fixed_exact(w), w
    assert [orc.weight_fixed((2 * k + 1) * 2.0 ** -62) for k in range(4)] == [0, 2, 2, 4]
