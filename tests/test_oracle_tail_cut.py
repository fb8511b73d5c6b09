"""Pins of the oracle's tail cut in the coarse step (Section 2.2.2, with the
support ends q(0), q(1) of the quantile iterator, Section 4.4): bin masses of
P rho at or below TAIL_MASS = 1e-10 are set to 0 and the rest renormalised.

1. The rule itself on a hand-built case where P is a cyclic shift, so that
   P m has entries just above, exactly at and just below 1e-10, a negative
   one and ordinary ones: exactly those <= 1e-10 vanish, the others keep
   their ratios, and a transposed P or a threshold 10x off fails.
2. The threshold sits far above the rounding noise of the matrix
   exponential: an independent scaling-and-squaring Taylor exponential in
   extended precision differs from the oracle's by < 1e-14 per entry, and
   the set of bins the cut keeps is the same for both routes over several
   coarse steps of the workloads' grids.
3. The threshold sits far below anything the results depend on: moving it
   anywhere in [1e-12, 1e-9] changes the oracle's parareal macroscopic
   states by W1 <= 1e-4 (the GPU parity tolerance) on the plain OU workload
   and on a reduced double-well workload."""
import numpy as np
import pytest

import workloads


def _cdf(m):
    c = np.concatenate([[0.0], np.cumsum(m)])
    return c / c[-1]


def test_cut_drops_exactly_masses_at_or_below_threshold(orc):
    assert orc.TAIL_MASS == 1e-10
    I = 9
    # P m for the cyclic shift P[i+1, i] = 1 is m moved one bin to the right
    P = np.zeros((I, I))
    for i in range(I):
        P[(i + 1) % I, i] = 1.0
    # input masses at the start of the CDF, where its values carry them
    # exactly enough (the first is exactly 1e-10, and so is its image)
    m = np.array([1e-10, 1.0000001e-10, 0.99999e-10, 5e-10, -1e-16, 0.3, 0.2, 0.1, 0.4])
    cdf_in = np.concatenate([[0.0], np.cumsum(m)])
    pm = np.roll(np.diff(cdf_in), 1)
    assert pm[1] == 1e-10
    out = orc.coarse_apply(P, cdf_in)[0]
    keep = pm > 1e-10
    assert list(np.nonzero(keep)[0]) == [0, 2, 4, 6, 7, 8]
    expect = np.where(keep, pm, 0.0)
    expect /= expect.sum()
    got = np.diff(out)
    # CDF values are O(1), so masses read back from them carry ~1e-16 absolute rounding
    np.testing.assert_allclose(out, np.concatenate([[0.0], np.cumsum(expect)]), rtol=0, atol=1e-15)
    assert np.all(got[~keep] == 0.0) and np.all(got[keep] > 0.0)
    assert out[0] == 0.0 and out[-1] == 1.0
    # a transposed P (shift to the left) or a threshold 10x higher would differ
    assert not np.allclose(np.diff(orc.coarse_apply(P.T, cdf_in)[0]), expect)
    saved = orc.TAIL_MASS
    try:
        orc.TAIL_MASS = 1e-9
        assert np.diff(orc.coarse_apply(P, cdf_in)[0])[4] == 0.0   # 5e-10 would be lost
    finally:
        orc.TAIL_MASS = saved


def _expm_taylor_longdouble(A, t):
    """exp(A t) by scaling and squaring of a degree-19 Taylor polynomial in
    extended precision (numpy longdouble): a route independent of scipy's
    Pade approximant."""
    A = np.asarray(A, dtype=np.longdouble) * np.longdouble(t)
    nrm = float(np.abs(A).sum(axis=0).max())
    s = max(0, int(np.ceil(np.log2(nrm / 0.05))))
    B = A / np.longdouble(2.0) ** s
    E = np.eye(A.shape[0], dtype=np.longdouble)
    term = np.eye(A.shape[0], dtype=np.longdouble)
    for k in range(1, 20):
        term = term @ B / np.longdouble(k)
        E = E + term
    for _ in range(s):
        E = E @ E
    return E


@pytest.mark.parametrize("wname", ["ou", "double_well_128"])
def test_threshold_far_above_exponential_noise(orc, wname):
    if np.finfo(np.longdouble).eps > 1e-18:
        pytest.skip("longdouble is not an extended format on this machine")
    w = workloads.OU_SMALL if wname == "ou" else workloads.DOUBLE_WELL.scaled(N=1 << 14, bins=128)
    model = orc.Model(w.kind, w.fast_dim, w.lam, w.beta, w.eps, w.tau_x)
    grid = orc.Grid(w.bins, w.lo, w.hi)
    dT = w.steps * w.step_dt
    P = orc.coarse_propagator(model, grid, dT)
    Pl = _expm_taylor_longdouble(orc.coarse_generator(model, grid), dT)
    assert float(np.abs(P - Pl).max()) < 1e-14
    x0, _ = workloads.initial_ensemble(w)
    m = np.diff(orc.restrict(x0[None], grid)[1][0])
    for _ in range(4):
        a = P @ m
        b = (Pl @ m.astype(np.longdouble)).astype(np.float64)
        assert np.array_equal(a > orc.TAIL_MASS, b > orc.TAIL_MASS)
        assert np.abs(a - b).max() < 1e-14
        m = np.diff(orc.coarse_apply(P, _cdf(m))[0])


@pytest.mark.parametrize("wname", ["ou", "double_well_reduced"])
def test_results_insensitive_to_threshold(orc, wname):
    if wname == "ou":
        w, iters = workloads.OU_SMALL, 4
    else:   # 2^12 particles, 10 slices of 1000 steps, 512 bins on [-3, 3]
        w, iters = workloads.DOUBLE_WELL.scaled(N=1 << 12, K=10, T=1.0), 3
    model = orc.Model(w.kind, w.fast_dim, w.lam, w.beta, w.eps, w.tau_x)
    grid = orc.Grid(w.bins, w.lo, w.hi)
    x0, y0 = workloads.initial_ensemble(w)
    saved = orc.TAIL_MASS
    runs = {}
    try:
        for thr in (1e-12, 1e-10, 1e-9):
            orc.TAIL_MASS = thr
            runs[thr] = orc.parareal(model, grid, w.seed, x0, y0, w.K, w.steps, w.step_dt, iters=iters).rho
    finally:
        orc.TAIL_MASS = saved
    worst = max(orc.w1(grid, runs[1e-10][k][n], runs[thr][k][n])
                for thr in (1e-12, 1e-9) for k in range(iters + 1) for n in range(w.K + 1))
    assert worst <= 1e-4
