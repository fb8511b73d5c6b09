"""Pins of the oracle's linear advection case (Section 6): the coarse
generator with potential x/eps and diffusion 1/beta against the closed-form
advection-diffusion of a Gaussian, and parareal with the discretised
Fokker-Planck equation as both propagators (the exactness theorem on
densities; an advection error in the coarse model corrected by the
quantile iterator in one iteration, since the fine and coarse results then
differ by a translation)."""
import math

import numpy as np
import pytest


def _gauss_cdf(grid, m, s):
    e = grid.edges()
    c = np.array([0.5 * (1 + math.erf((v - m) / (s * math.sqrt(2)))) for v in e])
    c = (c - c[0]) / (c[-1] - c[0])
    return c


def _moments(grid, cdf):
    e = grid.edges()
    m = np.diff(cdf)
    xi = 0.5 * (e[:-1] + e[1:])
    mean = (m * xi).sum()
    var = (m * (xi - mean) ** 2).sum() + grid.h ** 2 / 12.0   # uniform within a bin
    return mean, var


@pytest.mark.parametrize("eps,beta", [(1.0, 1.0), (0.5, 2.0), (2.0, 0.5)])
def test_advection_diffusion_closed_form(orc, eps, beta):
    """dp/dt = d/dx(p/eps + (1/beta) dp/dx): a Gaussian N(m, s^2) moves to
    N(m - t/eps, s^2 + 2t/beta); second-order convergence in h."""
    model = orc.Model(kind=orc.MODEL_ADVECTION, eps=eps, beta=beta)
    m0, s0, t = 1.0, 0.6, 0.8
    errs = []
    for bins in (160, 320):
        g = orc.Grid(bins, -8.0, 8.0)
        P = orc.coarse_propagator(model, g, t)
        out = orc.coarse_apply(P, _gauss_cdf(g, m0, s0))[0]
        mean, var = _moments(g, out)
        errs.append(max(abs(mean - (m0 - t / eps)), abs(var - (s0 ** 2 + 2 * t / beta))))
    assert errs[1] < 5e-3
    assert errs[0] / errs[1] > 3.0   # second order (4 in the limit)


def test_advection_generator_structure(orc):
    g = orc.Grid(64, -4.0, 4.0)
    A = orc.coarse_generator(orc.Model(kind=orc.MODEL_ADVECTION, eps=0.7, beta=1.3), g)
    np.testing.assert_allclose(A.sum(axis=0), 0.0, atol=1e-10)      # mass conserved
    off = A - np.diag(np.diag(A))
    assert np.all(off >= 0) and np.count_nonzero(np.triu(off, 2)) == 0 and np.count_nonzero(np.tril(off, -2)) == 0
    # equilibrium: masses proportional to h rho_inf(centre) with rho_inf ~ exp(-beta x / eps)
    xi = 0.5 * (g.edges()[:-1] + g.edges()[1:])
    m = np.exp(-1.3 * xi / 0.7) * g.h
    assert np.max(np.abs(A @ m)) < 1e-9 * np.max(np.abs(A)) * m.max()


def _setup(orc, eps_c=1.0, beta_c=1.0):
    g = orc.Grid(288, -12.0, 6.0)
    fine = orc.Model(kind=orc.MODEL_ADVECTION, eps=1.0, beta=1.0)
    coarse = orc.Model(kind=orc.MODEL_ADVECTION, eps=eps_c, beta=beta_c)
    return g, fine, coarse, _gauss_cdf(g, 1.0, 0.5)


@pytest.mark.parametrize("iterator", [0, 1])
def test_fp_parareal_exactness(orc, iterator):
    g, fine, coarse, rho0 = _setup(orc, eps_c=0.6, beta_c=2.0)
    K, dT = 8, 0.2
    res = orc.fp_parareal(g, fine, coarse, rho0, K, dT, iters=K, iterator=iterator)
    ref = orc.fp_serial(g, fine, rho0, K, dT)
    for k in range(K + 1):
        for n in range(k + 1):
            np.testing.assert_array_equal(res[k][n], ref[n], err_msg=f"k={k} n={n}")


def test_quantile_iterator_corrects_an_advection_error(orc):
    g, fine, coarse, rho0 = _setup(orc, eps_c=0.5, beta_c=1.0)   # coarse advects twice as fast
    K, dT = 10, 0.2
    ref = orc.fp_serial(g, fine, rho0, K, dT)
    err = {}
    for it in (0, 1, 2, 3):
        res = orc.fp_parareal(g, fine, coarse, rho0, K, dT, iters=1, iterator=it)
        err[it] = [max(orc.w1(g, res[k][n], ref[n]) for n in range(K + 1)) for k in range(2)]
    e0 = err[0][0]
    assert e0 > 1.0                            # iteration 0: the coarse model is off by ~2 in position
    assert err[0][1] < 0.02 * e0               # one quantile correction removes the translation
    # for Gaussians of one variance a b / c is the Gaussian of mean
    # mu_a + mu_b - mu_c, the quantile result: the multiplicative iterator
    # corrects the translation as well
    assert err[2][1] < 0.02 * e0
    for it in (1, 3):                          # the additive and rotation iterators do not
        assert err[0][1] < 0.2 * err[it][1], (it, err)
