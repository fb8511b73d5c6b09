"""Pins of the oracle's coarse propagator (Section 2.2.2): finite volumes on
the detailed-balance form, zero flux at the ends, exact in time.

Closed forms used: mass conservation, the discrete equilibrium, the Neumann
heat kernel by the method of images (lambda = 1: pure diffusion), the
Ornstein-Uhlenbeck transition density (lambda < 1), second-order convergence
in h, and an eigendecomposition route to exp(A dT) independent of expm."""
import numpy as np
import pytest
from scipy.stats import norm


def _cell_masses(grid, cdf_fn):
    e = np.linspace(grid.lo, grid.hi, grid.bins + 1)
    return np.diff(cdf_fn(e))


@pytest.mark.parametrize("kind,lam,beta", [(0, 1.0, 1.0), (0, 0.5, 2.0), (1, 0.5, 3.0)])
def test_generator_conserves_mass_and_equilibrium(orc, kind, lam, beta):
    g = orc.Grid(96, -3.0, 3.0)
    model = orc.Model(kind=kind, lam=lam, beta=beta)
    A = orc.coarse_generator(model, g)
    assert np.max(np.abs(A.sum(axis=0))) < 1e-12 * np.max(np.abs(A))
    off = A - np.diag(np.diag(A))
    assert np.all(off >= 0.0)
    # discrete equilibrium m_c = h rho_inf(xi_c) with the Gibbs density of the
    # averaged SDE: rho_inf ~ exp(-beta Fbar), Fbar = (1-lam) x^2/2 (OU),
    # x^4/4 - (1-lam) x^2/2 (double well)
    xi = np.linspace(g.lo, g.hi, g.bins + 1)[:-1] + 0.5 * g.h
    fbar = 0.5 * (1 - lam) * xi ** 2 if kind == 0 else 0.25 * xi ** 4 - 0.5 * (1 - lam) * xi ** 2
    m_inf = np.exp(-beta * fbar)
    m_inf /= m_inf.sum()
    assert np.max(np.abs(A @ m_inf)) < 1e-12 * np.max(np.abs(A))
    P = orc.coarse_propagator(model, g, 0.1)
    np.testing.assert_allclose(P @ m_inf, m_inf, rtol=0, atol=1e-13)
    np.testing.assert_allclose(P.sum(axis=0), 1.0, rtol=0, atol=1e-12)
    assert P.min() > -1e-15


def test_expm_against_eigendecomposition(orc):
    """A is similar to a symmetric matrix under diag(sqrt(m_inf)).  The domain
    is kept where m_inf spans few decades, so the similarity transform does not
    amplify the eigensolver's rounding."""
    g = orc.Grid(64, -2.0, 2.0)
    model = orc.Model(kind=1, lam=0.5, beta=3.0)
    A = orc.coarse_generator(model, g)
    P = orc.coarse_propagator(model, g, 0.37)
    xi = np.linspace(g.lo, g.hi, 65)[:-1] + 0.5 * g.h
    assert np.allclose(np.diff(np.linspace(g.lo, g.hi, 65)), g.h)
    m_inf = np.exp(-3.0 * (0.25 * xi ** 4 - 0.25 * xi ** 2))
    s = np.sqrt(m_inf)
    S = (A * s[None, :]) / s[:, None]            # D^-1/2 A D^1/2
    np.testing.assert_allclose(S, S.T, rtol=0, atol=1e-10 * np.abs(A).max())
    w, V = np.linalg.eigh(0.5 * (S + S.T))
    Pe = (V * np.exp(w * 0.37)) @ V.T
    Pe = (Pe * s[:, None]) / s[None, :]
    np.testing.assert_allclose(P, Pe, rtol=0, atol=1e-12)


def _heat_error(orc, bins):
    g = orc.Grid(bins, -4.0, 4.0)
    model = orc.Model(kind=0, lam=1.0, beta=1.0)
    P = orc.coarse_propagator(model, g, 0.5)
    # initial density mirrored at the wall x = 4 (method of images, Neumann)
    c0 = lambda x: norm.cdf(x, 3.0, 0.5) + 1.0 - norm.cdf(8.0 - x, 3.0, 0.5)
    st = np.sqrt(0.25 + 2.0 * 0.5)
    ct = lambda x: norm.cdf(x, 3.0, st) + 1.0 - norm.cdf(8.0 - x, 3.0, st)
    m0 = _cell_masses(g, c0)
    cdf0 = np.concatenate([[0.0], np.cumsum(m0)]) / m0.sum()
    out = orc.coarse_apply(P, cdf0)[0]
    mt = _cell_masses(g, ct)
    exact = np.concatenate([[0.0], np.cumsum(mt)]) / mt.sum()
    return orc.w1(g, out, exact)


def test_pure_diffusion_neumann_heat_kernel(orc):
    e1, e2 = _heat_error(orc, 64), _heat_error(orc, 128)
    assert e1 < 2e-3
    assert 3.0 < e1 / e2 < 5.0          # second order in h


def _ou_error(orc, bins):
    g = orc.Grid(bins, -5.0, 5.0)
    lam, beta, t = 0.5, 2.0, 0.6
    model = orc.Model(kind=0, lam=lam, beta=beta)
    P = orc.coarse_propagator(model, g, t)
    theta, D = 1.0 - lam, 1.0 / beta
    mu0, s0 = 1.2, 0.4
    mu = mu0 * np.exp(-theta * t)
    var = s0 ** 2 * np.exp(-2 * theta * t) + D / theta * (1 - np.exp(-2 * theta * t))
    m0 = _cell_masses(g, lambda x: norm.cdf(x, mu0, s0))
    mt = _cell_masses(g, lambda x: norm.cdf(x, mu, np.sqrt(var)))
    cdf0 = np.concatenate([[0.0], np.cumsum(m0)]) / m0.sum()
    exact = np.concatenate([[0.0], np.cumsum(mt)]) / mt.sum()
    out = orc.coarse_apply(P, cdf0)[0]
    return orc.w1(g, out, exact)


def test_ou_transition_density(orc):
    e1, e2 = _ou_error(orc, 80), _ou_error(orc, 160)
    assert e1 < 2e-3
    assert 3.0 < e1 / e2 < 5.0


def test_coarse_apply_keeps_unit_mass(orc):
    g = orc.Grid(50, -3.0, 3.0)
    P = orc.coarse_propagator(orc.Model(kind=1, lam=0.5, beta=3.0), g, 0.2)
    rng = np.random.default_rng(1)
    m = rng.random(50)
    cdf = np.concatenate([[0.0], np.cumsum(m)]) / m.sum()
    cdf[-1] = 1.0
    out = orc.coarse_apply(P, cdf)[0]
    assert out[0] == 0.0 and out[-1] == 1.0 and np.all(np.diff(out) >= 0)
