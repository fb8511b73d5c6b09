"""Pins of the oracle's chemically reacting system (Section 2.1.2, Eqs.
F_Bruna, G_Bruna, D, E_Bruna; coarse model of Section 2.2.3).

* The drifts and diffusions against sources independent of the oracle's C:
  symbolic derivatives (sympy) of the potentials exactly as printed, and the
  net rates and total propensities of the reaction network
  0 -> Y (k0), Y -> 0 (k1 y), 2Y -> 3Y (k2 y(y-1)), 3Y -> 2Y (k3 y(y-1)(y-2)),
  Y -> Y + X (k4 y), X -> 0 (k5 x), assembled from a stoichiometry table.
* One Euler-Maruyama step from a fixed point: sample mean and variance of
  2^16 particles within 5 standard errors of the closed form.
* With k2 = k3 = 0 both drifts are linear and the squared diffusions affine,
  so the EM mean and variance recursions are exact for the scheme; 300 steps
  of 2^15 particles sit within 5 standard errors of them.
* The mean ybar of the fast equilibrium: with k2 = k3 = 0 the density is a
  shifted Gamma, (k0 + k1 y)^(4 k0/k1 - 1) exp(-2y), whose mean is known; for
  the workload's rates the trapezoidal ybar agrees with adaptive quadrature.
* The readings: the workload's k3 makes the fast drift bistable with both
  wells and the saddle inside [0, 600]; the printed k3 gives one root far
  outside.
* log rho_inf against quadrature of its defining integral; generator mass
  conservation and its discrete equilibrium; the exactness theorem of the
  parareal driver on the chemical system."""
import math

import numpy as np
import pytest

import workloads

K_DEF = workloads.CHEM_RATES
K_PRINTED = workloads.CHEM_RATES_PRINTED


def _model(orc, kind=4, rates=K_DEF, eps=2.5e-2, tau_x=25.0):
    return orc.Model(kind, 1, eps=eps, tau_x=tau_x, rates=tuple(rates))


def _network(k, x, y):
    """Net rates (dX/dt, dY/dt) and total propensities (for X, for Y)."""
    reactions = [  # (change of X, change of Y, propensity)
        (0, +1, k[0]), (0, -1, k[1] * y), (0, +1, k[2] * y * (y - 1)), (0, -1, k[3] * y * (y - 1) * (y - 2)),
        (+1, 0, k[4] * y), (-1, 0, k[5] * x)]
    net_x = sum(dx * a for dx, _, a in reactions)
    net_y = sum(dy * a for _, dy, a in reactions)
    tot_x = sum(abs(dx) * a for dx, _, a in reactions)
    tot_y = sum(abs(dy) * a for _, dy, a in reactions)
    return net_x, net_y, tot_x, tot_y


@pytest.mark.parametrize("x,y", [(100.0, 105.0), (37.5, 412.25), (0.0, 0.0), (600.0, 3.0)])
def test_coefficients_against_potentials_and_network(orc, x, y):
    sp = pytest.importorskip("sympy")
    X, Y = sp.symbols("x y")
    k = [sp.Float(v, 30) for v in K_DEF]
    F = -k[4] * X * Y - sp.Rational(1, 2) * k[5] * X ** 2                      # as printed
    G = (-k[0] * Y - sp.Rational(1, 2) * k[1] * Y ** 2 + k[2] * Y ** 2 * (Y / 3 - sp.Rational(1, 2))
         - k[3] * Y ** 2 * (sp.Rational(1, 2) * Y - 1) ** 2)
    sub = {X: x, Y: y}
    dF, dG = float(sp.diff(F, X).subs(sub)), float(sp.diff(G, Y).subs(sub))
    net_x, net_y, tot_x, tot_y = _network(K_DEF, x, y)
    printed = orc.chem_coefficients(_model(orc, kind=5), x, y)
    langevin = orc.chem_coefficients(_model(orc, kind=4), x, y)
    scale = 1.0 + abs(tot_y)
    np.testing.assert_allclose(printed[:2], [dF, dG], rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(langevin[:2], [-net_x, -net_y], rtol=0, atol=1e-12 * scale)
    # 2D and 2E are the total propensities (the same in both readings)
    for c in (printed, langevin):
        np.testing.assert_allclose([2 * c[2], 2 * c[3]], [tot_x, tot_y], rtol=1e-14, atol=1e-12)


@pytest.mark.parametrize("kind", [4, 5])
def test_one_em_step_moments(orc, kind):
    n, dt, x0, y0 = 1 << 16, 1e-3, 120.0, 300.0
    m = _model(orc, kind)
    x = np.full((1, n), x0)
    y = np.full((1, 1, n), y0)
    xs, ys = orc.fine_propagate(m, 5, x, y, 3, 1, dt)
    net_x, net_y, tot_x, tot_y = _network(K_DEF, x0, y0)
    if kind == 5:   # drifts of the printed potentials
        net_x, net_y = K_DEF[4] * y0 + K_DEF[5] * x0, -orc.chem_coefficients(m, x0, y0)[1]
    for v, mean, var in ((xs[0], x0 + net_x / m.tau_x * dt, tot_x / m.tau_x * dt),
                         (ys[0, 0], y0 + net_y / m.eps * dt, tot_y / m.eps * dt)):
        assert abs(v.mean() - mean) < 5 * math.sqrt(var / n)
        assert abs(v.var() - var) < 5 * var * math.sqrt(2.0 / n)


def test_linear_case_exact_moment_recursion(orc):
    """k2 = k3 = 0: dX = (k4 Y - k5 X)/tau dt + ..., dY = (k0 - k1 Y)/eps dt + ...;
    the means and the second moments follow linear recursions exactly."""
    k = (60.0, 1.0, 0.0, 0.0, 0.833, 1.0)
    eps, tau, dt, n, steps = 0.05, 2.0, 1e-3, 1 << 15, 300
    m = _model(orc, 4, k, eps=eps, tau_x=tau)
    mx, my = 100.0, 40.0
    x = np.full((1, n), mx)
    y = np.full((1, 1, n), my)
    xs, ys = orc.fine_propagate(m, 9, x, y, 0, steps, dt)
    a, b = dt / tau, dt / eps
    vxx = vyy = vxy = 0.0
    for _ in range(steps):
        # (X', Y') = M (X, Y) + c + noise, noise variances (k4 Y + k5 X) a and (k0 + k1 Y) b
        nx = (1 - k[5] * a) * mx + k[4] * a * my
        ny = (1 - k[1] * b) * my + k[0] * b
        qxx = (1 - k[5] * a) ** 2 * vxx + 2 * (1 - k[5] * a) * k[4] * a * vxy + (k[4] * a) ** 2 * vyy
        qxx += (k[4] * my + k[5] * mx) * a
        qyy = (1 - k[1] * b) ** 2 * vyy + (k[0] + k[1] * my) * b
        qxy = (1 - k[5] * a) * (1 - k[1] * b) * vxy + k[4] * a * (1 - k[1] * b) * vyy
        mx, my, vxx, vyy, vxy = nx, ny, qxx, qyy, qxy
    X, Y = xs[0], ys[0, 0]
    assert abs(X.mean() - mx) < 5 * math.sqrt(vxx / n)
    assert abs(Y.mean() - my) < 5 * math.sqrt(vyy / n)
    assert abs(X.var() - vxx) < 5 * vxx * math.sqrt(2.0 / n)
    assert abs(Y.var() - vyy) < 5 * vyy * math.sqrt(2.0 / n)
    cxy = np.mean((X - X.mean()) * (Y - Y.mean()))
    assert abs(cxy - vxy) < 5 * math.sqrt(vxx * vyy / n)


def test_ybar_shifted_gamma(orc):
    from scipy import stats
    k0, k1 = 60.0, 1.5
    m = _model(orc, 4, (k0, k1, 0.0, 0.0, 0.833, 1.0))
    # u = k0 + k1 y ~ Gamma(shape 4 k0/k1, rate 2/k1), truncated to u >= k0
    g = stats.gamma(4 * k0 / k1, scale=k1 / 2)
    lo = k0
    mean_u = g.expect(lambda u: u, lb=lo) / g.sf(lo)
    exact = (mean_u - k0) / k1
    err = abs(orc.chem_ybar(m) - exact)
    assert err < 3e-5 * exact
    # the trapezoidal rule converges at second order: half the step, a quarter of the error
    saved = orc.CHEM_DY, orc.CHEM_J
    try:
        orc.CHEM_DY, orc.CHEM_J = 0.25, 8000
        orc._chem_ybar.cache_clear()
        err_half = abs(orc.chem_ybar(m) - exact)
    finally:
        orc.CHEM_DY, orc.CHEM_J = saved
        orc._chem_ybar.cache_clear()
    assert 3.5 < err / err_half < 4.5


@pytest.mark.parametrize("kind,rates", [(4, K_DEF), (5, K_PRINTED)])
def test_ybar_against_adaptive_quadrature(orc, kind, rates):
    from scipy import integrate
    m = _model(orc, kind, rates)
    k = rates
    if kind == 4:
        minus_dg = lambda s: k[0] - k[1] * s + k[2] * s * (s - 1) - k[3] * s * (s - 1) * (s - 2)
    else:
        minus_dg = lambda s: k[0] + k[1] * s - k[2] * s * (s - 1) + k[3] * s * (s - 1) * (s - 2)
    E = lambda s: 0.5 * (k[0] + k[1] * s + k[2] * s * (s - 1) + k[3] * s * (s - 1) * (s - 2))
    grid = np.linspace(0.0, 2000.0, 2001)
    inner = np.concatenate([[0.0], np.cumsum([integrate.quad(lambda s: minus_dg(s) / E(s), a, b)[0]
                                              for a, b in zip(grid[:-1], grid[1:])])])
    logphi = inner - np.log(E(grid))
    top = logphi.max()

    def dens(s):
        i = min(int(s), 1999)
        return math.exp(inner[i] + integrate.quad(lambda t: minus_dg(t) / E(t), grid[i], s)[0]
                        - math.log(E(s)) - top)
    pts = list(np.linspace(0, 2000, 81))
    num = integrate.quad(lambda s: s * dens(s), 0, 2000, points=pts, limit=400)[0]
    den = integrate.quad(dens, 0, 2000, points=pts, limit=400)[0]
    assert abs(orc.chem_ybar(m) - num / den) < 1e-5 * num / den


def test_readings_of_the_fast_drift():
    def roots(k):
        # -d_y G (net rate) as a cubic in y: k0 - (k1 + k2 + 2 k3) y + (k2 + 3 k3) y^2 - k3 y^3
        r = np.roots([-k[3], k[2] + 3 * k[3], -(k[1] + k[2] + 2 * k[3]), k[0]])
        return np.sort(r[np.abs(r.imag) < 1e-9].real)
    r = roots(K_DEF)
    assert len(r) == 3 and np.all((r > 0) & (r < 600))          # wells, saddle, well
    assert 90 < r[0] < 120 and 180 < r[1] < 240 and 380 < r[2] < 440
    rp = roots(K_PRINTED)
    assert len(rp) == 1 and rp[0] > 5000                         # the printed k3: one root far outside


@pytest.mark.parametrize("kind", [4, 5])
def test_log_rho_inf_against_quadrature(orc, kind):
    from scipy import integrate
    m = _model(orc, kind)
    yb = orc.chem_ybar(m)
    k = K_DEF
    D = lambda s: 0.5 * (k[4] * yb + k[5] * s)
    # Fbar' by central differences of the effective potential (independent of log_rho_inf)
    dF = lambda s: float(orc.effective_potential(m, s + 1e-4) - orc.effective_potential(m, s - 1e-4)) / 2e-4
    xs = [0.0, 1.0, 87.3, 218.0, 599.5]
    got = np.array([float(orc.log_rho_inf(m, v)) for v in xs])
    want = np.array([-math.log(D(v)) - integrate.quad(lambda s: dF(s) / D(s), 0, v)[0] for v in xs])
    np.testing.assert_allclose(got - got[0], want - want[0], rtol=0, atol=1e-6)


@pytest.mark.parametrize("kind", [4, 5])
def test_generator_mass_and_equilibrium(orc, kind):
    m = _model(orc, kind)
    g = orc.Grid(600, 0.0, 600.0)
    A = orc.coarse_generator(m, g)
    assert np.max(np.abs(A.sum(axis=0))) < 1e-12 * np.max(np.abs(A))
    assert np.all(A - np.diag(np.diag(A)) >= 0.0)
    xi = 0.5 + np.arange(600.0)
    lr = np.array([float(orc.log_rho_inf(m, v)) for v in xi])
    m_inf = np.exp(lr - lr.max())
    m_inf /= m_inf.sum()
    assert np.max(np.abs(A @ m_inf)) < 1e-12 * np.max(np.abs(A)) * np.max(m_inf)
    P = orc.coarse_propagator(m, g, 2.0)
    np.testing.assert_allclose(P @ m_inf, m_inf, rtol=0, atol=1e-13)
    assert P.min() > -1e-15


def test_exactness_theorem_chemical_system(orc):
    w = workloads.CHEM.scaled(N=512, K=4, T=0.4, iters=4)
    m = _model(orc, 4)
    g = orc.Grid(w.bins, w.lo, w.hi)
    x0, y0 = workloads.initial_ensemble(w)
    res = orc.parareal(m, g, w.seed, x0, y0, w.K, w.steps, w.step_dt, iters=w.K)
    xs, ys = [x0[None]], [y0[None]]
    for n in range(w.K):
        a, b = orc.fine_propagate(m, w.seed, xs[-1], ys[-1], n, w.steps, w.step_dt)
        xs.append(a)
        ys.append(b)
    for k in range(1, w.K + 1):
        for n in range(k + 1):
            np.testing.assert_array_equal(res.x[k][n], xs[n][0])
            np.testing.assert_array_equal(res.rho[k][n], orc.restrict(xs[n], g)[1][0])
