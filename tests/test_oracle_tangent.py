"""Pins of the oracle's tangent-linear (pathwise) derivatives of the EM
recursion: central finite differences of the oracle's own EM with common
random numbers, and, for the linear OU family, the derivative of E[X_T^2]
that the exact EM moment recursion gives."""
import numpy as np
import pytest


def _run(orc, model, x0, y0, slices, steps, dt):
    xs, ys = x0[None].copy(), y0[None, None].copy()
    for s in range(slices):
        xs, ys = orc.fine_propagate(model, 3, xs, ys, s, steps, dt)
    return xs[0], ys[0, 0]


@pytest.mark.parametrize("kind", [0, 1])
def test_tangent_matches_central_differences(orc, kind):
    rng = np.random.default_rng(kind)
    N, slices, steps, dt = 64, 3, 40, 1e-3
    lam, beta, eps, tau = 0.7, 2.0, 0.05, 1.3
    x0 = rng.normal(-0.5, 0.5, N)
    y0 = rng.normal(0.0, 0.7, N)
    model = orc.Model(kind, 1, lam, beta, eps, tau)
    X, Y, dX, dY = orc.fine_tangent(model, 3, x0, y0, 0, slices, steps, dt)
    Xr, Yr = _run(orc, model, x0, y0, slices, steps, dt)
    np.testing.assert_array_equal(X, Xr)
    h = 1e-6
    for k, name in enumerate(["lam", "beta", "eps"]):
        vals = dict(lam=lam, beta=beta, eps=eps)
        vp, vm = dict(vals), dict(vals)
        vp[name] += h
        vm[name] -= h
        Xp, Yp = _run(orc, orc.Model(kind, 1, vp["lam"], vp["beta"], vp["eps"], tau), x0, y0, slices, steps, dt)
        Xm, Ym = _run(orc, orc.Model(kind, 1, vm["lam"], vm["beta"], vm["eps"], tau), x0, y0, slices, steps, dt)
        np.testing.assert_allclose(dX[:, k], (Xp - Xm) / (2 * h), rtol=1e-5, atol=1e-8)
        np.testing.assert_allclose(dY[:, k], (Yp - Ym) / (2 * h), rtol=1e-5, atol=1e-7)
    for k, dx0, dy0 in [(3, h, 0.0), (4, 0.0, h)]:
        Xp, _ = _run(orc, model, x0 + dx0, y0 + dy0, slices, steps, dt)
        Xm, _ = _run(orc, model, x0 - dx0, y0 - dy0, slices, steps, dt)
        np.testing.assert_allclose(dX[:, k], (Xp - Xm) / (2 * h), rtol=1e-5, atol=1e-8)


def _second_moment(lam, beta, eps, dt, steps, m0, S0):
    M = np.array([[1.0 - dt, lam * dt], [dt / eps, 1.0 - dt / eps]])
    Q = np.diag([2.0 / beta * dt, 2.0 / eps * dt])
    m, S = m0.copy(), S0.copy()
    for _ in range(steps):
        m = M @ m
        S = M @ S @ M.T + Q
    return m[0] ** 2 + S[0, 0]


def test_tangent_second_moment_against_moment_recursion(orc):
    """d E[X_T^2] / d theta for the OU family: the exact EM moment recursion,
    differentiated by central differences (a deterministic recursion)."""
    N, steps, dt = 1 << 15, 200, 1e-3
    lam, beta, eps = 1.0, 1.0, 0.1
    rng = np.random.default_rng(0)
    x0 = rng.normal(1.0, 0.1, N)
    y0 = rng.normal(0.0, 1.0, N)
    X, Y, dX, dY = orc.fine_tangent(orc.Model(0, 1, lam, beta, eps), 0, x0, y0, 0, 1, steps, dt)
    z0 = np.stack([x0, y0])
    m0, S0 = z0.mean(axis=1), np.cov(z0, bias=True)
    g_mc = (2.0 * X[:, None] * dX[:, :3]).mean(axis=0)
    se = (2.0 * X[:, None] * dX[:, :3]).std(axis=0) / np.sqrt(N)
    h = 1e-6
    base = dict(lam=lam, beta=beta, eps=eps)
    for k, name in enumerate(["lam", "beta", "eps"]):
        vp, vm = dict(base), dict(base)
        vp[name] += h
        vm[name] -= h
        g = (_second_moment(vp["lam"], vp["beta"], vp["eps"], dt, steps, m0, S0)
             - _second_moment(vm["lam"], vm["beta"], vm["eps"], dt, steps, m0, S0)) / (2 * h)
        assert abs(g_mc[k] - g) < 5.0 * se[k] + 1e-9, (name, g_mc[k], g, se[k])
