"""Pins of the oracle's Euler-Maruyama fine propagator (Eqs. EMx/EMy).

For the linear OU family the EM scheme maps Gaussian moments exactly:
m' = M m, S' = M S M^T + diag(2D dt, 2E/eps dt) with
M = [[1 - dt, lambda dt], [dt/eps, 1 - dt/eps]].  The ensemble moments must
sit within a few standard errors of that recursion.  For the non-linear
families one EM step from a fixed state has a closed-form mean and variance.
"""
import numpy as np
import pytest


def _moments_recursion(m, S, lam, beta, eps, dt, steps):
    M = np.array([[1.0 - dt, lam * dt], [dt / eps, 1.0 - dt / eps]])
    Q = np.diag([2.0 / beta * dt, 2.0 / eps * dt])
    for _ in range(steps):
        m = M @ m
        S = M @ S @ M.T + Q
    return m, S


@pytest.mark.parametrize("lam,beta,eps", [(1.0, 1.0, 0.1), (0.6, 2.5, 0.05)])
def test_ou_moment_recursion(orc, lam, beta, eps):
    N, dt, steps = 1 << 15, 1e-3, 60
    rng = np.random.default_rng(11)
    x0 = rng.normal(1.0, 0.1, N)
    y0 = rng.normal(0.0, 1.0, N)
    model = orc.Model(kind=0, lam=lam, beta=beta, eps=eps)
    x, y = orc.fine_propagate(model, seed=0, x=x0[None], y=y0[None, None], slice_begin=0,
                              steps=steps, dt=dt)
    z0 = np.stack([x0, y0])
    m_hat0 = z0.mean(axis=1)
    S_hat0 = np.cov(z0, bias=True)
    m_pred, S_pred = _moments_recursion(m_hat0, S_hat0, lam, beta, eps, dt, steps)
    _, S_noise = _moments_recursion(np.zeros(2), np.zeros((2, 2)), lam, beta, eps, dt, steps)
    z = np.stack([x[0], y[0, 0]])
    se_mean = np.sqrt(np.diag(S_noise) / N)
    assert np.all(np.abs(z.mean(axis=1) - m_pred) < 4.5 * se_mean)
    S_emp = np.cov(z, bias=True)
    se_var = np.sqrt(2.0 / N) * np.diag(S_pred)
    assert np.all(np.abs(np.diag(S_emp) - np.diag(S_pred)) < 5.0 * se_var)
    se_cov = np.sqrt((S_pred[0, 0] * S_pred[1, 1] + S_pred[0, 1] ** 2) / N)
    assert abs(S_emp[0, 1] - S_pred[0, 1]) < 5.0 * se_cov


@pytest.mark.parametrize("kind,d,tau", [(1, 1, 1.0), (2, 16, 1.0), (1, 1, 2.0), (0, 1, 1.0)])
def test_one_step_closed_form(orc, kind, d, tau):
    """E and Var of one EM step from a fixed state (x0, y0)."""
    N, dt = 1 << 16, 1e-2
    lam, beta, eps = 0.5, 3.0, 0.05
    x0v = 1.3
    y0v = np.linspace(-0.4, 0.8, d) if d > 1 else np.array([-0.4])
    model = orc.Model(kind=kind, fast_dim=d, lam=lam, beta=beta, eps=eps, tau_x=tau)
    x0 = np.full((1, N), x0v)
    y0 = np.broadcast_to(y0v[None, :, None], (1, d, N)).copy()
    x, y = orc.fine_propagate(model, seed=123, x=x0, y=y0, slice_begin=4, steps=1, dt=dt)
    if kind == 0:
        dF = x0v - lam * y0v[0]
    elif kind == 1:
        dF = x0v ** 3 - x0v + lam * y0v[0]
    else:
        dF = x0v ** 3 - x0v + lam * y0v.mean()
    ex = x0v - dF / tau * dt
    vx = 2.0 / beta / tau * dt
    assert abs(x.mean() - ex) < 4.5 * np.sqrt(vx / N)
    assert abs(x.var() - vx) < 5.0 * vx * np.sqrt(2.0 / N)
    for j in range(d):
        ey = y0v[j] - (y0v[j] - x0v) / eps * dt
        vy = 2.0 / eps * dt
        assert abs(y[0, j].mean() - ey) < 4.5 * np.sqrt(vy / N)
        assert abs(y[0, j].var() - vy) < 5.0 * vy * np.sqrt(2.0 / N)
    # slow and fast noises are independent
    assert abs(np.corrcoef(x[0], y[0, 0])[0, 1]) < 5.0 / np.sqrt(N)


def test_reuse_of_numbers_and_slice_keys(orc):
    """Same slice + same start = same path (reuse across iterations); a
    different slice index draws different numbers."""
    model = orc.Model(kind=1, lam=0.5, beta=3.0, eps=0.01)
    rng = np.random.default_rng(3)
    x0 = rng.normal(-1, 0.2, (1, 64))
    y0 = x0[:, None, :].copy()
    a = orc.fine_propagate(model, 0, x0, y0, 7, 13, 1e-4)
    b = orc.fine_propagate(model, 0, x0, y0, 7, 13, 1e-4)
    c = orc.fine_propagate(model, 0, x0, y0, 8, 13, 1e-4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not np.array_equal(a[0], c[0])
    # several slices in one call = the slices one at a time
    xs = np.concatenate([x0, x0 + 0.1])
    ys = np.concatenate([y0, y0 - 0.1])
    both = orc.fine_propagate(model, 0, xs, ys, 7, 13, 1e-4)
    second = orc.fine_propagate(model, 0, xs[1:], ys[1:], 8, 13, 1e-4)
    assert np.array_equal(both[0][0], a[0][0])
    assert np.array_equal(both[0][1], second[0][0])


def test_odd_step_count_uses_half_block(orc):
    """With 2 normals per step one Philox block serves steps 2j and 2j+1;
    3 steps from x equal 2 steps then 1 step only through the counters, so
    check instead that steps taken one call at a time differ from a fresh
    start (the step index, not the call, keys the numbers)."""
    model = orc.Model(kind=0, lam=1.0, beta=1.0, eps=0.1)
    x0 = np.zeros((1, 8))
    y0 = np.zeros((1, 1, 8))
    x3, _ = orc.fine_propagate(model, 0, x0, y0, 0, 3, 1e-3)
    x1, _ = orc.fine_propagate(model, 0, x0, y0, 0, 1, 1e-3)
    assert not np.array_equal(x3, x1)
    assert np.all(np.isfinite(x3))


def test_sample_with_particle_ids(orc):
    """A sample of columns advanced with its particle indices reproduces those
    columns of the whole ensemble (used for sampled parity at full size)."""
    model = orc.Model(kind=1, lam=0.5, beta=3.0, eps=0.01)
    rng = np.random.default_rng(5)
    x0 = rng.normal(-1, 0.2, (2, 300))
    y0 = x0[:, None, :].copy()
    full = orc.fine_propagate(model, 0, x0, y0, 3, 9, 1e-4)
    ids = np.array([7, 0, 299, 150], dtype=np.uint32)
    part = orc.fine_propagate(model, 0, x0[:, ids], y0[:, :, ids], 3, 9, 1e-4, ids=ids)
    assert np.array_equal(part[0], full[0][:, ids])
    assert np.array_equal(part[1], full[1][:, :, ids])
