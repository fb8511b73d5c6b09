"""The pathwise adjoint (pr_fine_adjoint) and order statistics on the GPU
against the FP64 oracle's tangent-linear derivatives and against central
finite differences with common random numbers.

Tolerances: per-particle sensitivities <= 2e-3 relative (binary32 state
against FP64) to max(|value|, RMS over the ensemble), ensemble gradients <= 5e-3
relative against central differences (h = 1e-4, FP64 propagation on the
GPU)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1912_09240_gb300 import build as b
    b.build()
    from paper_1912_09240_gb300 import _lib
    return _lib


def _close(a, b, rel, abs_=0.0):
    """|a - b| <= rel max(|b|, RMS of b over the ensemble) + abs_: a
    sensitivity that crosses zero has no relative scale of its own, so the
    ensemble's RMS sets it."""
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    scale = np.maximum(np.abs(b), np.sqrt(np.mean(b * b)))
    return np.all(np.abs(a - b) <= rel * scale + abs_)


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("slices,steps,ckpt", [(3, 40, 32), (2, 125, 256), (1, 1, 256), (4, 7, 5), (3, 40, 12), (2, 31, 12),
                                               (2, 50, 2), (1, 50, 3), (2, 48, 24)])
def test_per_particle_against_tangent(L, orc, kind, slices, steps, ckpt):
    rng = np.random.default_rng(kind + steps)
    n, dt = 1000, 1e-3
    lam, beta, eps, tau = (1.0, 1.0, 0.1, 1.0) if kind == 0 else (0.5, 3.0, 0.05, 1.0)
    x0 = rng.normal(1.0 if kind == 0 else -1.0, 0.3, n).astype(np.float32)
    y0 = rng.normal(0.0, 1.0, n).astype(np.float32)
    gm = L.Model(kind, 1, lam, beta, eps, tau)
    om = orc.Model(kind, 1, lam, beta, eps, tau)
    gx0 = torch.tensor(x0, device="cuda")
    gy0 = torch.tensor(y0, device="cuda")
    xT = torch.empty(n, dtype=torch.float32, device="cuda")
    grads = torch.empty(n, 3, dtype=torch.float64, device="cuda")
    xb0 = torch.empty(n, dtype=torch.float64, device="cuda")
    yb0 = torch.empty(n, dtype=torch.float64, device="cuda")
    ws = torch.empty(L.pr_fine_adjoint_workspace(n, slices, steps, ckpt), dtype=torch.uint8, device="cuda")
    L.pr_fine_adjoint(gm, L.Rng(9, 2), gx0, gy0, n, 3, slices, steps, dt, ckpt, xT, None, None, None, grads,
                      xb0, yb0, ws)
    torch.cuda.synchronize()
    X, Y, dX, dY = orc.fine_tangent(om, 9, x0.astype(np.float64), y0.astype(np.float64), 3, slices, steps, dt,
                                    problem=2)
    assert np.all(np.abs(xT.cpu().numpy() - X) <= 2e-3 * np.maximum(np.abs(X), 1.0))
    g = grads.cpu().numpy()
    for k in range(3):
        assert _close(g[:, k], dX[:, k], 2e-3, 1e-7), k
    assert _close(xb0.cpu().numpy(), dX[:, 3], 2e-3, 1e-7)
    assert _close(yb0.cpu().numpy(), dX[:, 4], 2e-3, 1e-7)
    # the adjoint's forward pass takes exactly pr_fine_propagate's steps
    x = gx0.reshape(1, n).clone()
    y = gy0.reshape(1, 1, n).clone()
    for s in range(slices):
        L.pr_fine_propagate(gm, L.PR_F32, L.Rng(9, 2), x, y, False, x, y, n, 3 + s, 1, steps, dt)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(x.reshape(n).cpu().numpy(), xT.cpu().numpy())


def _reverse_walk(dt, eps, tau, ckpt, total):
    """The host's rule for the reverse-walk backward pass (include/pr.h):
    (1/(1-rel))^L (1/(1-ddt))^L <= 2 over a segment of L steps."""
    L_ = min(ckpt, max(total, 1))
    rel, ddt = dt / eps, dt / tau
    return rel < 0.5 and ddt < 0.5 and L_ * (-math.log1p(-rel) - math.log1p(-ddt)) <= math.log(2.0)


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("slices,steps,ckpt", [(2, 1000, 256), (2, 999, 256), (3, 400, 100), (1, 300, 300)])
def test_reverse_walk_per_particle_against_tangent(L, orc, kind, slices, steps, ckpt):
    """Configurations where the backward pass reconstructs the states by
    inverting the Euler steps (fine steps of 1e-4 at eps = 0.1 and 0.05,
    paired and unpaired step counts, one segment over the whole horizon):
    per-particle sensitivities against the oracle's tangent-linear, end
    state equal to pr_fine_propagate's."""
    rng = np.random.default_rng(kind + steps + ckpt)
    n, dt = 1000, 1e-4
    lam, beta, eps, tau = (1.0, 1.0, 0.1, 1.0) if kind == 0 else (0.5, 3.0, 0.05, 1.0)
    assert _reverse_walk(dt, eps, tau, ckpt, slices * steps)
    x0 = rng.normal(1.0 if kind == 0 else -1.0, 0.3, n).astype(np.float32)
    y0 = rng.normal(0.0, 1.0, n).astype(np.float32)
    gm = L.Model(kind, 1, lam, beta, eps, tau)
    om = orc.Model(kind, 1, lam, beta, eps, tau)
    gx0, gy0 = torch.tensor(x0, device="cuda"), torch.tensor(y0, device="cuda")
    xT = torch.empty(n, dtype=torch.float32, device="cuda")
    grads = torch.empty(n, 3, dtype=torch.float64, device="cuda")
    xb0 = torch.empty(n, dtype=torch.float64, device="cuda")
    yb0 = torch.empty(n, dtype=torch.float64, device="cuda")
    ws = torch.empty(L.pr_fine_adjoint_workspace(n, slices, steps, ckpt), dtype=torch.uint8, device="cuda")
    L.pr_fine_adjoint(gm, L.Rng(4, 1), gx0, gy0, n, 2, slices, steps, dt, ckpt, xT, None, None, None, grads,
                      xb0, yb0, ws)
    torch.cuda.synchronize()
    X, Y, dX, dY = orc.fine_tangent(om, 4, x0.astype(np.float64), y0.astype(np.float64), 2, slices, steps, dt,
                                    problem=1)
    g = grads.cpu().numpy()
    for k in range(3):
        assert _close(g[:, k], dX[:, k], 2e-3, 1e-7), k
    assert _close(xb0.cpu().numpy(), dX[:, 3], 2e-3, 1e-7)
    assert _close(yb0.cpu().numpy(), dX[:, 4], 2e-3, 1e-7)
    x = gx0.reshape(1, n).clone()
    y = gy0.reshape(1, 1, n).clone()
    for s in range(slices):
        L.pr_fine_propagate(gm, L.PR_F32, L.Rng(4, 1), x, y, False, x, y, n, 2 + s, 1, steps, dt)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(x.reshape(n).cpu().numpy(), xT.cpu().numpy())


def test_seeded_sum_equals_contracted_per_particle(L):
    n, slices, steps, dt = 5000, 2, 100, 1e-3
    gm = L.Model(0, 1, 0.8, 1.5, 0.1, 1.0)
    rng = np.random.default_rng(1)
    x0 = torch.tensor(rng.normal(1, 0.2, n), dtype=torch.float32, device="cuda")
    y0 = torch.tensor(rng.normal(0, 1, n), dtype=torch.float32, device="cuda")
    seeds = torch.tensor(rng.normal(0, 1, n), dtype=torch.float64, device="cuda")
    ws = torch.empty(L.pr_fine_adjoint_workspace(n, slices, steps, 256), dtype=torch.uint8, device="cuda")
    per = torch.empty(n, 3, dtype=torch.float64, device="cuda")
    L.pr_fine_adjoint(gm, L.Rng(0), x0, y0, n, 0, slices, steps, dt, 256, None, None, None, None, per, None, None, ws)
    tot = torch.zeros(3, dtype=torch.float64, device="cuda")
    L.pr_fine_adjoint(gm, L.Rng(0), x0, y0, n, 0, slices, steps, dt, 256, None, None, seeds, None, tot, None, None, ws)
    tot2 = torch.zeros(3, dtype=torch.float64, device="cuda")
    L.pr_fine_adjoint(gm, L.Rng(0), x0, y0, n, 0, slices, steps, dt, 256, None, None, seeds, None, tot2, None, None, ws)
    torch.cuda.synchronize()
    terms = (seeds[:, None] * per).cpu().numpy()
    ref = terms.sum(0)
    # both sides run the binary32 recursion over 200 steps (relative error per
    # particle up to ~200 x 2^-24 = 1.2e-5, differently rounded with the seed
    # folded in); the sum over particles cancels, so the bound scales with
    # the sum of magnitudes
    assert np.all(np.abs(tot.cpu().numpy() - ref) <= 2e-5 * np.abs(terms).sum(0))
    np.testing.assert_array_equal(tot.cpu().numpy(), tot2.cpu().numpy())   # deterministic reduction


@pytest.mark.parametrize("kind,eps_dw", [(0, None), (1, 0.01), (1, 0.05)])
def test_second_moment_gradient_against_central_differences(L, kind, eps_dw):
    """Central differences (h = 1e-4) of E[X_T^2] with common random numbers,
    propagated in FP64 on the GPU, against the binary32 adjoint (the OU case
    and the double well at eps = 0.05 take the reverse walk, the double well
    at eps = 0.01 the exact replay)."""
    from paper_1912_09240_gb300.adjoint import second_moment_gradient
    n, slices, steps, dt = 1 << 16, 2, 1000, 1e-4
    lam, beta, eps = (1.0, 1.0, 0.1) if kind == 0 else (0.5, 3.0, eps_dw)
    assert _reverse_walk(dt, eps, 1.0, 256, slices * steps) == (eps >= 0.05)
    rng = np.random.default_rng(3)
    x0n = rng.normal(1.0 if kind == 0 else -1.0, 0.1, n)
    y0n = rng.normal(0.0, 1.0, n) if kind == 0 else x0n.copy()
    x0 = torch.tensor(x0n, dtype=torch.float32, device="cuda")
    y0 = torch.tensor(y0n, dtype=torch.float32, device="cuda")
    val, grad = second_moment_gradient(L.Model(kind, 1, lam, beta, eps), L.Rng(0), x0, y0, 0, slices, steps, dt)
    torch.cuda.synchronize()

    def second_moment(l_, b_, e_):
        x = x0.double().reshape(1, n).clone()
        y = y0.double().reshape(1, 1, n).clone()
        for s in range(slices):
            L.pr_fine_propagate(L.Model(kind, 1, l_, b_, e_), L.PR_F64, L.Rng(0), x, y, False, x, y, n, s, 1,
                                steps, dt)
        return float((x ** 2).mean().item())

    h = 1e-4
    fd = [(second_moment(lam + h, beta, eps) - second_moment(lam - h, beta, eps)) / (2 * h),
          (second_moment(lam, beta + h, eps) - second_moment(lam, beta - h, eps)) / (2 * h),
          (second_moment(lam, beta, eps + h * eps) - second_moment(lam, beta, eps - h * eps)) / (2 * h * eps)]
    g = grad.cpu().numpy()
    for k in range(3):
        assert abs(g[k] - fd[k]) <= 5e-3 * max(abs(fd[k]), 1e-3 * max(abs(v) for v in fd)), (k, g[k], fd[k])
    assert abs(val.item() - second_moment(lam, beta, eps)) < 1e-4


def test_autograd_function_matches_adjoint(L):
    from paper_1912_09240_gb300.adjoint import fine_em
    n, slices, steps, dt = 4096, 2, 50, 1e-3
    rng = np.random.default_rng(4)
    x0 = torch.tensor(rng.normal(1, 0.2, n), dtype=torch.float32, device="cuda", requires_grad=True)
    y0 = torch.tensor(rng.normal(0, 1, n), dtype=torch.float32, device="cuda", requires_grad=True)
    theta = torch.tensor([0.9, 1.2, 0.1], dtype=torch.float64, device="cuda", requires_grad=True)
    xT, yT = fine_em(theta, x0, y0, 0, 1.0, L.Rng(5), 0, slices, steps, dt)
    loss = (xT.double() ** 2).mean() + 0.5 * (xT.double() * yT.double()).mean()
    loss.backward()
    torch.cuda.synchronize()
    # reference: the same loss through the oracle's tangent-linear
    from oracle import oracle as orc
    om = orc.Model(0, 1, 0.9, 1.2, 0.1)
    X, Y, dX, dY = orc.fine_tangent(om, 5, x0.detach().cpu().numpy().astype(np.float64),
                                    y0.detach().cpu().numpy().astype(np.float64), 0, slices, steps, dt)
    dl = ((2 * X + 0.5 * Y)[:, None] * dX + (0.5 * X)[:, None] * dY) / n
    np.testing.assert_allclose(theta.grad.cpu().numpy(), dl[:, :3].sum(0), rtol=3e-3)
    np.testing.assert_allclose(x0.grad.double().cpu().numpy(), dl[:, 3], rtol=3e-3, atol=1e-9)
    np.testing.assert_allclose(y0.grad.double().cpu().numpy(), dl[:, 4], rtol=3e-3, atol=1e-9)


def test_order_statistics(L):
    rng = np.random.default_rng(6)
    for n in (1, 7, 1000, 1 << 16, 100_003):
        x = rng.normal(0, 1, n).astype(np.float32)
        if n > 10:
            x[:10] = x[10]                      # ties are broken by particle index
        ranks = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, 50)]))
        gx = torch.tensor(x, device="cuda")
        gr = torch.tensor(np.concatenate([ranks, [n, -1]]), dtype=torch.int64, device="cuda")
        idx = torch.empty(gr.numel(), dtype=torch.int64, device="cuda")
        ws = torch.empty(L.pr_order_statistics_workspace(n), dtype=torch.uint8, device="cuda")
        L.pr_order_statistics(gx, n, gr, gr.numel(), idx, ws)
        torch.cuda.synchronize()
        order = np.lexsort((np.arange(n), x))
        got = idx.cpu().numpy()
        np.testing.assert_array_equal(got[:-2], order[ranks])
        assert got[-2] == -1 and got[-1] == -1


@pytest.mark.parametrize("case", ["normal_2^20", "bimodal", "rounded_ties", "all_equal_small", "all_equal_large",
                                  "cauchy", "with_inf_nan", "one_outlier", "ragged_tiny"])
def test_order_statistics_selection_cases(L, case):
    """The bucket selection and its fallback to the full sort against
    np.lexsort (value in the total order of binary32, -0 before +0, then
    index): a large normal ensemble with the 512
    quantile ranks, a bimodal one, values rounded to few levels (many ties),
    equal values (within and beyond one bucket's sort capacity), heavy tails,
    infinities and NaN, a single far outlier, and tiny ensembles."""
    rng = np.random.default_rng(hash(case) % (1 << 32))
    n = 1 << 20 if case == "normal_2^20" else 100_003
    if case in ("normal_2^20", "ragged_tiny"):
        x = rng.normal(0, 1, n)
    elif case == "bimodal":
        x = np.where(rng.random(n) < 0.3, rng.normal(-1, 0.1, n), rng.normal(1.5, 0.3, n))
    elif case == "rounded_ties":
        x = np.round(rng.normal(0, 1, n) * 20) / 20
    elif case == "all_equal_small":
        n = 3000
        x = np.full(n, 0.25)
    elif case == "all_equal_large":
        x = np.full(n, -1.5)
    elif case == "cauchy":
        x = rng.standard_cauchy(n)
    elif case == "with_inf_nan":
        x = rng.normal(0, 1, n)
        x[[5, 77, 1000]] = [np.inf, -np.inf, np.nan]
    else:   # one_outlier
        x = rng.normal(0, 1, n)
        x[12345] = 1e30
    if case == "ragged_tiny":
        n = 37
        x = x[:n]
    x = x.astype(np.float32)
    p = (np.arange(512) + 0.5) / 512
    ranks = np.unique(np.concatenate([np.ceil(p * n).astype(np.int64) - 1, [0, n - 1]]))
    gx = torch.tensor(x, device="cuda")
    gr = torch.tensor(ranks, dtype=torch.int64, device="cuda")
    idx = torch.empty(gr.numel(), dtype=torch.int64, device="cuda")
    ws = torch.empty(L.pr_order_statistics_workspace(n), dtype=torch.uint8, device="cuda")
    L.pr_order_statistics(gx, n, gr, gr.numel(), idx, ws)
    torch.cuda.synchronize()
    # the total order of binary32 values (-0 before +0, NaN above +inf), then the index
    k = x.view(np.uint32)
    key = np.where(k & 0x80000000, ~k, k | 0x80000000)
    order = np.lexsort((np.arange(n), key))
    np.testing.assert_array_equal(idx.cpu().numpy(), order[ranks])


def test_adjoint_workload_sampled_at_full_size(L, orc):
    """The adjoint workload at full size (2^20 particles, 20 slices x 1000
    steps, checkpoints every 256 steps): sampled particles' sensitivities
    against the oracle's tangent-linear on those particles (their own keys),
    and the 512-point quantile function's gradient at the ranked particles."""
    import workloads
    from paper_1912_09240_gb300.adjoint import quantile_gradient
    w = workloads.ADJOINT
    x0, y0 = workloads.initial_ensemble(w)
    gx0 = torch.tensor(x0, dtype=torch.float32, device="cuda")
    gy0 = torch.tensor(y0[0], dtype=torch.float32, device="cuda")
    model = L.Model(w.kind, 1, w.lam, w.beta, w.eps, w.tau_x)
    Q, dQ, idx = quantile_gradient(model, L.Rng(w.seed), gx0, gy0, 0, w.K, w.steps, w.step_dt)
    torch.cuda.synchronize()
    idx = idx.cpu().numpy()
    Q = Q.cpu().numpy()
    assert np.all(np.diff(Q) >= 0)
    sample = np.unique(np.concatenate([idx[::32], [idx[0], idx[-1]]])).astype(np.uint32)
    om = orc.Model(w.kind, 1, w.lam, w.beta, w.eps, w.tau_x)
    x0f = x0.astype(np.float32).astype(np.float64)
    y0f = y0[0].astype(np.float32).astype(np.float64)
    X, Y, dX, dY = orc.fine_tangent(om, w.seed, x0f[sample], y0f[sample], 0, w.K, w.steps, w.step_dt, ids=sample)
    pos = {int(p): i for i, p in enumerate(sample)}
    dq = dQ.cpu().numpy()
    # relative to max(|value|, RMS over the sampled particles): a sensitivity
    # that crosses zero is compared on the scale of the ensemble's sensitivities
    rms = np.sqrt((dX[:, :3] ** 2).mean(axis=0))
    for j, p in enumerate(idx):
        if int(p) in pos:
            i = pos[int(p)]
            assert abs(Q[j] - X[i]) <= 2e-3 * max(abs(X[i]), 1.0)
            for k in range(3):
                assert abs(dq[j, k] - dX[i, k]) <= 2e-3 * max(abs(dX[i, k]), rms[k]), (j, k, dq[j, k], dX[i, k])


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("steps,ckpt", [(40, 12), (31, 5), (100, 256)])
@pytest.mark.parametrize("scale,shift", [(None, 0.0), (0.3, -0.7), (0.0, None)])
def test_affine_seed_equals_given_seeds(L, kind, steps, ckpt, scale, shift):
    """pr_fine_adjoint_affine against pr_fine_adjoint with the seeds
    scale X_T + shift computed from the end states (scale = 2/n: the second
    moment; scale = 0, shift = 1/n: the mean): the gradient, the end states
    and the initial-state sensitivities bit for bit."""
    n, slices, dt = 3001, 3, 1e-3
    scale = 2.0 / n if scale is None else scale
    shift = 1.0 / n if shift is None else shift
    lam, beta, eps = (1.0, 1.0, 0.1) if kind == 0 else (0.5, 3.0, 0.05)
    rng = np.random.default_rng(steps + kind)
    x0 = torch.tensor(rng.normal(0.5, 0.4, n), dtype=torch.float32, device="cuda")
    y0 = torch.tensor(rng.normal(0.0, 1.0, n), dtype=torch.float32, device="cuda")
    m, r = L.Model(kind, 1, lam, beta, eps), L.Rng(21, 4)
    ws = torch.empty(L.pr_fine_adjoint_workspace(n, slices, steps, ckpt), dtype=torch.uint8, device="cuda")
    xT = torch.empty(n, dtype=torch.float32, device="cuda")
    g1 = torch.zeros(3, dtype=torch.float64, device="cuda")
    xb1 = torch.empty(n, dtype=torch.float64, device="cuda")
    yb1 = torch.empty(n, dtype=torch.float64, device="cuda")
    L.pr_fine_adjoint_affine(m, r, x0, y0, n, 2, slices, steps, dt, ckpt, scale, shift, xT, None, g1, xb1, yb1, ws)
    seeds = scale * xT.to(torch.float64) + shift
    g0 = torch.zeros(3, dtype=torch.float64, device="cuda")
    xT0 = torch.empty(n, dtype=torch.float32, device="cuda")
    xb0 = torch.empty(n, dtype=torch.float64, device="cuda")
    yb0 = torch.empty(n, dtype=torch.float64, device="cuda")
    L.pr_fine_adjoint(m, r, x0, y0, n, 2, slices, steps, dt, ckpt, xT0, None, seeds, None, g0, xb0, yb0, ws)
    torch.cuda.synchronize()
    assert torch.equal(xT, xT0)
    assert torch.equal(g1, g0), (g1, g0)
    assert torch.equal(xb1, xb0) and torch.equal(yb1, yb0)


@pytest.mark.parametrize("n", [1, 37])
def test_adjoint_without_steps(L, n):
    """No steps at all (steps = 0): X_T = X_0, every parameter derivative is
    0 and dX_T/dX_0 = 1, dX_T/dY_0 = 0, per particle and seeded."""
    rng = np.random.default_rng(n)
    x0 = torch.tensor(rng.normal(size=n), dtype=torch.float32, device="cuda")
    y0 = torch.tensor(rng.normal(size=n), dtype=torch.float32, device="cuda")
    m = L.Model(L.PR_MODEL_DOUBLE_WELL, 1, 0.5, 3.0, 0.05)
    ws = torch.empty(L.pr_fine_adjoint_workspace(n, 2, 0, 12), dtype=torch.uint8, device="cuda")
    xT = torch.empty(n, dtype=torch.float32, device="cuda")
    grads = torch.empty(n, 3, dtype=torch.float64, device="cuda")
    xb0 = torch.empty(n, dtype=torch.float64, device="cuda")
    yb0 = torch.empty(n, dtype=torch.float64, device="cuda")
    L.pr_fine_adjoint(m, L.Rng(1, 0), x0, y0, n, 0, 2, 0, 1e-3, 12, xT, None, None, None, grads, xb0, yb0, ws)
    torch.cuda.synchronize()
    assert torch.equal(xT, x0)
    assert torch.all(grads == 0.0) and torch.all(xb0 == 1.0) and torch.all(yb0 == 0.0)
    g = torch.full((3,), 7.0, dtype=torch.float64, device="cuda")
    L.pr_fine_adjoint_affine(m, L.Rng(1, 0), x0, y0, n, 0, 2, 0, 1e-3, 12, 2.0 / n, 0.0, xT, None, g, None, None,
                             ws)
    torch.cuda.synchronize()
    assert torch.all(g == 0.0)


def test_adjoint_single_particle_against_tangent(L, orc):
    """One particle, the paired and the step-by-step kernels (even and odd
    steps per slice): against the oracle's tangent-linear derivatives."""
    for steps in (40, 41):
        x0 = np.array([0.7], dtype=np.float32)
        y0 = np.array([-0.2], dtype=np.float32)
        gm = L.Model(L.PR_MODEL_OU, 1, 0.8, 1.5, 0.1)
        om = orc.Model(0, 1, 0.8, 1.5, 0.1)
        ws = torch.empty(L.pr_fine_adjoint_workspace(1, 3, steps, 16), dtype=torch.uint8, device="cuda")
        xT = torch.empty(1, dtype=torch.float32, device="cuda")
        grads = torch.empty(1, 3, dtype=torch.float64, device="cuda")
        L.pr_fine_adjoint(gm, L.Rng(4, 1), torch.tensor(x0, device="cuda"), torch.tensor(y0, device="cuda"), 1, 2, 3,
                          steps, 1e-3, 16, xT, None, None, None, grads, None, None, ws)
        torch.cuda.synchronize()
        rx, _, dx, _ = orc.fine_tangent(om, 4, x0.astype(np.float64), y0.astype(np.float64), 2, 3, steps, 1e-3,
                                        problem=1)
        g = grads.cpu().numpy()[0]
        ref = dx[0, :3]
        assert np.all(np.abs(g - ref) <= 2e-3 * np.maximum(np.abs(ref), 1e-3)), (steps, g, ref)
        assert abs(float(xT.item()) - rx[0]) <= 2e-3 * max(abs(rx[0]), 1.0)
