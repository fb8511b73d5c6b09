"""The Monte Carlo estimator (Section 2.1.3, Eq. MCestimator) on the GPU
against the oracle: power observables of the slow variable and of one fast
component, with and without weights, binary32 and binary64 ensembles, ragged
sizes and several slices.  Every term is the same binary64 product on both
sides; only the order of the additions differs, so the tolerance is a few
units of rounding of the sum of absolute terms."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def L():
    from paper_1912_09240_gb300 import build as b
    b.build()
    from paper_1912_09240_gb300 import _lib
    return _lib


def _gpu_moments(L, prec, v, stride, w, n, n_slices, Q):
    out = torch.empty(n_slices, Q, dtype=torch.float64, device=DEV)
    ws = torch.empty(L.pr_moments_workspace(n, n_slices, Q), dtype=torch.uint8, device=DEV)
    L.pr_moments(prec, v, stride, w, n, n_slices, Q, out, ws)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _check(got, ref, v64, w, Q):
    n = v64.shape[1]
    for q in range(1, Q + 1):
        terms = np.abs(v64) ** q * (np.abs(w) if w is not None else 1.0 / n)
        scale = terms.sum(axis=1)
        err = np.abs(got[:, q - 1] - ref[:, q - 1])
        assert np.all(err <= 1e-13 * scale + 1e-300), (q, err, scale)


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("n", [1, 7, 4096, 4097, 100003])
def test_moments_against_oracle(L, orc, prec, weighted, n):
    rng = np.random.default_rng(n + 11 * weighted)
    n_slices, Q = 3, 4
    v64 = rng.normal(0.3, 1.2, size=(n_slices, n))
    dt = torch.float32 if prec == "f32" else torch.float64
    v = torch.tensor(v64, dtype=dt, device=DEV)
    v64 = v.double().cpu().numpy()            # the values the GPU sees
    w = rng.random((n_slices, n)) if weighted else None
    if weighted:
        w /= w.sum(axis=1, keepdims=True)
    wt = torch.tensor(w, device=DEV) if weighted else None
    got = _gpu_moments(L, L.PR_F32 if prec == "f32" else L.PR_F64, v, n, wt, n, n_slices, Q)
    ref = orc.moments(v64, Q, w)
    _check(got, ref, v64, w, Q)


def test_fast_component_with_stride(L, orc):
    """Component c of y[n_slices][d][n]: the slice stride is d n."""
    rng = np.random.default_rng(5)
    n_slices, d, n, c, Q = 4, 3, 5003, 1, 2
    y = torch.tensor(rng.standard_normal((n_slices, d, n)), dtype=torch.float32, device=DEV)
    # the base pointer of component c and the stride between slices
    out = torch.empty(n_slices, Q, dtype=torch.float64, device=DEV)
    ws = torch.empty(L.pr_moments_workspace(n, n_slices, Q), dtype=torch.uint8, device=DEV)
    base = y.reshape(-1)[c * n:]
    L.pr_moments(L.PR_F32, base, d * n, None, n, n_slices, Q, out, ws)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    v64 = y[:, c, :].double().cpu().numpy()
    _check(got, orc.moments(v64, Q), v64, None, Q)


def test_moments_deterministic_and_exact_cases(L):
    """Two calls give the same bits; constant ensembles give c^q; the mean
    of an ensemble symmetric about 0 is 0 exactly (dyadic values pair off)."""
    n = 1 << 20
    rng = np.random.default_rng(9)
    v = torch.tensor(rng.standard_normal((2, n)), dtype=torch.float32, device=DEV)
    a = _gpu_moments(L, L.PR_F32, v, n, None, n, 2, 4)
    b = _gpu_moments(L, L.PR_F32, v, n, None, n, 2, 4)
    assert np.array_equal(a, b)
    c = torch.full((1, 12345), 1.5, dtype=torch.float64, device=DEV)
    got = _gpu_moments(L, L.PR_F64, c, 12345, None, 12345, 1, 4)[0]
    np.testing.assert_allclose(got, [1.5, 2.25, 3.375, 5.0625], rtol=1e-15)
    half = (torch.arange(1, 4097, dtype=torch.float64, device=DEV) / 64).reshape(1, -1)
    sym = torch.cat([half, -half], dim=1).contiguous()
    got = _gpu_moments(L, L.PR_F64, sym, 8192, None, 8192, 1, 3)[0]
    assert got[0] == 0.0 and got[2] == 0.0
    k = np.arange(1, 4097, dtype=np.float64)
    assert got[1] == float((k * k).sum()) / 64 / 64 * 2 / 8192


def test_second_moment_helper_uses_the_estimator(L, orc):
    """adjoint.second_moment_gradient's value is E[X_T^2] of the end states
    (compared with the oracle estimator on the propagated ensemble)."""
    from paper_1912_09240_gb300.adjoint import second_moment_gradient
    n, slices, steps, dt = 3001, 2, 40, 1e-3
    rng = np.random.default_rng(2)
    x0 = torch.tensor(rng.normal(1.0, 0.1, n), dtype=torch.float32, device=DEV)
    y0 = torch.tensor(rng.standard_normal(n), dtype=torch.float32, device=DEV)
    model = L.Model(L.PR_MODEL_OU, 1, 1.0, 1.0, 0.1)
    val, _ = second_moment_gradient(model, L.Rng(4), x0, y0, 0, slices, steps, dt)
    x = x0.reshape(1, n).clone()
    y = y0.reshape(1, 1, n).clone()
    for s in range(slices):
        L.pr_fine_propagate(model, L.PR_F32, L.Rng(4), x, y, False, x, y, n, s, 1, steps, dt)
    torch.cuda.synchronize()
    ref = orc.moments(x.double().cpu().numpy(), 2)[0, 1]
    assert abs(float(val) - ref) <= 1e-13 * ref


@pytest.mark.parametrize("matching", ["quantile", "reweight"])
def test_solver_moments(L, orc, matching):
    """PararealSolver.moments(): the estimator over the fine end states of the
    latest iteration, slow variable and a fast component, with the weights
    those states carry."""
    import workloads
    from paper_1912_09240_gb300.parareal import PararealSolver
    w = workloads.LARGE_FAST.scaled(N=3001, K=5, T=0.05, dt=1e-3, bins=64, fast_dim=3, eps=0.1)
    model = L.Model(w.kind, w.fast_dim, w.lam, w.beta, w.eps, w.tau_x)
    s = PararealSolver(model, L.Grid(w.bins, w.lo, w.hi), w.N, w.K, w.steps, w.step_dt, rng=L.Rng(w.seed, 0),
                       matching=matching)
    x0, y0 = workloads.initial_ensemble(w)
    s.set_initial(torch.tensor(x0, dtype=torch.float32, device=DEV), torch.tensor(y0, dtype=torch.float32, device=DEV))
    for _ in range(2):
        s.iterate()
    xa, ya, _ = s.state()
    wts = s.weights()
    wn = wts.cpu().numpy() if wts is not None else None
    got_x = s.moments(3).cpu().numpy()
    got_y = s.moments(2, component=1).cpu().numpy()
    v64 = xa.double().cpu().numpy()
    _check(got_x, orc.moments(v64, 3, wn), v64, wn, 3)
    y64 = ya[:, 1, :].double().cpu().numpy()
    _check(got_y, orc.moments(y64, 2, wn), y64, wn, 2)
    with pytest.raises(ValueError):
        s.moments(2, component=3)
    s.close()


def test_moments_many_slices(L, orc):
    """More slices than the grid's block budget (one block per slice then)."""
    rng = np.random.default_rng(21)
    S, n = 3000, 37
    v64 = rng.normal(0.0, 1.0, (S, n))
    w = rng.random((S, n))
    w /= w.sum(axis=1, keepdims=True)
    v = torch.tensor(v64, dtype=torch.float32, device=DEV)
    v64 = v.double().cpu().numpy()
    got = _gpu_moments(L, L.PR_F32, v, n, torch.tensor(w, device=DEV), n, S, 3)
    _check(got, orc.moments(v64, 3, w), v64, w, 3)
