"""Skipping the fine propagation of converged slices (exactness property,
Section 3.2.4: iterate k is the serial fine solution on slices n <= k, so
K(K-1)/2 slice propagations need not be repeated over K iterations).

With the quantile iterator, whose J(a, b, a) = b holds bit for bit, an
iteration that skips slices n < k gives the macroscopic states, the fine end
states and the carried weights of the full iteration bit for bit, for every
matching and schedule, through iteration K + 1; with the additive iterator
they agree within rounding."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1912_09240_gb300 import build as b
    b.build()
    from paper_1912_09240_gb300 import _lib
    return _lib


def _solver(L, w, matching, chunk, skip, iterator=0, precision=None):
    from paper_1912_09240_gb300.parareal import PararealSolver
    precision = L.PR_F32 if precision is None else precision
    model = L.Model(w.kind, w.fast_dim, w.lam, w.beta, w.eps, w.tau_x)
    s = PararealSolver(model, L.Grid(w.bins, w.lo, w.hi), w.N, w.K, w.steps, w.step_dt, precision=precision,
                       rng=L.Rng(w.seed, 0), chunk=chunk, matching=matching, iterator=iterator,
                       skip_converged=skip)
    x0, y0 = workloads.initial_ensemble(w)
    dt = torch.float32 if precision == L.PR_F32 else torch.float64
    s.set_initial(torch.tensor(x0, dtype=dt, device="cuda"), torch.tensor(y0, dtype=dt, device="cuda"))
    return s


@pytest.mark.parametrize("matching", ["quantile", "resample", "resample_det", "reweight"])
@pytest.mark.parametrize("chunk", [0, 1, 3])
def test_skip_equals_full_iterations(L, matching, chunk):
    w = workloads.DOUBLE_WELL.scaled(N=5003, K=7, T=0.07, dt=1e-3, bins=96)
    full = _solver(L, w, matching, chunk, False)
    skip = _solver(L, w, matching, chunk, True)
    for k in range(1, w.K + 3):
        full.iterate()
        skip.iterate()
        np.testing.assert_array_equal(skip.rho.cpu().numpy(), full.rho.cpu().numpy(), err_msg=f"rho k={k}")
        xf, yf, _ = full.state()
        xs, ys, _ = skip.state()
        assert torch.equal(xs, xf), k
        assert torch.equal(ys, yf), k
        if matching == "reweight":
            assert torch.equal(skip.weights(), full.weights()), k
    # slice n is propagated in iterations 0..n only, so fewer library launches
    assert skip.launches < full.launches
    assert int(skip.status.item()) == 0
    full.close()
    skip.close()


def test_skip_with_additive_iterator(L):
    """Additive iterator (J(a, b, a) = b only within rounding on the GPU):
    the macroscopic states stay within rounding of the full iterations."""
    w = workloads.DOUBLE_WELL.scaled(N=4001, K=6, T=0.06, dt=1e-3, bins=80)
    full = _solver(L, w, "quantile", 2, False, iterator=L.PR_ITER_ADD)
    skip = _solver(L, w, "quantile", 2, True, iterator=L.PR_ITER_ADD)
    wv = torch.empty(w.K + 1, dtype=torch.float64, device="cuda")
    for k in range(1, w.K + 2):
        full.iterate()
        skip.iterate()
        L.pr_w1(L.Grid(w.bins, w.lo, w.hi), w.K + 1, skip.rho, full.rho, wv)
        assert float(wv.max().item()) <= 1e-6, k
    full.close()
    skip.close()


def test_skip_fp64_and_run_to_tolerance(L):
    """Binary64 states, sequential schedule: run(tol) stops at the same
    iteration with the same states as the full iterations."""
    w = workloads.OU_SMALL.scaled(K=8, iters=4)
    full = _solver(L, w, "quantile", 0, False, precision=L.PR_F64)
    skip = _solver(L, w, "quantile", 0, True, precision=L.PR_F64)
    kf = full.run(1e-3)
    ks = skip.run(1e-3)
    assert kf == ks
    np.testing.assert_array_equal(skip.rho.cpu().numpy(), full.rho.cpu().numpy())
    assert torch.equal(skip.state()[0], full.state()[0])
    full.close()
    skip.close()


def test_skip_is_not_graph_replayed(L):
    from paper_1912_09240_gb300.parareal import PararealSolver
    w = workloads.OU_SMALL
    with pytest.raises(ValueError):
        PararealSolver(L.Model(w.kind, w.fast_dim, w.lam, w.beta, w.eps, w.tau_x), L.Grid(w.bins, w.lo, w.hi),
                       w.N, w.K, w.steps, w.step_dt, graph=True, skip_converged=True)
