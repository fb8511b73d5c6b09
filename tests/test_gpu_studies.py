"""The convergence-study harness (Section 6) on the chemical system: the L2
and W1 error arrays it computes on the GPU equal the oracle's evaluation of
the same macroscopic states against the same reference, and the reference
(serial fine solution with ten times the particles, binary32) agrees with
the oracle's serial run of the same particles within the binary32 whole-run
tolerance of that grid (W1 <= 1e-3 * 512/6, see test_gpu_chem.py)."""
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


@pytest.mark.parametrize("iterator,matching", [(0, "quantile"), (1, "resample"), (2, "reweight")])
def test_study_errors_equal_oracle_evaluation(L, orc, iterator, matching):
    from paper_1912_09240_gb300.studies import ConvergenceStudy
    w = workloads.CHEM.scaled(N=2000, K=5, T=10.0)
    extra = workloads.CHEM.scaled(N=9 * w.N)
    x0, y0 = workloads.initial_ensemble(w)
    xe, ye = workloads.initial_ensemble(extra, seed=w.seed + 1)
    xr, yr = np.concatenate([x0, xe]), np.concatenate([y0, ye], axis=1)
    gm = L.Model(w.kind, 1, 0.0, 1.0, w.eps, w.tau_x, w.rates)
    grid = L.Grid(w.bins, w.lo, w.hi)
    st = ConvergenceStudy(gm, grid, w.K, w.steps, w.step_dt, x0, y0, xr, yr, seed=w.seed)
    res = st.run(3, iterator=iterator, matching=matching, keep_states=True)
    assert res["status"] == 0
    og = orc.Grid(w.bins, w.lo, w.hi)
    ref = st.ref.cpu().numpy()
    states = res["states"].numpy()
    l2 = np.array([[orc.l2_density(og, states[k][n], ref[n]) for n in range(w.K + 1)] for k in range(4)])
    w1 = np.array([[orc.w1(og, states[k][n], ref[n]) for n in range(w.K + 1)] for k in range(4)])
    np.testing.assert_allclose(res["l2"].numpy(), l2, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(res["w1"].numpy(), w1, rtol=1e-12, atol=1e-15)
    # the reference against the oracle's serial fine run of the same 10 N particles
    om = orc.Model(w.kind, 1, eps=w.eps, tau_x=w.tau_x, rates=w.rates)
    x = xr.astype(np.float32).astype(np.float64)[None]
    y = yr.astype(np.float32).astype(np.float64)[None]
    for n in range(w.K):
        x, y = orc.fine_propagate(om, w.seed, x, y, n, w.steps, w.step_dt)
        c = orc.restrict(x, og)[1][0]
        assert orc.w1(og, ref[n + 1], c) <= 1e-3 * 512 / 6
