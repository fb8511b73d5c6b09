"""Whole parareal runs of the binary32 path at the geometry of the two large
workloads against the FP64 oracle run on the same inputs, by W1 between the
macroscopic states at every slice and iteration (tolerance 1e-3, the bar of
the binary32 path), in the pipelined launch configuration bench.py uses:

* double well: 50 slices x 1000 steps of dt = 1e-4, eps = 1e-2, 512 bins on
  [-3, 3], at 2^16 particles (the bench's 2^20 would take the oracle
  minutes), 3 iterations;
* 16-dimensional fast space: 100 slices x 1000 steps of dt = 1e-5, eps =
  1e-3, 1024 bins on [-3, 3], at 2^11 particles, 2 iterations.

The oracle runs the same algorithm in FP64 from the binary32-rounded
initial ensemble; pathwise the two drift apart near the barrier, so the
comparison is by W1 of the restricted densities, as the parity tolerances
state for long horizons in the double well."""
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


@pytest.mark.parametrize("case", ["double_well_k50_n2^16", "fast16_k100_n2^11"])
def test_binary32_whole_run_at_workload_geometry(L, orc, case):
    from paper_1912_09240_gb300.parareal import PararealSolver
    if case.startswith("double_well"):
        w, iters = workloads.DOUBLE_WELL.scaled(N=1 << 16), 3
    else:
        w, iters = workloads.LARGE_FAST.scaled(N=1 << 11), 2
    assert w.K in (50, 100) and w.steps == 1000
    model = L.Model(w.kind, w.fast_dim, w.lam, w.beta, w.eps, w.tau_x)
    grid = L.Grid(w.bins, w.lo, w.hi)
    x0, y0 = workloads.initial_ensemble(w)
    x0f = x0.astype(np.float32)
    y0f = np.ascontiguousarray(np.broadcast_to(y0, (w.fast_dim, w.N))).astype(np.float32)
    s = PararealSolver(model, grid, w.N, w.K, w.steps, w.step_dt, precision=L.PR_F32, rng=L.Rng(w.seed, 0),
                       chunk=5)
    s.set_initial(torch.tensor(x0f, device="cuda"), torch.tensor(y0f, device="cuda"))
    rho = [s.rho.cpu().numpy().copy()]
    for _ in range(iters):
        s.iterate()
        rho.append(s.rho.cpu().numpy().copy())
    assert int(s.status.item()) == 0
    s.close()
    om = orc.Model(w.kind, w.fast_dim, w.lam, w.beta, w.eps, w.tau_x)
    og = orc.Grid(w.bins, w.lo, w.hi)
    ref = orc.parareal(om, og, w.seed, x0f.astype(np.float64), y0f.astype(np.float64), w.K, w.steps, w.step_dt,
                       iters=iters)
    w1 = np.array([[orc.w1(og, rho[k][n], ref.rho[k][n]) for n in range(w.K + 1)] for k in range(iters + 1)])
    print(f"{case}: max W1 per iteration {w1.max(axis=1)}")
    assert np.all(w1 <= 1e-3), w1.max(axis=1)
