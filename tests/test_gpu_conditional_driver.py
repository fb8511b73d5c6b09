"""The parareal driver with the matchings of Section 5.2 on the GPU: the
exactness theorem bit for bit (sequential, pipelined and graph-replayed
schedules), schedules equal to each other, and whole runs against the FP64
oracle's driver with the same matching."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads

pytestmark = pytest.mark.gpu
MODES = ["resample", "resample_det", "reweight"]


@pytest.fixture(scope="module")
def L():
    from paper_1912_09240_gb300 import build as b
    b.build()
    from paper_1912_09240_gb300 import _lib
    return _lib


def _solver(L, w, precision, matching, chunk=0, graph=False, problem=0):
    from paper_1912_09240_gb300.parareal import PararealSolver
    model = L.Model(w.kind, w.fast_dim, w.lam, w.beta, w.eps, w.tau_x)
    s = PararealSolver(model, L.Grid(w.bins, w.lo, w.hi), w.N, w.K, w.steps, w.step_dt, precision=precision,
                       rng=L.Rng(w.seed, problem), chunk=chunk, graph=graph, matching=matching)
    x0, y0 = workloads.initial_ensemble(w)
    dt = torch.float32 if precision == L.PR_F32 else torch.float64
    s.set_initial(torch.tensor(x0, dtype=dt, device="cuda"), torch.tensor(y0, dtype=dt, device="cuda"))
    return s, x0, y0


@pytest.mark.parametrize("matching", MODES)
@pytest.mark.parametrize("chunk,graph", [(0, False), (2, False), (0, True)])
def test_exactness_theorem_conditional(L, matching, chunk, graph):
    w = workloads.DOUBLE_WELL.scaled(N=6007, K=6, T=0.06, dt=1e-3, bins=128)
    s, _, _ = _solver(L, w, L.PR_F32, matching, chunk, graph)
    xs, ys, rs = s.serial_reference()
    rs_ = rs.cpu().numpy()
    xs_ = xs.cpu().numpy()
    for k in range(1, w.K + 1):
        s.iterate()
        rho = s.rho.cpu().numpy()
        xa = s.state()[0].cpu().numpy()
        for n in range(k + 1):
            np.testing.assert_array_equal(rho[n], rs_[n], err_msg=f"k={k} n={n}")
        for n in range(1, k + 1):
            np.testing.assert_array_equal(xa[n - 1], xs_[n], err_msg=f"k={k} n={n}")
        if matching == "reweight":
            wts = s.weights().cpu().numpy()
            assert np.all(wts[:k] == 1.0 / w.N)
    assert int(s.status.item()) == 0
    s.close()


@pytest.mark.parametrize("matching", MODES)
def test_schedules_agree(L, matching):
    """Pipelined (chunks of 3) and graph-replayed iterations equal the
    sequential driver bit for bit, over several iterations."""
    w = workloads.DOUBLE_WELL.scaled(N=5003, K=8, T=0.08, dt=1e-3, bins=96)
    runs = []
    for chunk, graph in [(0, False), (3, False), (3, True)]:
        s, _, _ = _solver(L, w, L.PR_F32, matching, chunk, graph)
        out = []
        for _ in range(4):
            s.iterate()
            out.append((s.rho.cpu().numpy().copy(), s.state()[0].cpu().numpy().copy()))
        runs.append(out)
        s.close()
    for other in runs[1:]:
        for (r0, x0), (r1, x1) in zip(runs[0], other):
            np.testing.assert_array_equal(r0, r1)
            np.testing.assert_array_equal(x0, x1)


@pytest.mark.parametrize("matching", MODES)
def test_fp64_runs_against_oracle(L, orc, matching):
    """The plain FP64 OU workload shape (N = 4096, K = 8, 256 bins) through 3
    iterations against the oracle's driver with the same matching: W1 between
    the macroscopic states <= 1e-3 at every slice (a particle whose bin or
    selection flips on the last bit of a transcendental moves mass 1/N)."""
    w = workloads.OU_SMALL.scaled(iters=3)
    s, x0, y0 = _solver(L, w, L.PR_F64, matching)
    om = orc.Model(w.kind, w.fast_dim, w.lam, w.beta, w.eps, w.tau_x)
    og = orc.Grid(w.bins, w.lo, w.hi)
    ref = orc.parareal(om, og, w.seed, x0, y0, w.K, w.steps, w.step_dt, iters=w.iters, matching=matching)
    worst = 0.0
    for k in range(w.iters + 1):
        if k:
            s.iterate()
        rho = s.rho.cpu().numpy()
        worst = max(worst, max(orc.w1(og, rho[n], ref.rho[k][n]) for n in range(w.K + 1)))
    assert worst <= 1e-3, worst
    assert int(s.status.item()) == 0
    s.close()
