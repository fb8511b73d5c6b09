"""Batched serving (pr_batch_*) against single-problem runs: a problem p of a
batch draws the numbers of pr_rng{seed, p}, takes the same fused fine steps
and the same serial update, so its macroscopic states and fine states equal
a PararealSolver run of that problem alone, bit for bit -- through the
eager zeroth iteration, the graph-replayed iterations of both parities, a
second run after set_initial, and re-tuned scheduling."""
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


def _problems(L):
    return [
        L.Problem(L.Model(0, 1, 1.0, 1.0, 0.1), L.Grid(64, -4.0, 4.0), 1000, 4, 31, 1e-3, 7),
        L.Problem(L.Model(1, 1, 0.5, 3.0, 0.02), L.Grid(256, -3.0, 3.0), 5003, 3, 100, 2e-4, 7),
        L.Problem(L.Model(0, 1, 0.3, 2.0, 0.05), L.Grid(32, -4.0, 4.0), 333, 5, 7, 1e-3, 9),
        L.Problem(L.Model(1, 1, 0.2, 1.0, 0.1), L.Grid(128, -2.5, 3.5), 20000, 2, 55, 5e-4, 3),
    ]


def _inits(probs):
    xs, ys = [], []
    for i, p in enumerate(probs):
        rng = np.random.default_rng(100 + i)
        x = rng.normal(-0.5 if p.model.kind else 1.0, 0.3, p.n).astype(np.float32)
        xs.append(x)
        ys.append((x + rng.normal(0, 0.5, p.n)).astype(np.float32))
    return xs, ys


def _single(L, p, idx, x0, y0, iters):
    from paper_1912_09240_gb300.parareal import PararealSolver
    s = PararealSolver(p.model, p.grid, p.n, p.n_slices, p.steps, p.dt, precision=L.PR_F32,
                       rng=L.Rng(p.seed, idx))
    s.set_initial(torch.tensor(x0, device="cuda"), torch.tensor(y0, device="cuda").reshape(1, -1))
    out = [s.rho.cpu().numpy().copy()]
    for _ in range(iters):
        s.iterate()
        out.append(s.rho.cpu().numpy().copy())
    xa = s.xa.cpu().numpy().copy()
    s.close()
    return out, xa


def test_batch_equals_single_problem_runs(L):
    from paper_1912_09240_gb300.batch import BatchSolver
    probs = _problems(L)
    xs, ys = _inits(probs)
    iters = 4
    b = BatchSolver(probs)
    ref = [_single(L, p, i, xs[i], ys[i], iters) for i, p in enumerate(probs)]
    for run in range(2):                      # the second run replays the captured graphs
        b.set_initial(xs, ys)
        for i in range(len(probs)):
            np.testing.assert_array_equal(b.rho(i).cpu().numpy(), ref[i][0][0])
        for k in range(1, iters + 1):
            b.iterate()
            for i in range(len(probs)):
                np.testing.assert_array_equal(b.rho(i).cpu().numpy(), ref[i][0][k], err_msg=f"run {run} k {k} p {i}")
        for i in range(len(probs)):
            np.testing.assert_array_equal(b.fine_state(i)[0].cpu().numpy(), ref[i][1])
    assert b.status() == 0
    b.close()


def test_tuning_changes_nothing_but_speed(L):
    from paper_1912_09240_gb300.batch import BatchSolver
    probs = _problems(L)
    xs, ys = _inits(probs)
    b = BatchSolver(probs)
    b.set_initial(xs, ys)
    for _ in range(2):
        b.iterate()
    before = [b.rho(i).cpu().numpy().copy() for i in range(len(probs))]
    ms = b.tune(steps_div=4)
    assert ms > 0.0
    ppt, work, items = b.config()
    assert ppt in (1, 2, 4) and work >= 1.0 and items >= sum(p.n_slices for p in probs)
    b.set_initial(xs, ys)
    for _ in range(2):
        b.iterate()
    for i in range(len(probs)):
        np.testing.assert_array_equal(b.rho(i).cpu().numpy(), before[i])
    for ppt in (1, 2):
        b.set_config(ppt, 5e4)
        b.set_initial(xs, ys)
        for _ in range(2):
            b.iterate()
        for i in range(len(probs)):
            np.testing.assert_array_equal(b.rho(i).cpu().numpy(), before[i])
    b.close()


def test_batched_workload_shape(L):
    """The 64-problem batched workload (eps log-uniform in [1e-3, 1e-1], lambda
    uniform in [0, 1], particle counts log-uniform in [1e4, 1e6], 32 slices,
    dt = eps/50) with particle counts scaled by 1/20: two iterations, three
    problems checked against single runs."""
    from paper_1912_09240_gb300.batch import BatchSolver
    bw = workloads.batched_problems()
    probs, xs, ys = [], [], []
    for w in bw.problems:
        n = max(500, w.N // 20)
        probs.append(L.Problem(L.Model(w.kind, 1, w.lam, w.beta, w.eps), L.Grid(w.bins, w.lo, w.hi), n, w.K,
                               w.steps, w.step_dt, w.seed))
        x0, y0 = workloads.initial_ensemble(w.scaled(N=n))
        xs.append(x0.astype(np.float32))
        ys.append(y0[0].astype(np.float32))
    b = BatchSolver(probs)
    b.set_initial(xs, ys)
    for _ in range(2):
        b.iterate()
    assert b.status() == 0
    for i in (0, 17, 63):
        ref, _ = _single(L, probs[i], i, xs[i], ys[i], 2)
        np.testing.assert_array_equal(b.rho(i).cpu().numpy(), ref[2])
    b.close()


def test_batch_with_tiny_problems(L):
    """Problems at the small end beside an ordinary one: one particle, one
    slice, a single bin, an odd number of steps; each equals its
    single-problem run bit for bit over three iterations."""
    from paper_1912_09240_gb300.batch import BatchSolver
    probs = [
        L.Problem(L.Model(0, 1, 1.0, 1.0, 0.1), L.Grid(64, -4.0, 4.0), 1, 3, 11, 1e-3, 5),
        L.Problem(L.Model(1, 1, 0.5, 3.0, 0.05), L.Grid(48, -3.0, 3.0), 777, 1, 20, 1e-3, 5),
        L.Problem(L.Model(0, 1, 0.5, 2.0, 0.1), L.Grid(1, -4.0, 4.0), 300, 3, 9, 1e-3, 6),
        L.Problem(L.Model(1, 1, 0.2, 1.0, 0.1), L.Grid(128, -2.5, 3.5), 4099, 4, 13, 5e-4, 3),
    ]
    xs, ys = _inits(probs)
    iters = 3
    b = BatchSolver(probs)
    ref = [_single(L, p, i, xs[i], ys[i], iters) for i, p in enumerate(probs)]
    b.set_initial(xs, ys)
    for k in range(1, iters + 1):
        b.iterate()
        for i in range(len(probs)):
            np.testing.assert_array_equal(b.rho(i).cpu().numpy(), ref[i][0][k], err_msg=f"k {k} p {i}")
    for i in range(len(probs)):
        np.testing.assert_array_equal(b.fine_state(i)[0].cpu().numpy(), ref[i][1])
    assert b.status() == 0
    b.close()


def test_batch_run_to_tolerance(L, orc):
    """BatchSolver.run(tol): stops at the first iteration where every
    problem's change of its macroscopic states is within tol (the increments
    against the oracle's W1 of the host copies), and its states equal those
    of iterating that many times."""
    from paper_1912_09240_gb300.batch import BatchSolver
    probs = _problems(L)
    xs, ys = _inits(probs)
    a = BatchSolver(probs)
    a.set_initial(xs, ys)
    k, inc = a.run(1e-3)
    inc = inc.cpu().numpy()
    assert 1 <= k <= max(p.n_slices for p in probs) + 1
    assert np.all(inc <= 1e-3), inc
    b = BatchSolver(probs)
    b.set_initial(xs, ys)
    for _ in range(k - 1):
        b.iterate()
    before = [b.rho(i).cpu().numpy() for i in range(len(probs))]
    b.iterate()
    for i, p in enumerate(probs):
        after = b.rho(i).cpu().numpy()
        np.testing.assert_array_equal(after, a.rho(i).cpu().numpy())
        og = orc.Grid(p.grid.bins, p.grid.lo, p.grid.hi)
        ref = max(orc.w1(og, after[n], before[i][n]) for n in range(p.n_slices + 1))
        assert abs(ref - inc[i]) <= 1e-12 + 1e-9 * ref, (i, ref, inc[i])
    a.close()
    b.close()
