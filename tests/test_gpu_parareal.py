"""Whole micro-macro parareal runs on the GPU against the FP64 oracle, the
exactness theorem on the GPU itself, and sampled per-particle parity at the
full double-well size (2^20 particles, 50 slices of 1000 steps) in the same
launch configuration as bench.py."""
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


def _solver(L, w, precision, iterator=0, qmode=0):
    from paper_1912_09240_gb300.parareal import PararealSolver
    model = L.Model(w.kind, w.fast_dim, w.lam, w.beta, w.eps, w.tau_x)
    grid = L.Grid(w.bins, w.lo, w.hi)
    s = PararealSolver(model, grid, w.N, w.K, w.steps, w.step_dt, precision=precision,
                       rng=L.Rng(w.seed, 0), iterator=iterator, qmode=qmode)
    x0, y0 = workloads.initial_ensemble(w)
    dt = torch.float32 if precision == L.PR_F32 else torch.float64
    s.set_initial(torch.tensor(x0, dtype=dt, device="cuda"), torch.tensor(y0, dtype=dt, device="cuda"))
    return s, x0, y0


def _oracle_objs(orc, w):
    return (orc.Model(w.kind, w.fast_dim, w.lam, w.beta, w.eps, w.tau_x), orc.Grid(w.bins, w.lo, w.hi))


def test_ou_fp64_full_workload_against_oracle(L, orc):
    """The plain FP64 workload in full: N = 4096, K = 8, dt = 1e-3, 256 bins, 4 iterations."""
    w = workloads.OU_SMALL
    s, x0, y0 = _solver(L, w, L.PR_F64)
    om, og = _oracle_objs(orc, w)
    ref = orc.parareal(om, og, w.seed, x0, y0, w.K, w.steps, w.step_dt, iters=w.iters)
    rho = [s.rho.cpu().numpy().copy()]
    for _ in range(w.iters):
        s.iterate()
        rho.append(s.rho.cpu().numpy().copy())
    worst = max(orc.w1(og, rho[k][n], ref.rho[k][n]) for k in range(w.iters + 1) for n in range(w.K + 1))
    assert worst <= 1e-4, worst
    # per-particle: the fine end states of the last iteration
    xs_gpu = s.xa.cpu().numpy()
    xbar_ref, _ = orc.fine_propagate(om, w.seed, ref.x[w.iters - 1][: w.K], ref.y[w.iters - 1][: w.K], 0,
                                     w.steps, w.step_dt)
    assert np.max(np.abs(xs_gpu - xbar_ref)) <= 1e-5
    s.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("qmode", [0])
def test_exactness_theorem_on_gpu(L, orc, prec, qmode):
    """Iterate k equals the serial fine solution on slices n <= k, bit for bit."""
    w = workloads.DOUBLE_WELL.scaled(N=20_000, K=6, T=0.06, dt=1e-4, bins=256)
    precision = L.PR_F64 if prec == "f64" else L.PR_F32
    s, x0, y0 = _solver(L, w, precision, qmode=qmode)
    xs, ys, rs = s.serial_reference()
    for k in range(1, w.K + 1):
        s.iterate()
        torch.cuda.synchronize()
        rho = s.rho.cpu().numpy()
        rs_ = rs.cpu().numpy()
        for n in range(k + 1):
            np.testing.assert_array_equal(rho[n], rs_[n])
        xa = s.xa.cpu().numpy()
        xsn = xs.cpu().numpy()
        for n in range(1, k + 1):
            np.testing.assert_array_equal(xa[n - 1], xsn[n])
    s.close()


def test_double_well_fp32_small_against_oracle(L, orc):
    """FP32 path against the FP64 oracle by W1 of the restricted densities."""
    w = workloads.DOUBLE_WELL.scaled(N=1 << 14, K=5, T=0.05, dt=1e-4, bins=512, iters=3)
    s, x0, y0 = _solver(L, w, L.PR_F32)
    om, og = _oracle_objs(orc, w)
    ref = orc.parareal(om, og, w.seed, x0.astype(np.float32).astype(np.float64),
                       y0.astype(np.float32).astype(np.float64), w.K, w.steps, w.step_dt, iters=w.iters)
    worst = 0.0
    for k in range(1, w.iters + 1):
        s.iterate()
        rho = s.rho.cpu().numpy()
        worst = max(worst, max(orc.w1(og, rho[n], ref.rho[k][n]) for n in range(w.K + 1)))
    assert worst <= 1e-3, worst
    s.close()


@pytest.mark.parametrize("iterator", [1, 2, 3])
def test_other_iterators_run_and_converge(L, orc, iterator):
    w = workloads.OU_SMALL.scaled(N=2048, K=4, T=0.5, iters=4)
    s, x0, y0 = _solver(L, w, L.PR_F64, iterator=iterator)
    _, _, rs = s.serial_reference()
    for _ in range(w.K):
        s.iterate()
    torch.cuda.synchronize()
    w1 = s.w1_to(rs).cpu().numpy()
    assert np.max(w1) < 1e-12
    assert int(s.status.item()) == 0
    s.close()


def test_full_size_double_well_sampled_parity(L, orc):
    """2^20 particles x 50 slices x 1000 steps, FP32, as bench.py runs it: one
    parareal iteration from the zeroth (coarse sweep + matching against X_0);
    sampled particles of several slices against the oracle run on those
    particles only (their own Philox keys)."""
    w = workloads.DOUBLE_WELL
    s, x0, y0 = _solver(L, w, L.PR_F32)
    s.iterate()
    torch.cuda.synchronize()
    xbar = s.xa.cpu().numpy()          # Xbar_0^{n+1} = F_n(X_0^n)
    om, og = _oracle_objs(orc, w)
    x0f = x0.astype(np.float32).astype(np.float64)
    y0f = y0.astype(np.float32).astype(np.float64)
    _, cdf0 = orc.restrict(x0f[None], og)
    P = orc.coarse_propagator(om, og, w.slice_dt)
    rho = [cdf0[0]]
    for n in range(w.K):
        rho.append(orc.coarse_apply(P, rho[-1])[0])
    rng = np.random.default_rng(0)
    ids = np.sort(rng.choice(w.N, 256, replace=False)).astype(np.uint32)
    ids[0], ids[-1] = 0, w.N - 1
    for n in (0, 1, 17, 49):
        start = x0f[ids] if n == 0 else orc.match(x0f[ids][None], og, cdf0, rho[n][None])[0]
        ox, _ = orc.fine_propagate(om, w.seed, start[None], y0f[:, ids][None], n, w.steps, w.step_dt, ids=ids)
        got = xbar[n, ids].astype(np.float64)
        assert np.all(np.abs(got - ox[0]) <= 2e-3 * np.maximum(np.abs(ox[0]), 1.0)), n
    # coarse sweep of iteration 0 matches the oracle's
    s2, _, _ = _solver(L, w, L.PR_F32)
    r0 = s2.rho.cpu().numpy()
    np.testing.assert_allclose(r0, np.stack(rho), rtol=0, atol=1e-11)
    s.close()
    s2.close()


@pytest.mark.parametrize("chunk", [1, 3, 7])
def test_pipelined_driver_equals_sequential(L, chunk):
    """Chunked fine launches on two streams with the serial sweep on a third
    (hidden behind the fine work) give the sequential driver's results bit for
    bit, over several iterations and a second run."""
    w = workloads.DOUBLE_WELL.scaled(N=3001, K=10, T=0.1, dt=1e-3, bins=128)
    ref, x0, y0 = _solver(L, w, L.PR_F32)
    rho_ref, xa_ref = [], []
    for _ in range(4):
        ref.iterate()
        rho_ref.append(ref.rho.cpu().numpy().copy())
        xa_ref.append(ref.xa.cpu().numpy().copy())
    ref.close()
    from paper_1912_09240_gb300.parareal import PararealSolver
    model = L.Model(w.kind, w.fast_dim, w.lam, w.beta, w.eps, w.tau_x)
    s = PararealSolver(model, L.Grid(w.bins, w.lo, w.hi), w.N, w.K, w.steps, w.step_dt, precision=L.PR_F32,
                       rng=L.Rng(w.seed, 0), chunk=chunk)
    for run in range(2):
        s.set_initial(torch.tensor(x0, dtype=torch.float32, device="cuda"),
                      torch.tensor(y0, dtype=torch.float32, device="cuda"))
        for k in range(4):
            s.iterate()
            if run == 1 or k == 3:
                np.testing.assert_array_equal(s.rho.cpu().numpy(), rho_ref[k])
                np.testing.assert_array_equal(s.state()[0].cpu().numpy(), xa_ref[k])
    assert int(s.status.item()) == 0
    s.close()


@pytest.mark.parametrize("chunk", [0, 3])
def test_host_buffer_path_equals_device_path(L, chunk):
    """set_initial_host (X_0, Y_0 copied from page-locked host memory by
    pr_copy_to_device) and rho_to_host (pr_copy_to_host, then
    pr_stream_synchronize) give the device path's macroscopic states bit for
    bit, after the zeroth iteration (in the pipelined schedule, the zeroth
    sweep chunk by chunk) and after two iterations."""
    w = workloads.DOUBLE_WELL.scaled(N=3001, K=10, T=0.1, dt=1e-3, bins=128)
    ref, x0, y0 = _solver(L, w, L.PR_F32)
    rho_ref = [ref.rho.cpu().numpy().copy()]
    for _ in range(2):
        ref.iterate()
        rho_ref.append(ref.rho.cpu().numpy().copy())
    ref.close()
    from paper_1912_09240_gb300.parareal import PararealSolver
    model = L.Model(w.kind, w.fast_dim, w.lam, w.beta, w.eps, w.tau_x)
    s = PararealSolver(model, L.Grid(w.bins, w.lo, w.hi), w.N, w.K, w.steps, w.step_dt, precision=L.PR_F32,
                       rng=L.Rng(w.seed, 0), chunk=chunk)
    xh = torch.tensor(x0, dtype=torch.float32).pin_memory()
    yh = torch.tensor(y0, dtype=torch.float32).pin_memory()
    out = torch.empty(w.K + 1, w.bins + 1, dtype=torch.float64).pin_memory()
    for run in range(2):
        s.set_initial_host(xh, yh)
        s.rho_to_host(out)
        L.pr_stream_synchronize()
        np.testing.assert_array_equal(out.numpy(), rho_ref[0])
        for k in range(2):
            s.iterate()
            s.rho_to_host(out)
            L.pr_stream_synchronize()
            np.testing.assert_array_equal(out.numpy(), rho_ref[k + 1])
    s.close()


@pytest.mark.parametrize("chunk", [0, 2])
def test_exactness_theorem_fast16_on_gpu(L, chunk):
    """The 16-dimensional fast space (coupling lambda mean(y)): iterate k equals
    the serial fine solution on slices n <= k, bit for bit, with the sequential
    and the pipelined driver."""
    from paper_1912_09240_gb300.parareal import PararealSolver
    w = workloads.LARGE_FAST.scaled(N=5003, K=5, T=5e-3, bins=1024)
    model = L.Model(w.kind, w.fast_dim, w.lam, w.beta, w.eps, w.tau_x)
    s = PararealSolver(model, L.Grid(w.bins, w.lo, w.hi), w.N, w.K, w.steps, w.step_dt, precision=L.PR_F32,
                       rng=L.Rng(w.seed, 3), chunk=chunk)
    x0, y0 = workloads.initial_ensemble(w)
    s.set_initial(torch.tensor(x0, dtype=torch.float32, device="cuda"),
                  torch.tensor(y0, dtype=torch.float32, device="cuda"))
    xs, ys, rs = s.serial_reference()
    rs_ = rs.cpu().numpy()
    for k in range(1, w.K + 1):
        s.iterate()
        rho = s.rho.cpu().numpy()
        for n in range(k + 1):
            np.testing.assert_array_equal(rho[n], rs_[n])
        xa, ya, _ = s.state()
        for n in range(1, k + 1):
            np.testing.assert_array_equal(xa[n - 1].cpu().numpy(), xs[n].cpu().numpy())
            np.testing.assert_array_equal(ya[n - 1].cpu().numpy(), ys[n].cpu().numpy())
    assert int(s.status.item()) == 0
    s.close()


def test_fast16_full_size_sampled_parity(L, orc):
    """4e6 particles x 100 slices x 1000 steps with a 16-dimensional fast
    space, 1024 bins, binary32, pipelined as bench.py runs it: the first
    parareal iteration (every slice matched from X_0 to the coarse sweep);
    sampled particles of several slices, all 17 coordinates, against the
    oracle run on those particles only (their own Philox keys)."""
    from paper_1912_09240_gb300.parareal import PararealSolver
    w = workloads.LARGE_FAST
    model = L.Model(w.kind, w.fast_dim, w.lam, w.beta, w.eps, w.tau_x)
    grid = L.Grid(w.bins, w.lo, w.hi)
    s = PararealSolver(model, grid, w.N, w.K, w.steps, w.step_dt, precision=L.PR_F32, rng=L.Rng(w.seed, 0),
                       chunk=5)
    x0 = workloads.initial_slow(w)
    x0t = torch.tensor(x0, dtype=torch.float32, device="cuda")
    s.set_initial(x0t, x0t.expand(w.fast_dim, w.N).contiguous())
    rho0 = s.rho.cpu().numpy().copy()
    s.iterate()
    xa, ya, _ = s.state()
    rng = np.random.default_rng(5)
    ids = np.sort(rng.choice(w.N, 128, replace=False)).astype(np.uint32)
    ids[0], ids[-1] = 0, w.N - 1
    om, og = _oracle_objs(orc, w)
    x0f = x0.astype(np.float32).astype(np.float64)
    _, cdf0 = orc.restrict(x0f[None], og)
    np.testing.assert_array_equal(rho0[0], cdf0[0])
    for n in (0, 1, 42, 99):
        start = x0f[ids] if n == 0 else orc.match(x0f[ids][None], og, cdf0, rho0[n][None])[0]
        ystart = np.repeat(x0f[ids][None], w.fast_dim, axis=0)
        ox, oy = orc.fine_propagate(om, w.seed, start[None], ystart[None], n, w.steps, w.step_dt, ids=ids)
        gx = xa[n][torch.from_numpy(ids.astype(np.int64)).cuda()].double().cpu().numpy()
        gy = ya[n][:, torch.from_numpy(ids.astype(np.int64)).cuda()].double().cpu().numpy()
        assert np.all(np.abs(gx - ox[0]) <= 2e-3 * np.maximum(np.abs(ox[0]), 1.0)), n
        assert np.all(np.abs(gy - oy[0]) <= 2e-3 * np.maximum(np.abs(oy[0]), 1.0)), n
    assert int(s.status.item()) == 0
    s.close()


@pytest.mark.parametrize("chunk", [0, 3])
def test_graph_mode_equals_eager(L, chunk):
    """Iterations replayed as CUDA graphs give the eager sequential driver's
    results bit for bit, for both bindings of the double buffers (a second run
    starts after an odd number of iterations)."""
    from paper_1912_09240_gb300.parareal import PararealSolver
    w = workloads.DOUBLE_WELL.scaled(N=3001, K=10, T=0.1, dt=1e-3, bins=128)
    ref, x0, y0 = _solver(L, w, L.PR_F32)
    rho_ref, xa_ref = [], []
    for _ in range(5):
        ref.iterate()
        rho_ref.append(ref.rho.cpu().numpy().copy())
        xa_ref.append(ref.xa.cpu().numpy().copy())
    ref.close()
    model = L.Model(w.kind, w.fast_dim, w.lam, w.beta, w.eps, w.tau_x)
    s = PararealSolver(model, L.Grid(w.bins, w.lo, w.hi), w.N, w.K, w.steps, w.step_dt, precision=L.PR_F32,
                       rng=L.Rng(w.seed, 0), chunk=chunk, graph=True)
    for iters in (3, 5):
        s.set_initial(torch.tensor(x0, dtype=torch.float32, device="cuda"),
                      torch.tensor(y0, dtype=torch.float32, device="cuda"))
        for k in range(iters):
            s.iterate()
            np.testing.assert_array_equal(s.rho.cpu().numpy(), rho_ref[k])
            np.testing.assert_array_equal(s.state()[0].cpu().numpy(), xa_ref[k])
    assert all(g is not None for g in s._graphs)
    assert int(s.status.item()) == 0
    s.close()


@pytest.mark.parametrize("K", [1, 2])
@pytest.mark.parametrize("chunk,graph", [(0, False), (1, False), (5, False), (0, True), (5, True)])
def test_driver_with_one_or_two_slices(L, K, chunk, graph):
    """One and two slices, chunks larger than the horizon, eager and graph
    replay: every schedule equals the sequential one bit for bit, and after
    iteration k the slices n <= k equal the serial fine solution (the
    exactness theorem), so iteration K is the serial solution itself."""
    from paper_1912_09240_gb300.parareal import PararealSolver
    w = workloads.DOUBLE_WELL.scaled(N=2049, K=K, T=0.02 * K, dt=1e-3, bins=64)
    model = L.Model(w.kind, w.fast_dim, w.lam, w.beta, w.eps, w.tau_x)
    x0, y0 = workloads.initial_ensemble(w)
    gx, gy = (torch.tensor(v, dtype=torch.float32, device="cuda") for v in (x0, y0))

    def run(ch, gr):
        s = PararealSolver(model, L.Grid(w.bins, w.lo, w.hi), w.N, w.K, w.steps, w.step_dt, precision=L.PR_F32,
                           rng=L.Rng(w.seed, 0), chunk=ch, graph=gr)
        s.set_initial(gx, gy)
        rho = []
        for _ in range(K + 2):
            s.iterate()
            rho.append(s.rho.cpu().numpy().copy())
        _, _, rser = s.serial_reference()
        assert int(s.status.item()) == 0
        s.close()
        return rho, rser.cpu().numpy()

    ref, rser = run(0, False)
    got, _ = run(chunk, graph)
    for k in range(K + 2):
        np.testing.assert_array_equal(got[k], ref[k], err_msg=f"k={k}")
    for j in range(K + 2):             # got[j] is iterate k = j + 1
        for n in range(min(j + 1, K) + 1):
            np.testing.assert_array_equal(got[j][n], rser[n], err_msg=f"k={j + 1} n={n}")


@pytest.mark.parametrize("chunk,graph", [(0, False), (3, False), (3, True)])
def test_increment_and_run(L, orc, chunk, graph):
    """increment() is W1 between consecutive macroscopic iterates (checked
    against the oracle's W1 on the host), it vanishes from iteration K + 1
    on (the exactness theorem), and run(tol) stops at the first iteration
    whose increment is within tol."""
    from paper_1912_09240_gb300.parareal import PararealSolver
    w = workloads.DOUBLE_WELL.scaled(N=4099, K=6, T=0.06, dt=1e-3, bins=96)
    model = L.Model(w.kind, w.fast_dim, w.lam, w.beta, w.eps, w.tau_x)
    x0, y0 = workloads.initial_ensemble(w)
    gx, gy = (torch.tensor(v, dtype=torch.float32, device="cuda") for v in (x0, y0))
    og = orc.Grid(w.bins, w.lo, w.hi)
    s = PararealSolver(model, L.Grid(w.bins, w.lo, w.hi), w.N, w.K, w.steps, w.step_dt, precision=L.PR_F32,
                       rng=L.Rng(w.seed, 0), chunk=chunk, graph=graph)
    s.set_initial(gx, gy)
    prev = s.rho.cpu().numpy().copy()
    incs = []
    for k in range(1, w.K + 2):
        s.iterate()
        cur = s.rho.cpu().numpy().copy()
        inc = s.increment().cpu().numpy()
        ref = np.array([orc.w1(og, cur[n], prev[n]) for n in range(w.K + 1)])
        np.testing.assert_allclose(inc, ref, rtol=1e-12, atol=1e-15)
        incs.append(inc.max())
        prev = cur
    assert incs[-1] == 0.0 and incs[0] > 0.0
    tol = sorted(incs)[len(incs) // 2]
    s.set_initial(gx, gy)
    k = s.run(tol)
    assert k == next(i + 1 for i, v in enumerate(incs) if v <= tol)
    s.close()
