"""pr_fine_adjoint_noalloc: the adjoint for callers that cannot allocate
device memory while they run (real-time control loops, hosts whose device
memory belongs to another allocator).  Its scratch is a fixed array inside
the library, shared by every call.  Checked against pr_fine_adjoint (which
takes a caller workspace) on two calls in a row, so that a call after
another, finding the array holding the previous call's contents, still
agrees; and a problem larger than the array is refused before it runs.

This file is collected last on purpose: run alone in a fresh process the
array's first use is the first call here; run after the other tests it is
not.  The array's device address is looked up once per device and kept for
the life of the process, so no test here resets the device (a reset would
make that address stale, as the header states)."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    from paper_1912_09240_gb300 import build as b
    b.build()
    from paper_1912_09240_gb300 import _lib
    return _lib


@pytest.mark.gpu
def test_no_alloc_adjoint_matches_workspace_adjoint(L):
    n, sb, slices, steps, ckpt, dt = 3000, 2, 3, 100, 64, 1e-3
    model = L.Model(L.PR_MODEL_DOUBLE_WELL, 1, 0.5, 3.0, 0.05, 1.0)
    rng = L.Rng(11, 4)
    g = np.random.default_rng(12)
    x0 = torch.tensor(g.normal(-1.0, 0.3, n), dtype=torch.float32, device="cuda")
    y0 = torch.tensor(g.normal(-1.0, 0.5, n), dtype=torch.float32, device="cuda")
    seeds = torch.tensor(g.normal(0.0, 1.0, n), dtype=torch.float64, device="cuda")
    assert L.pr_fine_adjoint_workspace(n, slices, steps, ckpt) <= L.pr_fine_adjoint_noalloc_capacity()

    # reference: the entry point with a caller workspace
    ws = torch.empty(L.pr_fine_adjoint_workspace(n, slices, steps, ckpt), dtype=torch.uint8, device="cuda")
    ref_sum = torch.zeros(3, dtype=torch.float64, device="cuda")
    ref_x0bar = torch.empty(n, dtype=torch.float64, device="cuda")
    L.pr_fine_adjoint(model, rng, x0, y0, n, sb, slices, steps, dt, ckpt, None, None, seeds, None, ref_sum,
                      ref_x0bar, None, ws)
    ref_pp = torch.empty(n, 3, dtype=torch.float64, device="cuda")
    ref_xT = torch.empty(n, dtype=torch.float32, device="cuda")
    L.pr_fine_adjoint(model, rng, x0, y0, n, sb, slices, steps, dt, ckpt, ref_xT, None, None, None, ref_pp,
                      None, None, ws)
    torch.cuda.synchronize()

    # two calls in a row through the fixed array: seeded sum, then per particle
    got_sum = torch.zeros(3, dtype=torch.float64, device="cuda")
    got_x0bar = torch.empty(n, dtype=torch.float64, device="cuda")
    L.pr_fine_adjoint_noalloc(model, rng, x0, y0, n, sb, slices, steps, dt, ckpt, None, None, seeds, None,
                              got_sum, got_x0bar, None)
    got_pp = torch.empty(n, 3, dtype=torch.float64, device="cuda")
    got_xT = torch.empty(n, dtype=torch.float32, device="cuda")
    L.pr_fine_adjoint_noalloc(model, rng, x0, y0, n, sb, slices, steps, dt, ckpt, got_xT, None, None, None,
                              got_pp, None, None)
    torch.cuda.synchronize()

    np.testing.assert_allclose(got_sum.cpu().numpy(), ref_sum.cpu().numpy(), rtol=1e-12, atol=0)
    np.testing.assert_allclose(got_x0bar.cpu().numpy(), ref_x0bar.cpu().numpy(), rtol=1e-12, atol=0)
    np.testing.assert_allclose(got_pp.cpu().numpy(), ref_pp.cpu().numpy(), rtol=1e-12, atol=0)
    np.testing.assert_array_equal(got_xT.cpu().numpy(), ref_xT.cpu().numpy())


@pytest.mark.gpu
def test_no_alloc_adjoint_rejects_problems_larger_than_its_array(L):
    cap = L.pr_fine_adjoint_noalloc_capacity()
    n, slices, steps, ckpt = 1 << 20, 20, 1000, 256        # ~632 MiB of checkpoints
    assert L.pr_fine_adjoint_workspace(n, slices, steps, ckpt) > cap
    x = torch.zeros(n, dtype=torch.float32, device="cuda")
    grad = torch.zeros(3, dtype=torch.float64, device="cuda")
    seeds = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(L.PrError) as e:
        L.pr_fine_adjoint_noalloc(L.Model(0), L.Rng(), x, x, n, 0, slices, steps, 1e-4, ckpt, None, None, seeds,
                                  None, grad, None, None)
    assert e.value.code == L.PR_ERR_NOMEM
