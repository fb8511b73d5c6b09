"""The matching preserving the conditional distribution (Section 5.2) on the
GPU against the FP64 oracle: reweighting, stratified and deterministic
resampling with the gather of the states, and the weighted restriction --
all bit for bit (the cumulative weights are exact integers on both sides)."""
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


def _t(a, dtype=None):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def _case(orc, rng, S, n, bins, lo, hi, f32):
    og = orc.Grid(bins, lo, hi)
    x = rng.normal(0.2, 0.7, (S, n))
    x[:, :4] = [lo - 1.0, hi + 1.0, lo, og.edges()[bins // 3]]
    if f32:
        x = x.astype(np.float32).astype(np.float64)
    _, cp = orc.restrict(x, og)
    m = rng.gamma(2.0, 1.0, (S, bins)) * (rng.random((S, bins)) < 0.75)
    m /= m.sum(axis=1, keepdims=True)
    ct = np.concatenate([np.zeros((S, 1)), np.cumsum(m, axis=1)], axis=1)
    ct[:, -1] = 1.0
    return og, x, cp, ct


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("bins,lo,hi", [(64, -3.0, 3.0), (512, -3.0, 3.0), (37, -1.7, 2.2)])
@pytest.mark.parametrize("with_w", [False, True])
def test_reweight_bit_exact(L, orc, prec, bins, lo, hi, with_w):
    rng = np.random.default_rng(bins + prec)
    S, n = 3, 20011
    og, x, cp, ct = _case(orc, rng, S, n, bins, lo, hi, prec == 0)
    wbar = rng.random((S, n)) / n if with_w else None
    ref = orc.reweight(x, og, cp, ct, wbar)
    dt = torch.float32 if prec == 0 else torch.float64
    out = torch.empty(S, n, dtype=torch.float64, device=DEV)
    L.pr_reweight(prec, _t(x, dt), False, None if wbar is None else _t(wbar), n, S, L.Grid(bins, lo, hi),
                  _t(cp), _t(ct), out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), ref)


def test_reweight_broadcast_and_strong_projection(L, orc):
    rng = np.random.default_rng(3)
    n, S, bins = 4099, 4, 128
    og, x, cp, ct = _case(orc, rng, 1, n, bins, -3.0, 3.0, False)
    cps = np.repeat(cp, S, axis=0)
    cts = np.concatenate([cp, np.repeat(ct, S - 1, axis=0)])   # slice 0: target == prior
    out = torch.empty(S, n, dtype=torch.float64, device=DEV)
    L.pr_reweight(1, _t(x[0]), True, None, n, S, L.Grid(bins, -3.0, 3.0), _t(cps), _t(cts), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.all(got[0] == 1.0 / n)
    np.testing.assert_array_equal(got, orc.reweight(np.repeat(x, S, axis=0), og, cps, cts))


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("n", [1, 5, 2048, 2049, 10007])
def test_resample_bit_exact_and_gather(L, orc, mode, n):
    rng = np.random.default_rng(n + mode)
    S, d = 3, 3
    w = rng.gamma(0.6, 1.0, (S, n)) * (rng.random((S, n)) < 0.8)
    w[:, 0] += 1e-3
    w /= w.sum(axis=1, keepdims=True)
    ref = orc.resample(w, mode, seed=77, slice_begin=5, problem=9)
    x = rng.normal(size=(S, n)).astype(np.float32)
    y = rng.normal(size=(S, d, n)).astype(np.float32)
    idx = torch.empty(S, n, dtype=torch.int32, device=DEV)
    xo = torch.empty(S, n, dtype=torch.float32, device=DEV)
    yo = torch.empty(S, d, n, dtype=torch.float32, device=DEV)
    ws = torch.empty(L.pr_resample_workspace(n, S), dtype=torch.uint8, device=DEV)
    L.pr_resample(0, d, _t(x), _t(y), False, _t(w), n, S, 5, mode, L.Rng(77, 9), idx, xo, yo, ws)
    torch.cuda.synchronize()
    got = idx.cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(got, ref)
    gi = got.astype(np.int64)
    np.testing.assert_array_equal(xo.cpu().numpy(), np.take_along_axis(x, gi, axis=1))
    for s in range(S):
        np.testing.assert_array_equal(yo[s].cpu().numpy(), y[s][:, gi[s]])


@pytest.mark.parametrize("mode", [0, 1])
def test_resample_equal_weights_identity_and_broadcast(L, mode):
    n, S = 30001, 4
    w = torch.full((S, n), 1.0 / n, dtype=torch.float64, device=DEV)
    x0 = torch.randn(n, dtype=torch.float64, device=DEV)
    y0 = torch.randn(1, n, dtype=torch.float64, device=DEV)
    idx = torch.empty(S, n, dtype=torch.int32, device=DEV)
    xo = torch.empty(S, n, dtype=torch.float64, device=DEV)
    yo = torch.empty(S, 1, n, dtype=torch.float64, device=DEV)
    ws = torch.empty(L.pr_resample_workspace(n, S), dtype=torch.uint8, device=DEV)
    L.pr_resample(1, 1, x0, y0, True, w, n, S, 0, mode, L.Rng(1, 0), idx, xo, yo, ws)
    torch.cuda.synchronize()
    ar = torch.arange(n, dtype=torch.int32, device=DEV)
    for s in range(S):
        assert torch.equal(idx[s], ar)
        assert torch.equal(xo[s], x0) and torch.equal(yo[s], y0)


@pytest.mark.parametrize("prec", [0, 1])
def test_restrict_weighted_bit_exact(L, orc, prec):
    rng = np.random.default_rng(11 + prec)
    S, n, bins = 3, 50001, 256
    og = orc.Grid(bins, -3.0, 3.0)
    x = rng.normal(0.0, 1.1, (S, n))
    x[:, :3] = [-7.0, 7.0, 0.0]
    if prec == 0:
        x = x.astype(np.float32).astype(np.float64)
    w = rng.random((S, n))
    w /= w.sum(axis=1, keepdims=True)
    w[1] = 0.0                                   # a slice without weight: the uniform CDF
    ref = orc.restrict_weighted(x, w, og)
    cdf = torch.empty(S, bins + 1, dtype=torch.float64, device=DEV)
    ws = torch.empty(L.pr_restrict_weighted_workspace(S, bins), dtype=torch.uint8, device=DEV)
    dt = torch.float32 if prec == 0 else torch.float64
    L.pr_restrict_weighted(prec, _t(x, dt), False, _t(w), n, S, L.Grid(bins, -3.0, 3.0), cdf, ws)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(cdf.cpu().numpy(), ref)
    # one shared ensemble, per-slice weights
    L.pr_restrict_weighted(prec, _t(x[2], dt), True, _t(w), n, S, L.Grid(bins, -3.0, 3.0), cdf, ws)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(cdf.cpu().numpy(), orc.restrict_weighted(np.repeat(x[2:3], S, axis=0), w, og))


def test_full_size_reweight_resample(L, orc):
    """2^20 binary32 particles x 4 slices, 512 bins, double-well-like state:
    reweighting to a shifted target and stratified resampling, every weight
    and every index against the oracle."""
    rng = np.random.default_rng(21)
    S, n, bins = 4, 1 << 20, 512
    og = orc.Grid(bins, -3.0, 3.0)
    x = np.concatenate([rng.normal(-1.0, 0.3, (S, n // 2)), rng.normal(1.0, 0.3, (S, n - n // 2))], axis=1)
    x = x.astype(np.float32).astype(np.float64)
    _, cp = orc.restrict(x, og)
    _, ct = orc.restrict(x + 0.05 * rng.normal(size=(S, n)), og)
    w_ref = orc.reweight(x, og, cp, ct)
    idx_ref = orc.resample(w_ref, 0, seed=0, slice_begin=1)
    gx = _t(x, torch.float32)
    w = torch.empty(S, n, dtype=torch.float64, device=DEV)
    L.pr_reweight(0, gx, False, None, n, S, L.Grid(bins, -3.0, 3.0), _t(cp), _t(ct), w)
    idx = torch.empty(S, n, dtype=torch.int32, device=DEV)
    ws = torch.empty(L.pr_resample_workspace(n, S), dtype=torch.uint8, device=DEV)
    L.pr_resample(0, 1, None, None, False, w, n, S, 1, 0, L.Rng(0, 0), idx, None, None, ws)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(w.cpu().numpy(), w_ref)
    np.testing.assert_array_equal(idx.cpu().numpy().view(np.uint32), idx_ref)


@pytest.mark.parametrize("prec", [0, 1])
def test_reweight_target_outside_prior_support(L, orc, prec):
    """Target mass only left of, only right of, and on both sides of the
    prior's support (the relocation of Section 5.2's reweighting), with the
    ensemble's own restriction as prior: bit for bit against the oracle, and
    all the weight inside the prior's support."""
    rng = np.random.default_rng(40 + prec)
    bins, lo, hi, n = 96, -4.0, 4.0, 12289
    og = orc.Grid(bins, lo, hi)
    x = rng.normal(0.0, 0.3, (3, n))
    if prec == 0:
        x = x.astype(np.float32).astype(np.float64)
    _, cp = orc.restrict(x, og)
    e = og.edges()
    m = np.zeros((3, bins))
    m[0, e[:-1] < -2.0] = 1.0                      # left of the support only
    m[1, e[1:] > 2.5] = 1.0                        # right of it only
    m[2, (e[:-1] < -2.0) | (e[1:] > 2.5)] = 1.0    # both sides
    m /= m.sum(axis=1, keepdims=True)
    ct = np.concatenate([np.zeros((3, 1)), np.cumsum(m, axis=1)], axis=1)
    ct[:, -1] = 1.0
    ref = orc.reweight(x, og, cp, ct)
    dt = torch.float32 if prec == 0 else torch.float64
    out = torch.empty(3, n, dtype=torch.float64, device=DEV)
    L.pr_reweight(prec, _t(x, dt), False, None, n, 3, L.Grid(bins, lo, hi), _t(cp), _t(ct), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    np.testing.assert_array_equal(got, ref)
    np.testing.assert_allclose(got.sum(axis=1), 1.0, rtol=0, atol=1e-12)
    # slice 0: the weight sits in the leftmost occupied bin, slice 1 in the
    # rightmost (up to the ulp of mass that C_I = 1 leaves in the last bin)
    b = np.array([[orc.lib().or_bin(v, bins, lo, hi) for v in row] for row in x[:2]])
    assert got[0][b[0] != b[0].min()].sum() < 1e-14 and got[1][b[1] != b[1].max()].sum() < 1e-14
    assert abs(got[0][b[0] == b[0].min()].sum() - 1.0) < 1e-12


@pytest.mark.parametrize("mode", [0, 1])
def test_resample_zero_weight_slice(L, orc, mode):
    """A slice with no weight at all keeps its particles (index j -> j) while
    the slices beside it resample as the oracle does."""
    rng = np.random.default_rng(50 + mode)
    S, n = 3, 7001
    w = rng.gamma(0.5, 1.0, (S, n))
    w /= w.sum(axis=1, keepdims=True)
    w[1] = 0.0
    ref = orc.resample(w, mode, seed=12, slice_begin=3, problem=2)
    idx = torch.empty(S, n, dtype=torch.int32, device=DEV)
    x = torch.randn(S, n, dtype=torch.float32, device=DEV)
    xo = torch.empty_like(x)
    ws = torch.empty(L.pr_resample_workspace(n, S), dtype=torch.uint8, device=DEV)
    L.pr_resample(0, 1, x, None, False, _t(w), n, S, 3, mode, L.Rng(12, 2), idx, xo, None, ws)
    torch.cuda.synchronize()
    got = idx.cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(got, ref)
    np.testing.assert_array_equal(got[1], np.arange(n))
    assert torch.equal(xo[1], x[1])


def test_weight_fixed_point_rounding(L, orc):
    """The device's fixed point round(w 2^61) (integer arithmetic on the
    binary64 encoding) on crafted weights -- exact ties, one ulp either side,
    subnormals, signed zeros, negative values -- each alone in its bin of a
    weighted restriction whose total stays small, so that every fixed value
    shows in the CDF: bit for bit against the oracle, and the bin sums
    recovered from the CDF equal the exact rational rounding."""
    from _fixed_point import crafted_weights, fixed_exact
    w = crafted_weights()
    bins = len(w)
    og = orc.Grid(bins, 0.0, float(bins))
    x = np.arange(bins, dtype=np.float64) + 0.5
    ref = orc.restrict_weighted(x[None], w[None], og)
    fx = [fixed_exact(v) for v in w]
    T = sum(fx)
    assert T < 2 ** 52
    cdf = torch.empty(1, bins + 1, dtype=torch.float64, device=DEV)
    ws = torch.empty(L.pr_restrict_weighted_workspace(1, bins), dtype=torch.uint8, device=DEV)
    for prec, dt in ((0, torch.float32), (1, torch.float64)):
        L.pr_restrict_weighted(prec, _t(x[None], dt), False, _t(w[None]), bins, 1, L.Grid(bins, 0.0, float(bins)),
                               cdf, ws)
        torch.cuda.synchronize()
        got = cdf.cpu().numpy()
        np.testing.assert_array_equal(got, ref)
        below = np.rint(got[0] * T).astype(np.int64)
        np.testing.assert_array_equal(np.diff(below), fx)


@pytest.mark.parametrize("bins", [1, 5, 600, 4096])
def test_reweight_sparse_prior_support(L, orc, bins):
    """A prior supported on a scattered third of the bins (runs of empty bins
    of every length, empty bins at both ends) against a dense target: every
    unsupported target bin is relocated; bit for bit against the oracle for
    grids smaller and larger than the block."""
    rng = np.random.default_rng(60 + bins)
    lo, hi, n, S = -2.0, 2.0, 30011, 2
    og = orc.Grid(bins, lo, hi)
    e = og.edges()
    keep = rng.random(bins) < 0.33
    keep[rng.integers(bins)] = True
    centres = 0.5 * (e[:-1] + e[1:])[keep]
    x = rng.choice(centres, size=(S, n)) + (rng.random((S, n)) - 0.5) * 0.5 * (hi - lo) / bins
    x = x.astype(np.float32).astype(np.float64)
    _, cp = orc.restrict(x, og)
    m = rng.random((S, bins)) + 0.01
    m /= m.sum(axis=1, keepdims=True)
    ct = np.concatenate([np.zeros((S, 1)), np.cumsum(m, axis=1)], axis=1)
    ct[:, -1] = 1.0
    ref = orc.reweight(x, og, cp, ct)
    out = torch.empty(S, n, dtype=torch.float64, device=DEV)
    L.pr_reweight(0, _t(x, torch.float32), False, None, n, S, L.Grid(bins, lo, hi), _t(cp), _t(ct), out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), ref)
    np.testing.assert_allclose(out.cpu().numpy().sum(axis=1), 1.0, rtol=0, atol=1e-11)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("pattern", ["sparse", "heavy", "runs"])
def test_resample_concentrated_weights(L, orc, mode, pattern):
    """Weights that stretch one block of outputs over many particles (weight on
    every 37th particle only: ranges far beyond what a block stages), that
    send most outputs to one particle, and long runs of zero weight between
    dense stretches: every index bit for bit against the oracle."""
    rng = np.random.default_rng({"sparse": 70, "heavy": 71, "runs": 72}[pattern] + 10 * mode)
    S, n = 3, 100003
    w = np.zeros((S, n))
    if pattern == "sparse":
        w[:, ::37] = rng.random((S, len(range(0, n, 37)))) + 0.1
    elif pattern == "heavy":
        w[:] = rng.random((S, n)) * 1e-3
        w[np.arange(S), rng.integers(n, size=S)] = 50.0
    else:
        on = (np.arange(n) // 9001) % 3 == 1
        w[:, on] = rng.random((S, on.sum()))
    w /= w.sum(axis=1, keepdims=True)
    ref = orc.resample(w, mode, seed=31, slice_begin=4, problem=3)
    idx = torch.empty(S, n, dtype=torch.int32, device=DEV)
    ws = torch.empty(L.pr_resample_workspace(n, S), dtype=torch.uint8, device=DEV)
    L.pr_resample(0, 1, None, None, False, _t(w), n, S, 4, mode, L.Rng(31, 3), idx, None, None, ws)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(idx.cpu().numpy().view(np.uint32), ref)


@pytest.mark.parametrize("prec", [0, 1])
def test_reweight_foreign_prior(L, orc, prec):
    """A prior CDF restricted from another sample than the particles: the
    particles in bins the prior calls empty get weight 0, the others the
    relocated target's factors; bit for bit against the oracle."""
    rng = np.random.default_rng(80 + prec)
    bins, lo, hi, n, S = 128, -3.0, 3.0, 30011, 2
    og = orc.Grid(bins, lo, hi)
    x = rng.normal(0.0, 1.0, (S, n))
    if prec == 0:
        x = x.astype(np.float32).astype(np.float64)
    _, cp = orc.restrict(rng.normal(0.6, 0.4, (S, 5000)), og)
    _, ct = orc.restrict(rng.normal(-0.3, 0.8, (S, 5000)), og)
    ref = orc.reweight(x, og, cp, ct)
    dt = torch.float32 if prec == 0 else torch.float64
    out = torch.empty(S, n, dtype=torch.float64, device=DEV)
    L.pr_reweight(prec, _t(x, dt), False, None, n, S, L.Grid(bins, lo, hi), _t(cp), _t(ct), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    np.testing.assert_array_equal(got, ref)
    assert np.any(got == 0.0) and np.any(got > 0.0)
