"""Ensembles beyond 2^31 particles: every kernel's particle index must be
64-bit wide (a 32-bit product or sum would wrap past 2^31).  Inputs are
built on the device in chunks; expected values come from closed forms and
from the oracle run on sampled particles (with their own indices as Philox
particle ids), among them the ones just below and above 2^31."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
DEV = "cuda"
N_BIG = (1 << 31) + 77
BINS, LO, HI = 512, -3.0, 3.0          # h = 3/256: bin centres are exact in binary32
SAMPLE = np.array([0, 1, 511, 512, (1 << 31) - 1, 1 << 31, (1 << 31) + 1, N_BIG - 1, 123456789, 1500000001])


@pytest.fixture(scope="module")
def L():
    from paper_1912_09240_gb300 import build as b
    b.build()
    from paper_1912_09240_gb300 import _lib
    yield _lib
    torch.cuda.empty_cache()   # these tests hold tens of GB; give them back to the device


def _centres(n):
    """x_p = centre of bin (p mod BINS), filled in chunks."""
    h = (HI - LO) / BINS
    x = torch.empty(n, dtype=torch.float32, device=DEV)
    step = 1 << 27
    for a in range(0, n, step):
        b = min(n, a + step)
        i = torch.arange(a, b, dtype=torch.int64, device=DEV) % BINS
        x[a:b] = (LO + (i.to(torch.float64) + 0.5) * h).to(torch.float32)
    return x


def _expected_counts(n):
    i = np.arange(BINS)
    return (n - i + BINS - 1) // BINS


def _cdf_of(counts):
    c = np.concatenate([[0], np.cumsum(counts)]).astype(np.float64)
    return c / c[-1]


def test_restrict_beyond_2_31(L):
    x = _centres(N_BIG)
    counts = torch.empty(1, BINS, dtype=torch.int32, device=DEV)
    cdf = torch.empty(1, BINS + 1, dtype=torch.float64, device=DEV)
    L.pr_restrict(L.PR_F32, x, N_BIG, 1, L.Grid(BINS, LO, HI), counts, cdf)
    torch.cuda.synchronize()
    exp = _expected_counts(N_BIG)
    np.testing.assert_array_equal(counts.cpu().numpy()[0].astype(np.int64), exp)
    np.testing.assert_array_equal(cdf.cpu().numpy()[0], np.concatenate([[0], np.cumsum(exp)]) / N_BIG)


def test_match_beyond_2_31(L, orc):
    """Target = the prior moved up by one bin (bin 0 left empty, the last
    bin keeping its own mass too): a map that moves every particle, sampled
    particles against the oracle's matching of the same values."""
    x = _centres(N_BIG)
    exp = _expected_counts(N_BIG).astype(np.float64)
    cp = _cdf_of(exp)
    tgt = np.concatenate([[0.0], exp[:-1]])
    tgt[-1] += exp[-1]
    ct = _cdf_of(tgt)
    out = torch.empty_like(x)
    L.pr_match(L.PR_F32, x, out, N_BIG, 1, L.Grid(BINS, LO, HI), torch.tensor(cp[None], device=DEV),
               torch.tensor(ct[None], device=DEV))
    torch.cuda.synchronize()
    og = orc.Grid(BINS, LO, HI)
    xs = x[torch.tensor(SAMPLE, device=DEV)].cpu().numpy().astype(np.float64)
    ref = orc.match(xs[None], og, cp[None], ct[None])[0]
    got = out[torch.tensor(SAMPLE, device=DEV)].cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= 2e-3 * np.maximum(np.abs(ref), 1.0)), (got, ref)
    assert np.all(np.abs(got - xs) > 1e-3)   # every sampled particle moved


def test_fine_propagate_beyond_2_31(L, orc):
    """Two EM steps of the OU system over 2^31 + 77 particles in place, with
    the end-state restriction fused: sampled particles against the oracle
    with their own particle ids, and the counts sum to n."""
    x = _centres(N_BIG).reshape(1, -1)
    y = torch.zeros(1, 1, N_BIG, dtype=torch.float32, device=DEV)
    x0 = x[0, torch.tensor(SAMPLE, device=DEV)].cpu().numpy().astype(np.float64)
    counts = torch.empty(1, BINS, dtype=torch.int32, device=DEV)
    m = L.Model(L.PR_MODEL_OU, 1, 0.7, 2.0, 0.1)
    L.pr_fine_propagate(m, L.PR_F32, L.Rng(11, 3), x, y, False, x, y, N_BIG, 4, 1, 2, 1e-3,
                        grid=L.Grid(BINS, LO, HI), counts_end=counts)
    torch.cuda.synchronize()
    assert int(counts.to(torch.int64).sum().item()) == N_BIG
    idx = torch.tensor(SAMPLE, device=DEV)
    gx = x[0, idx].cpu().numpy().astype(np.float64)
    gy = y[0, 0, idx].cpu().numpy().astype(np.float64)
    rx, ry = orc.fine_propagate(orc.Model(kind=0, fast_dim=1, lam=0.7, beta=2.0, eps=0.1), 11, x0[None],
                                np.zeros((1, 1, len(SAMPLE))), 4, 2, 1e-3, problem=3, ids=SAMPLE.astype(np.uint32))
    assert np.all(np.abs(gx - rx[0]) <= 2e-3 * np.maximum(np.abs(rx[0]), 1.0)), (gx, rx[0])
    assert np.all(np.abs(gy - ry[0, 0]) <= 2e-3 * np.maximum(np.abs(ry[0, 0]), 1.0)), (gy, ry[0, 0])


def test_resample_equal_weights_beyond_2_31(L):
    """Equal weights over 2^31 + 77 particles: both resampling modes give
    the identity (strong projection), checked on every index in chunks."""
    n = N_BIG
    w = torch.full((1, n), 1.0 / n, dtype=torch.float64, device=DEV)
    idx = torch.empty(1, n, dtype=torch.int32, device=DEV)
    ws = torch.empty(L.pr_resample_workspace(n, 1), dtype=torch.uint8, device=DEV)
    for mode in (L.PR_RESAMPLE_STRATIFIED, L.PR_RESAMPLE_DETERMINISTIC):
        L.pr_resample(0, 1, None, None, False, w, n, 1, 2, mode, L.Rng(4, 0), idx, None, None, ws)
        torch.cuda.synchronize()
        step = 1 << 27
        for a in range(0, n, step):
            b = min(n, a + step)
            got = idx[0, a:b].to(torch.int64) & 0xFFFFFFFF
            assert torch.equal(got, torch.arange(a, b, dtype=torch.int64, device=DEV)), (mode, a)


def test_reweight_and_weighted_restriction_beyond_2_31(L):
    """Reweighting to a target that doubles the mass of the even bins (the
    factors are exact: 4/3 on even bins, 2/3 on odd ones up to the rounding
    of the CDF differences, checked on sampled particles against the same
    arithmetic), then the weighted restriction of those weights, whose CDF
    must be the target's within the rounding of the fixed point."""
    x = _centres(N_BIG)
    exp = _expected_counts(N_BIG).astype(np.float64)
    cp = _cdf_of(exp)
    tgt = exp * np.where(np.arange(BINS) % 2 == 0, 2.0, 1.0)
    ct = _cdf_of(tgt)
    w = torch.empty(1, N_BIG, dtype=torch.float64, device=DEV)
    g = L.Grid(BINS, LO, HI)
    L.pr_reweight(L.PR_F32, x, False, None, N_BIG, 1, g, torch.tensor(cp[None], device=DEV),
                  torch.tensor(ct[None], device=DEV), w)
    torch.cuda.synchronize()
    bins_s = SAMPLE % BINS
    r = (ct[bins_s + 1] - ct[bins_s]) / (cp[bins_s + 1] - cp[bins_s])
    np.testing.assert_allclose(w[0, torch.tensor(SAMPLE, device=DEV)].cpu().numpy(), r / N_BIG, rtol=1e-14)
    cdf = torch.empty(1, BINS + 1, dtype=torch.float64, device=DEV)
    ws = torch.empty(L.pr_restrict_weighted_workspace(1, BINS), dtype=torch.uint8, device=DEV)
    L.pr_restrict_weighted(L.PR_F32, x, False, w, N_BIG, 1, g, cdf, ws)
    torch.cuda.synchronize()
    np.testing.assert_allclose(cdf.cpu().numpy()[0], ct, rtol=0, atol=1e-12)


def test_slice_count_at_its_limit(L, orc):
    """65535 slices (the largest count the entry points accept) of 7
    particles: restriction counts against their closed form, the fine
    propagator on the first and last slices against the oracle, and
    equal-weight resampling (the identity) on every slice."""
    S, n = 65535, 7
    h = (HI - LO) / BINS
    i = (torch.arange(S * n, dtype=torch.int64, device=DEV) * 37) % BINS
    x = (LO + (i.to(torch.float64) + 0.5) * h).to(torch.float32).reshape(S, n)
    g = L.Grid(BINS, LO, HI)
    counts = torch.empty(S, BINS, dtype=torch.int32, device=DEV)
    L.pr_restrict(L.PR_F32, x, n, S, g, counts, None)
    ref = torch.zeros(S, BINS, dtype=torch.int32, device=DEV)
    ref.scatter_add_(1, i.reshape(S, n), torch.ones(S, n, dtype=torch.int32, device=DEV))
    torch.cuda.synchronize()
    assert torch.equal(counts, ref)
    y = torch.zeros(S, 1, n, dtype=torch.float32, device=DEV)
    xo, yo = torch.empty_like(x), torch.empty_like(y)
    m = L.Model(L.PR_MODEL_DOUBLE_WELL, 1, 0.5, 3.0, 0.1)
    L.pr_fine_propagate(m, L.PR_F32, L.Rng(2, 0), x, y, False, xo, yo, n, 9, S, 4, 1e-3)
    torch.cuda.synchronize()
    om = orc.Model(kind=1, fast_dim=1, lam=0.5, beta=3.0, eps=0.1)
    for s in (0, S - 1):
        rx, _ = orc.fine_propagate(om, 2, x[s:s + 1].cpu().numpy(), np.zeros((1, 1, n)), 9 + s, 4, 1e-3)
        got = xo[s].cpu().numpy().astype(np.float64)
        assert np.all(np.abs(got - rx[0]) <= 2e-3 * np.maximum(np.abs(rx[0]), 1.0)), (s, got, rx[0])
    w = torch.full((S, n), 1.0 / n, dtype=torch.float64, device=DEV)
    idx = torch.empty(S, n, dtype=torch.int32, device=DEV)
    ws = torch.empty(L.pr_resample_workspace(n, S), dtype=torch.uint8, device=DEV)
    L.pr_resample(0, 1, None, None, False, w, n, S, 0, L.PR_RESAMPLE_STRATIFIED, L.Rng(1, 0), idx, None, None, ws)
    torch.cuda.synchronize()
    assert torch.equal(idx, torch.arange(n, dtype=torch.int32, device=DEV).expand(S, n))
