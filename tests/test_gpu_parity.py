"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances:
  RNG words, restriction counts/CDFs, the FP64 matching and the quantile
  iterator on identical inputs: bit-exact.
  FP64 fine propagator, one slice from identical inputs: |dx| <= 1e-5 per
  particle (observed ~1e-13: only libm vs CUDA log/sin/cos differ).
  FP32 fine propagator, one slice: |dx| <= 2e-3 * max(|x|, 1) per particle.
  Coarse propagator: 1e-12 absolute on P and on the propagated CDFs.
  Whole parareal runs: W1 between restricted densities <= 1e-4 (FP64) and
  <= 1e-3 (FP32) at every slice and iteration.
"""
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


DEV = "cuda"


def _t(a, dtype=None):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV, dtype=dtype)


def _models(L, orc):
    return [
        (L.Model(L.PR_MODEL_OU, 1, 1.0, 1.0, 0.1), orc.Model(0, 1, 1.0, 1.0, 0.1)),
        (L.Model(L.PR_MODEL_DOUBLE_WELL, 1, 0.5, 3.0, 1e-2), orc.Model(1, 1, 0.5, 3.0, 1e-2)),
        (L.Model(L.PR_MODEL_DW_MULTI, 16, 0.5, 3.0, 1e-2), orc.Model(2, 16, 0.5, 3.0, 1e-2)),
        (L.Model(L.PR_MODEL_DW_MULTI, 3, 0.5, 3.0, 5e-2, 2.0), orc.Model(2, 3, 0.5, 3.0, 5e-2, 2.0)),
        # fast dimensions whose step needs a number of normals that is 2, 3 or 1 mod 4
        (L.Model(L.PR_MODEL_DW_MULTI, 1, 0.5, 3.0, 1e-2), orc.Model(2, 1, 0.5, 3.0, 1e-2)),
        (L.Model(L.PR_MODEL_DW_MULTI, 2, 0.4, 2.0, 2e-2), orc.Model(2, 2, 0.4, 2.0, 2e-2)),
        (L.Model(L.PR_MODEL_DW_MULTI, 8, 0.5, 3.0, 1e-2), orc.Model(2, 8, 0.5, 3.0, 1e-2)),
        # 1 + d = 5 and 6 normals per step: one and two shared tail blocks per four steps
        (L.Model(L.PR_MODEL_DW_MULTI, 4, 0.5, 3.0, 1e-2), orc.Model(2, 4, 0.5, 3.0, 1e-2)),
        (L.Model(L.PR_MODEL_DW_MULTI, 5, 0.5, 3.0, 1e-2), orc.Model(2, 5, 0.5, 3.0, 1e-2)),
    ]


N_MODELS = 9


# ---------------------------------------------------------------------------
# random numbers
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [0, 0xDEADBEEFCAFEF00D])
def test_rng_words_bit_exact(L, orc, seed):
    rng = np.random.default_rng(1)
    ctr = rng.integers(0, 2**32, size=(4099, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:3] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 2, 3, 4]]
    c = _t(ctr.view(np.int32))
    out = torch.empty_like(c)
    L.pr_rng_words(L.Rng(seed), c, ctr.shape[0], out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(got, orc.philox(ctr, seed))


# ---------------------------------------------------------------------------
# fine propagator, one slice from identical inputs
# ---------------------------------------------------------------------------

def _initial(n, d, seed=0):
    rng = np.random.default_rng(seed)
    x = rng.normal(-0.3, 0.8, n)
    y = x[None, :] + rng.normal(0.0, 0.5, (d, n))
    return x, y


@pytest.mark.parametrize("mi", range(N_MODELS))
@pytest.mark.parametrize("n,steps", [(1000, 125), (4096, 7), (1, 3), (257, 0)])
def test_fine_f64_matches_oracle(L, orc, mi, n, steps):
    gm, om = _models(L, orc)[mi]
    d = gm.fast_dim
    n_slices, slice_begin, dt = 3, 5, 1e-3 if gm.kind == 0 else 1e-4
    xs, ys = [], []
    for s in range(n_slices):
        x, y = _initial(n, d, seed=s)
        xs.append(x)
        ys.append(y)
    x0, y0 = np.stack(xs), np.stack(ys)
    gx, gy = _t(x0), _t(y0)
    L.pr_fine_propagate(gm, L.PR_F64, L.Rng(7, 3), gx, gy, False, gx, gy, n, slice_begin, n_slices, steps, dt)
    torch.cuda.synchronize()
    ox, oy = orc.fine_propagate(om, 7, x0, y0, slice_begin, steps, dt, problem=3)
    np.testing.assert_allclose(gx.cpu().numpy(), ox, rtol=0, atol=1e-5)
    np.testing.assert_allclose(gy.cpu().numpy(), oy, rtol=0, atol=1e-5)
    assert np.max(np.abs(gx.cpu().numpy() - ox)) < 1e-10


@pytest.mark.parametrize("mi", range(N_MODELS))
@pytest.mark.parametrize("ppt", [1, 2, 4])
def test_fine_f32_matches_oracle(L, orc, mi, ppt):
    gm, om = _models(L, orc)[mi]
    d = gm.fast_dim
    n, n_slices, slice_begin, steps = 3000, 2, 11, 125
    dt = 1e-3 if gm.kind == 0 else 1e-4
    x0, y0 = _initial(n, d)
    x0 = np.stack([x0, x0 + 0.5]).astype(np.float32)
    y0 = np.stack([y0, y0 - 0.5]).astype(np.float32)
    gx, gy = _t(x0), _t(y0)
    ox_, oy_ = gx.clone(), gy.clone()
    L.pr_set_particles_per_thread(ppt)
    try:
        L.pr_fine_propagate(gm, L.PR_F32, L.Rng(0), gx, gy, False, ox_, oy_, n, slice_begin, n_slices, steps, dt)
        torch.cuda.synchronize()
    finally:
        L.pr_set_particles_per_thread(0)
    ox, oy = orc.fine_propagate(om, 0, x0.astype(np.float64), y0.astype(np.float64), slice_begin, steps, dt)
    gxn, gyn = ox_.cpu().numpy(), oy_.cpu().numpy()
    assert np.all(np.abs(gxn - ox) <= 2e-3 * np.maximum(np.abs(ox), 1.0))
    assert np.all(np.abs(gyn - oy) <= 2e-3 * np.maximum(np.abs(oy), 1.0))
    # the inputs are untouched when out-of-place
    np.testing.assert_array_equal(gx.cpu().numpy(), x0)


def test_fine_broadcast_input(L, orc):
    gm, om = _models(L, orc)[1]
    n, K, steps, dt = 999, 4, 20, 1e-4
    x0, y0 = _initial(n, 1)
    gx, gy = _t(x0), _t(y0)
    ox = torch.empty(K, n, dtype=torch.float64, device=DEV)
    oy = torch.empty(K, 1, n, dtype=torch.float64, device=DEV)
    L.pr_fine_propagate(gm, L.PR_F64, L.Rng(0), gx, gy, True, ox, oy, n, 2, K, steps, dt)
    torch.cuda.synchronize()
    ref, _ = orc.fine_propagate(om, 0, np.repeat(x0[None], K, 0), np.repeat(y0[None], K, 0), 2, steps, dt)
    np.testing.assert_allclose(ox.cpu().numpy(), ref, rtol=0, atol=1e-10)


# ---------------------------------------------------------------------------
# restriction
# ---------------------------------------------------------------------------

def _awkward_x(n_slices, n, grid, rng):
    e = grid.edges()
    x = rng.normal(0.2, 1.3, (n_slices, n))
    k = min(n, 64)
    x[:, :k] = e[rng.integers(0, grid.bins + 1, (n_slices, k))]
    if n > 70:
        x[:, 64:70] = [grid.lo - 3.0, grid.hi + 3.0, grid.lo, grid.hi, np.nextafter(grid.hi, 0),
                       np.nextafter(grid.lo, -10)]
    return x


@pytest.mark.parametrize("bins,lo,hi", [(256, -4.0, 4.0), (512, -3.0, 3.0), (37, -1.3, 2.9), (1, 0.0, 1.0),
                                        (4096, -3.0, 3.0)])
@pytest.mark.parametrize("prec", [0, 1])
def test_restrict_bit_exact(L, orc, bins, lo, hi, prec):
    og = orc.Grid(bins, lo, hi)
    rng = np.random.default_rng(bins)
    n, S = 50_001, 3
    x = _awkward_x(S, n, og, rng)
    if prec == 0:
        x = x.astype(np.float32)
    gx = _t(x)
    counts = torch.empty(S, bins, dtype=torch.int32, device=DEV)
    cdf = torch.empty(S, bins + 1, dtype=torch.float64, device=DEV)
    L.pr_restrict(prec, gx, n, S, L.Grid(bins, lo, hi), counts, cdf)
    torch.cuda.synchronize()
    oc, ocdf = orc.restrict(x.astype(np.float64), og)
    np.testing.assert_array_equal(counts.cpu().numpy().view(np.uint32), oc)
    np.testing.assert_array_equal(cdf.cpu().numpy(), ocdf)


# ---------------------------------------------------------------------------
# matching
# ---------------------------------------------------------------------------

def _cdf_pair(orc, og, rng, n):
    prior_x = rng.normal(-0.4, 0.9, n)
    target_x = rng.gamma(3.0, 0.5, 4 * n) - 1.0
    _, cp = orc.restrict(prior_x[None], og)
    _, ct = orc.restrict(target_x[None], og)
    return prior_x, cp[0], ct[0]


@pytest.mark.parametrize("bins,lo,hi", [(64, -3.0, 3.0), (512, -3.0, 3.0), (37, -2.2, 4.1), (2400, -3.0, 3.0),
                                       (4096, -3.0, 3.0)])
def test_match_f64_bit_exact(L, orc, bins, lo, hi):
    og = orc.Grid(bins, lo, hi)
    rng = np.random.default_rng(3)
    n, S = 20_000, 3
    xs, cps, cts = [], [], []
    for s in range(S):
        x, cp, ct = _cdf_pair(orc, og, rng, n)
        x[:8] = [lo - 1, hi + 1, lo, hi, og.edges()[3], -1e9, 1e9, 0.0]
        xs.append(x)
        cps.append(cp)
        cts.append(ct)
    x, cp, ct = np.stack(xs), np.stack(cps), np.stack(cts)
    out = torch.empty(S, n, dtype=torch.float64, device=DEV)
    L.pr_match(L.PR_F64, _t(x), out, n, S, L.Grid(bins, lo, hi), _t(cp), _t(ct))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), orc.match(x, og, cp, ct))


@pytest.mark.parametrize("bins,lo,hi", [(64, -3.0, 3.0), (512, -3.0, 3.0), (1024, -3.0, 3.0), (2900, -3.0, 3.0)])
def test_match_f32_close(L, orc, bins, lo, hi):
    og = orc.Grid(bins, lo, hi)
    rng = np.random.default_rng(4)
    n = 100_003
    x, cp, ct = _cdf_pair(orc, og, rng, n)
    x32 = x.astype(np.float32)
    _, cp = orc.restrict(x32.astype(np.float64)[None], og)
    out = torch.empty(1, n, dtype=torch.float32, device=DEV)
    L.pr_match(L.PR_F32, _t(x32[None]), out, n, 1, L.Grid(bins, lo, hi), _t(cp), _t(ct[None]))
    torch.cuda.synchronize()
    ref = orc.match(x32.astype(np.float64)[None], og, cp, ct[None])
    got = out.cpu().numpy().astype(np.float64)
    err = np.abs(got - ref)
    assert np.all(err <= 2e-3 * np.maximum(np.abs(ref), 1.0))
    assert np.median(err) < 1e-6
    # matched ensembles restrict to the same histogram up to edge-straddlers
    _, c_got = orc.restrict(got, og)
    _, c_ref = orc.restrict(ref, og)
    assert orc.w1(og, c_got[0], c_ref[0]) < 1e-5


@pytest.mark.parametrize("off_in,off_out", [(0, 0), (1, 1), (3, 0), (0, 2), (2, 2)])
def test_match_f32_alignment_paths(L, orc, off_in, off_out):
    """Slices of a ragged length at every offset from a 16-byte boundary, in
    place and out of place: the vector and scalar paths of the standalone
    binary32 matching give the same bits, and agree with the oracle."""
    og = orc.Grid(512, -3.0, 3.0)
    rng = np.random.default_rng(11)
    n, S = 40_001, 3
    xs, cps, cts = [], [], []
    for _ in range(S):
        x, _, ct = _cdf_pair(orc, og, rng, n)
        x32 = x.astype(np.float32)
        _, cp = orc.restrict(x32.astype(np.float64)[None], og)
        xs.append(x32)
        cps.append(cp[0])
        cts.append(ct)
    x32, cp, ct = np.stack(xs), np.stack(cps), np.stack(cts)
    buf_in = torch.zeros(S * n + 8, dtype=torch.float32, device=DEV)
    gin = buf_in[off_in:off_in + S * n]
    gin.copy_(_t(x32.reshape(-1)))
    if off_in == off_out:     # in place
        gout = gin
        src = gin.clone()
        L.pr_match(L.PR_F32, gin, gout, n, S, L.Grid(512, -3.0, 3.0), _t(cp), _t(ct))
    else:
        src = gin
        buf_out = torch.zeros(S * n + 8, dtype=torch.float32, device=DEV)
        gout = buf_out[off_out:off_out + S * n]
        L.pr_match(L.PR_F32, gin, gout, n, S, L.Grid(512, -3.0, 3.0), _t(cp), _t(ct))
    # per-slice launches at a 16-byte-aligned copy are the reference bits
    ref_bits = []
    for s_ in range(S):
        a = src[s_ * n:(s_ + 1) * n].clone()
        o = torch.empty_like(a)
        L.pr_match(L.PR_F32, a, o, n, 1, L.Grid(512, -3.0, 3.0), _t(cp[s_:s_ + 1]), _t(ct[s_:s_ + 1]))
        ref_bits.append(o)
    torch.cuda.synchronize()
    got = gout.reshape(S, n).cpu().numpy()
    np.testing.assert_array_equal(got, torch.stack(ref_bits).cpu().numpy())
    ref = orc.match(x32.astype(np.float64), og, cp, ct)
    assert np.all(np.abs(got - ref) <= 2e-3 * np.maximum(np.abs(ref), 1.0))


@pytest.mark.parametrize("off", [1, 2, 3])
def test_restrict_f32_offsets(L, orc, off):
    """Binary32 restriction of ragged slices starting off a 16-byte boundary."""
    og = orc.Grid(512, -3.0, 3.0)
    rng = np.random.default_rng(12)
    n, S = 70_003, 5
    x = _awkward_x(S, n, og, rng).astype(np.float32)
    buf = torch.zeros(S * n + 8, dtype=torch.float32, device=DEV)
    gx = buf[off:off + S * n]
    gx.copy_(_t(x.reshape(-1)))
    counts = torch.empty(S, 512, dtype=torch.int32, device=DEV)
    L.pr_restrict(0, gx, n, S, L.Grid(512, -3.0, 3.0), counts, None)
    torch.cuda.synchronize()
    oc, _ = orc.restrict(x.astype(np.float64), og)
    np.testing.assert_array_equal(counts.cpu().numpy().view(np.uint32), oc)


@pytest.mark.parametrize("prec", [0, 1])
def test_match_strong_projection_exact(L, orc, prec):
    og = orc.Grid(128, -3.0, 3.0)
    rng = np.random.default_rng(9)
    n = 30_000
    x = np.concatenate([rng.normal(0.1, 0.8, n - 4), [-5.0, 5.0, -3.0, 3.0]])[None]
    if prec == 0:
        x = x.astype(np.float32)
    _, cdf = orc.restrict(x.astype(np.float64), og)
    gx = _t(x)
    out = torch.empty_like(gx)
    L.pr_match(prec, gx, out, n, 1, L.Grid(128, -3.0, 3.0), _t(cdf), _t(cdf))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), x)


# ---------------------------------------------------------------------------
# coarse propagator, iterators, W1
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind,lam,beta,bins,lo,hi,dT", [(0, 1.0, 1.0, 256, -4.0, 4.0, 0.125),
                                                        (1, 0.5, 3.0, 512, -3.0, 3.0, 0.1),
                                                        (0, 0.3, 2.0, 100, -5.0, 5.0, 0.7),
                                                        (1, 0.5, 3.0, 1, -3.0, 3.0, 0.1),
                                                        (1, 0.5, 3.0, 2, -3.0, 3.0, 0.1),
                                                        (0, 1.0, 1.0, 1024, -4.0, 4.0, 2.0)])
def test_coarse_matches_oracle(L, orc, kind, lam, beta, bins, lo, hi, dT):
    gm = L.Model(kind, 1, lam, beta, 0.1)
    om = orc.Model(kind, 1, lam, beta, 0.1)
    og = orc.Grid(bins, lo, hi)
    h = L.pr_coarse_create(gm, L.Grid(bins, lo, hi), dT)
    try:
        P_ref = orc.coarse_propagator(om, og, dT)
        Pg = torch.empty(bins, bins, dtype=torch.float64, device=DEV)
        L.pr_coarse_matrix(h, Pg)
        torch.cuda.synchronize()
        np.testing.assert_allclose(Pg.cpu().numpy(), P_ref, rtol=0, atol=1e-12)
        rng = np.random.default_rng(2)
        cdfs = np.stack([np.concatenate([[0.0], np.cumsum(m)]) / m.sum() for m in rng.random((5, bins)) ** 3])
        cdfs[:, -1] = 1.0
        out = torch.empty(5, bins + 1, dtype=torch.float64, device=DEV)
        L.pr_coarse_fp(h, _t(cdfs), out, 5)
        torch.cuda.synchronize()
        np.testing.assert_allclose(out.cpu().numpy(), orc.coarse_apply(P_ref, cdfs), rtol=0, atol=1e-12)
    finally:
        L.pr_coarse_destroy(h)


def _rand_cdf(rng, bins, empty=0.3, n=4096):
    m = rng.gamma(0.7, 1.0, bins)
    m[rng.random(bins) < empty] = 0.0
    m[rng.integers(0, bins)] += 0.5
    c = np.round(m / m.sum() * n).astype(np.int64)
    c[0] += max(0, 1 - c.sum())
    cdf = np.concatenate([[0], np.cumsum(c)]) / c.sum()
    cdf[-1] = 1.0
    return cdf


@pytest.mark.parametrize("qmode", [0, 1])
@pytest.mark.parametrize("bins", [1, 2, 3, 64, 512, 1024])
def test_quantile_iterator_bit_exact(L, orc, qmode, bins):
    og = orc.Grid(bins, -3.0, 3.0)
    rng = np.random.default_rng(bins + qmode)
    V = 6
    a = np.stack([_rand_cdf(rng, bins) for _ in range(V)])
    b = np.stack([_rand_cdf(rng, bins) for _ in range(V)])
    c = np.stack([_rand_cdf(rng, bins) for _ in range(V)])
    c[0] = a[0]                       # J(a, b, a) = b
    out = torch.empty(V, bins + 1, dtype=torch.float64, device=DEV)
    st = torch.zeros(1, dtype=torch.int32, device=DEV)
    L.pr_iterate(L.PR_ITER_QUANTILE, qmode, L.Grid(bins, -3.0, 3.0), V, _t(a), _t(b), _t(c), out, st)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert int(st.item()) == 0
    for v in range(V):
        np.testing.assert_array_equal(got[v], orc.iterate(og, a[v], b[v], c[v], 0, qmode))
    if qmode == 0:
        np.testing.assert_array_equal(got[0], b[0])


@pytest.mark.parametrize("it", [1, 2, 3])
def test_mass_iterators(L, orc, it):
    bins = 200
    og = orc.Grid(bins, 0.0, 1.0)
    rng = np.random.default_rng(it)
    lin = np.linspace(0, 1, bins + 1)
    a = np.stack([0.5 * (_rand_cdf(rng, bins, 0.0) + lin) for _ in range(3)])
    b = np.stack([_rand_cdf(rng, bins, 0.1) for _ in range(3)])
    c = np.stack([0.5 * (_rand_cdf(rng, bins, 0.0) + lin) for _ in range(3)])
    out = torch.empty(3, bins + 1, dtype=torch.float64, device=DEV)
    L.pr_iterate(it, 0, L.Grid(bins, 0.0, 1.0), 3, _t(a), _t(b), _t(c), out)
    torch.cuda.synchronize()
    for v in range(3):
        np.testing.assert_allclose(out.cpu().numpy()[v], orc.iterate(og, a[v], b[v], c[v], it), rtol=0, atol=1e-13)


def test_iterator_flags_bad_input(L):
    bins = 8
    a = np.linspace(0, 1, bins + 1)
    bad = a.copy()
    bad[3], bad[4] = bad[4], bad[3]        # not monotone
    out = torch.empty(1, bins + 1, dtype=torch.float64, device=DEV)
    st = torch.zeros(1, dtype=torch.int32, device=DEV)
    L.pr_iterate(L.PR_ITER_QUANTILE, 0, L.Grid(bins, 0.0, 1.0), 1, _t(a[None]), _t(bad[None]), _t(a[None]), out, st)
    torch.cuda.synchronize()
    assert int(st.item()) == L.PR_ERR_NUMERIC


def test_w1_matches_oracle(L, orc):
    bins = 300
    og = orc.Grid(bins, -2.0, 3.0)
    rng = np.random.default_rng(0)
    c1 = np.stack([_rand_cdf(rng, bins) for _ in range(4)])
    c2 = np.stack([_rand_cdf(rng, bins) for _ in range(4)])
    w = torch.empty(4, dtype=torch.float64, device=DEV)
    L.pr_w1(L.Grid(bins, -2.0, 3.0), 4, _t(c1), _t(c2), w)
    torch.cuda.synchronize()
    ref = [orc.w1(og, c1[v], c2[v]) for v in range(4)]
    np.testing.assert_allclose(w.cpu().numpy(), ref, rtol=1e-13, atol=0)


def test_parareal_update_matches_oracle(L, orc):
    bins, K = 128, 6
    gm, om = L.Model(1, 1, 0.5, 3.0, 0.01), orc.Model(1, 1, 0.5, 3.0, 0.01)
    og = orc.Grid(bins, -3.0, 3.0)
    rng = np.random.default_rng(5)
    cdf0 = _rand_cdf(rng, bins, 0.5)
    fs = np.stack([_rand_cdf(rng, bins, 0.3) for _ in range(K)])
    cs = np.stack([_rand_cdf(rng, bins, 0.0) for _ in range(K)])
    h = L.pr_coarse_create(gm, L.Grid(bins, -3.0, 3.0), 0.1)
    try:
        out = torch.empty(K + 1, bins + 1, dtype=torch.float64, device=DEV)
        st = torch.zeros(1, dtype=torch.int32, device=DEV)
        L.pr_parareal_update(h, L.PR_ITER_QUANTILE, 0, K, _t(cdf0), _t(fs), _t(cs), out, st)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        P = orc.coarse_propagator(om, og, 0.1)
        r = cdf0
        got = out.cpu().numpy()
        np.testing.assert_array_equal(got[0], cdf0)
        for n in range(K):
            # from the GPU's own previous state, so that rounding does not accumulate
            a = orc.coarse_apply(P, got[n])[0]
            ref = orc.iterate(og, a, fs[n], cs[n])
            assert orc.w1(og, got[n + 1], ref) < 1e-12
            r = ref
        # iteration-0 sweep (no correction) equals repeated coarse steps
        L.pr_parareal_update(h, L.PR_ITER_NONE, 0, K, _t(cdf0), None, None, out, st)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        r = cdf0
        for n in range(K):
            r = orc.coarse_apply(P, r)[0]
            np.testing.assert_allclose(got[n + 1], r, rtol=0, atol=1e-12)
    finally:
        L.pr_coarse_destroy(h)


@pytest.mark.parametrize("bins", [64, 512, 1024])
def test_update_cluster_sizes_agree(L, bins):
    """The serial sweep split over a cluster of 2, 4 or 8 CTAs gives the
    one-CTA sweep's results bit for bit, for every iterator and both quantile
    modes (each element is computed by one CTA with the same arithmetic)."""
    K = 7
    gm = L.Model(1, 1, 0.5, 3.0, 0.01)
    rng = np.random.default_rng(bins)
    cdf0 = _rand_cdf(rng, bins, 0.5)
    fs = np.stack([_rand_cdf(rng, bins, 0.3) for _ in range(K)])
    cs = np.stack([_rand_cdf(rng, bins, 0.0) for _ in range(K)])
    h = L.pr_coarse_create(gm, L.Grid(bins, -3.0, 3.0), 0.1)
    try:
        cases = [(L.PR_ITER_QUANTILE, 0), (L.PR_ITER_QUANTILE, 1), (L.PR_ITER_ADD, 0), (L.PR_ITER_NONE, 0)]
        for it, qm in cases:
            ref = None
            for cl in (1, 2, 4, 8):
                L.pr_set_update_cluster(cl)
                out = torch.full((K + 1, bins + 1), float("nan"), dtype=torch.float64, device=DEV)
                st = torch.full((1,), -1, dtype=torch.int32, device=DEV)
                none = it == L.PR_ITER_NONE
                L.pr_parareal_update(h, it, qm, K, _t(cdf0), None if none else _t(fs), None if none else _t(cs),
                                     out, st)
                torch.cuda.synchronize()
                assert int(st.item()) == 0, (it, qm, cl)
                got = out.cpu().numpy()
                if ref is None:
                    ref = got
                else:
                    np.testing.assert_array_equal(got, ref, err_msg=f"iterator {it} mode {qm} cluster {cl}")
    finally:
        L.pr_set_update_cluster(8)
        L.pr_coarse_destroy(h)


@pytest.mark.parametrize("bins", [3100, 4096])
def test_match_f32_beyond_table_limit(L, orc, bins):
    """Binary32 matching on grids whose binary32 table does not fit one
    CTA's shared memory: each particle takes the binary64 map (bit-exact
    with the oracle's, test_match_f64_bit_exact), so the result is the
    oracle's image rounded to binary32, bit for bit, on ragged slices with
    edge points and escapees; in place too, and identity on a slice whose
    prior and target agree."""
    og = orc.Grid(bins, -3.0, 3.0)
    rng = np.random.default_rng(bins)
    n, S = 30_001, 3
    xs, cps, cts = [], [], []
    for s_ in range(S):
        x, _, ct = _cdf_pair(orc, og, rng, n)
        x[:8] = [-4.0, 4.0, -3.0, 3.0, og.edges()[5], -1e9, 1e9, 0.0]
        x32 = x.astype(np.float32)
        _, cp = orc.restrict(x32.astype(np.float64)[None], og)
        xs.append(x32)
        cps.append(cp[0])
        cts.append(ct)
    x32, cp, ct = np.stack(xs), np.stack(cps), np.stack(cts)
    ct[1] = cp[1]
    want = orc.match(x32.astype(np.float64), og, cp, ct).astype(np.float32)
    np.testing.assert_array_equal(want[1], x32[1])
    g = L.Grid(bins, -3.0, 3.0)
    out = torch.empty(S, n, dtype=torch.float32, device=DEV)
    L.pr_match(L.PR_F32, _t(x32), out, n, S, g, _t(cp), _t(ct))
    inplace = _t(x32)
    L.pr_match(L.PR_F32, inplace, inplace, n, S, g, _t(cp), _t(ct))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), want)
    np.testing.assert_array_equal(inplace.cpu().numpy(), want)


@pytest.mark.parametrize("broadcast", [False, True])
@pytest.mark.parametrize("kind,d", [(1, 1), (2, 3)])
def test_fused_matching_beyond_table_limit(L, orc, broadcast, kind, d):
    """pr_fine_propagate in binary32 with matching on a 4096-bin grid (its
    table does not fit beside the histograms): the call equals pr_match,
    pr_restrict and pr_fine_propagate without matching in turn, bit for bit,
    with a broadcast start ensemble and out of place, or in place; the
    propagated states agree with the oracle's propagation of the matched
    states within the binary32 tolerance."""
    bins, n, S, steps, dt = 4096, 4003, 2, 20, 1e-3
    rng = np.random.default_rng(4096 + d + int(broadcast))
    og = orc.Grid(bins, -3.0, 3.0)
    nin = 1 if broadcast else S
    px = rng.normal(-0.3, 0.8, (nin, n)).astype(np.float32)
    _, cp1 = orc.restrict(px.astype(np.float64), og)
    cp = np.repeat(cp1, S, axis=0) if broadcast else cp1
    _, ct = orc.restrict(rng.normal(0.4, 0.6, (S, 4 * n)), og)
    x = torch.tensor(px, device=DEV)
    y = torch.tensor(rng.normal(0.0, 1.0, (nin, d, n)), dtype=torch.float32, device=DEV)
    g = L.Grid(bins, -3.0, 3.0)
    m = L.Model(kind, d, 0.5, 3.0, 0.05)
    cpt, ctt = _t(cp), _t(ct)
    cs, ce = (torch.empty(S, bins, dtype=torch.int32, device=DEV) for _ in range(2))
    cds, cde = (torch.empty(S, bins + 1, dtype=torch.float64, device=DEV) for _ in range(2))
    if broadcast:
        xf = torch.empty(S, n, dtype=torch.float32, device=DEV)
        yf = torch.empty(S, d, n, dtype=torch.float32, device=DEV)
        L.pr_fine_propagate(m, 0, L.Rng(7, 2), x, y, True, xf, yf, n, 1, S, steps, dt, grid=g, cdf_prior=cpt,
                            cdf_target=ctt, counts_start=cs, cdf_start=cds, counts_end=ce, cdf_end=cde)
    else:
        xf, yf = x.clone(), y.clone()
        L.pr_fine_propagate(m, 0, L.Rng(7, 2), xf, yf, False, xf, yf, n, 1, S, steps, dt, grid=g, cdf_prior=cpt,
                            cdf_target=ctt, counts_start=cs, cdf_start=cds, counts_end=ce, cdf_end=cde)
    xb = x.expand(S, n).contiguous() if broadcast else x
    yb = y.expand(S, d, n).contiguous() if broadcast else y
    xm = torch.empty_like(xb)
    L.pr_match(0, xb, xm, n, S, g, cpt, ctt)
    cs_ref, ce_ref = (torch.empty(S, bins, dtype=torch.int32, device=DEV) for _ in range(2))
    cds_ref, cde_ref = (torch.empty(S, bins + 1, dtype=torch.float64, device=DEV) for _ in range(2))
    L.pr_restrict(0, xm, n, S, g, cs_ref, cds_ref)
    xs, ys = torch.empty_like(xb), torch.empty_like(yb)
    L.pr_fine_propagate(m, 0, L.Rng(7, 2), xm, yb, False, xs, ys, n, 1, S, steps, dt)
    L.pr_restrict(0, xs, n, S, g, ce_ref, cde_ref)
    torch.cuda.synchronize()
    assert torch.equal(xf, xs) and torch.equal(yf, ys)
    assert torch.equal(cs, cs_ref) and torch.equal(cds, cds_ref)
    assert torch.equal(ce, ce_ref) and torch.equal(cde, cde_ref)
    # the propagation against the oracle's, from the same matched states
    om = orc.Model(kind, d, 0.5, 3.0, 0.05)
    ox, _ = orc.fine_propagate(om, 7, xm.cpu().numpy().astype(np.float64), yb.cpu().numpy().astype(np.float64),
                               1, steps, dt, problem=2)
    got = xf.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ox) <= 2e-3 * np.maximum(np.abs(ox), 1.0))


@pytest.mark.parametrize("prec,bins,kind,d", [(0, 64, 1, 1), (0, 512, 1, 1), (0, 2900, 0, 1), (0, 512, 2, 3),
                                              (0, 4096, 1, 1), (0, 3500, 2, 3),
                                              (1, 64, 0, 1), (1, 2400, 1, 1), (1, 256, 2, 3), (1, 4096, 1, 1)])
def test_fused_matching_equals_standalone(L, orc, prec, bins, kind, d):
    """pr_fine_propagate with the matching fused into its prologue equals
    pr_match followed by pr_fine_propagate without it, bit for bit, and the
    fused restrictions (counts and CDFs) of the start and end states equal
    pr_restrict of the matched and propagated states: binary32 and binary64,
    d = 1 and d = 3, grids up to the shared-memory limit of the matching
    table."""
    rng = np.random.default_rng(bins + d + prec)
    og = orc.Grid(bins, -3.0, 3.0)
    n, S, steps, dt = 5003, 2, 20, 1e-3
    px = rng.normal(-0.3, 0.8, (S, n))
    _, cp = orc.restrict(px, og)
    _, ct = orc.restrict(rng.normal(0.4, 0.6, (S, 4 * n)), og)
    dt_t = torch.float32 if prec == 0 else torch.float64
    if prec == 0:
        px = px.astype(np.float32).astype(np.float64)
        _, cp = orc.restrict(px, og)
    x = torch.tensor(px, dtype=dt_t, device=DEV)
    y = torch.tensor(rng.normal(0.0, 1.0, (S, d, n)), dtype=dt_t, device=DEV)
    g = L.Grid(bins, -3.0, 3.0)
    m = L.Model(kind, d, 0.5, 3.0, 0.05) if kind != 0 else L.Model(0, 1, 1.0, 1.0, 0.1)
    cpt, ctt = torch.tensor(cp, device=DEV), torch.tensor(ct, device=DEV)
    xf, yf = torch.empty_like(x), torch.empty_like(y)
    cs, ce = (torch.empty(S, bins, dtype=torch.int32, device=DEV) for _ in range(2))
    cds, cde = (torch.empty(S, bins + 1, dtype=torch.float64, device=DEV) for _ in range(2))
    L.pr_fine_propagate(m, prec, L.Rng(5, 1), x, y, False, xf, yf, n, 3, S, steps, dt, grid=g, cdf_prior=cpt,
                        cdf_target=ctt, counts_start=cs, cdf_start=cds, counts_end=ce, cdf_end=cde)
    xm = torch.empty_like(x)
    L.pr_match(prec, x, xm, n, S, g, cpt, ctt)
    cs_ref, ce_ref = (torch.empty(S, bins, dtype=torch.int32, device=DEV) for _ in range(2))
    cds_ref, cde_ref = (torch.empty(S, bins + 1, dtype=torch.float64, device=DEV) for _ in range(2))
    L.pr_restrict(prec, xm, n, S, g, cs_ref, cds_ref)
    xs, ys = torch.empty_like(x), torch.empty_like(y)
    L.pr_fine_propagate(m, prec, L.Rng(5, 1), xm, y, False, xs, ys, n, 3, S, steps, dt)
    L.pr_restrict(prec, xs, n, S, g, ce_ref, cde_ref)
    torch.cuda.synchronize()
    assert torch.equal(xf, xs) and torch.equal(yf, ys)
    assert torch.equal(cs, cs_ref) and torch.equal(cds, cds_ref)
    assert torch.equal(ce, ce_ref) and torch.equal(cde, cde_ref)


@pytest.mark.parametrize("kind,n,S", [(1, 5003, 2), (1, 100000, 5), (4, 100000, 5), (1, 200003, 4),
                                      (1, 1 << 20, 2)])
def test_particles_per_thread_bit_identical(L, orc, kind, n, S):
    """The binary32 d = 1 propagator gives the same bits whatever number of
    particles each thread carries: 1, 2 and 4 forced, and the per-launch
    choice (0), whose value changes across these sizes (on 152 SMs: 1 up to
    5e5 particles, 2 at 8e5, 4 at 2^21), with the matching fused in and both
    restrictions."""
    rng = np.random.default_rng(n + kind)
    if kind == 4:
        bins, lo, hi = 600, 0.0, 600.0
        m = L.Model(4, 1, 0.0, 1.0, 1e-2, 25.0, tuple(workloads.CHEM_RATES))
        px = rng.lognormal(np.log(98.0), 0.2, (S, n))
        tgt = rng.lognormal(np.log(101.0), 0.2, (S, 2 * n))
        y0 = rng.lognormal(np.log(98.0), 0.2, (S, n))
        dt, steps = 1e-3, 40
    else:
        bins, lo, hi = 512, -3.0, 3.0
        m = L.Model(kind, 1, 0.5, 3.0, 1e-2)
        px = rng.normal(-0.3, 0.8, (S, n))
        tgt = rng.normal(0.4, 0.6, (S, 2 * n))
        y0 = rng.normal(0.0, 1.0, (S, n))
        dt, steps = 1e-4, 30
    og = orc.Grid(bins, lo, hi)
    px = px.astype(np.float32)
    _, cp = orc.restrict(px.astype(np.float64), og)
    _, ct = orc.restrict(tgt, og)
    g = L.Grid(bins, lo, hi)
    x, y = _t(px), _t(y0.astype(np.float32))
    cpt, ctt = _t(cp), _t(ct)
    outs = []
    try:
        for ppt in (1, 2, 4, 0):
            L.pr_set_particles_per_thread(ppt)
            xf, yf = torch.empty_like(x), torch.empty_like(y)
            cs, ce = (torch.empty(S, bins, dtype=torch.int32, device=DEV) for _ in range(2))
            cds, cde = (torch.empty(S, bins + 1, dtype=torch.float64, device=DEV) for _ in range(2))
            L.pr_fine_propagate(m, L.PR_F32, L.Rng(9), x, y, False, xf, yf, n, 1, S, steps, dt, grid=g,
                                cdf_prior=cpt, cdf_target=ctt, counts_start=cs, cdf_start=cds, counts_end=ce,
                                cdf_end=cde)
            outs.append((xf, yf, cs, cds, ce, cde))
        torch.cuda.synchronize()
    finally:
        L.pr_set_particles_per_thread(0)
    assert torch.isfinite(outs[0][0]).all()
    for o in outs[1:]:
        assert all(torch.equal(a, b) for a, b in zip(outs[0], o))


@pytest.mark.parametrize("bins", [1, 2, 3])
@pytest.mark.parametrize("it", [1, 2, 3])
def test_mass_iterators_tiny_grids(L, orc, it, bins):
    """The additive, multiplicative and rotation iterators on grids of 1, 2
    and 3 bins with empty bins, against the oracle."""
    og = orc.Grid(bins, 0.0, 1.0)
    rng = np.random.default_rng(10 * it + bins)
    V = 8
    a, b, c = (np.stack([_rand_cdf(rng, bins) for _ in range(V)]) for _ in range(3))
    out = torch.empty(V, bins + 1, dtype=torch.float64, device=DEV)
    L.pr_iterate(it, 0, L.Grid(bins, 0.0, 1.0), V, _t(a), _t(b), _t(c), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for v in range(V):
        np.testing.assert_allclose(got[v], orc.iterate(og, a[v], b[v], c[v], it, 0), rtol=0, atol=1e-13)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("case", ["foreign_prior", "point_masses", "prior_in_target_gap"])
def test_match_degenerate_cdfs(L, orc, prec, case):
    """Matching with CDFs that are not the ensemble's own: a prior from
    another sample (particles in bins the prior calls empty), prior and
    target each concentrated in a single bin, and a prior whose support lies
    in a gap of the target.  Binary64 bit for bit, binary32 within its
    tolerance, both against the oracle."""
    bins, lo, hi, n = 96, -3.0, 3.0, 20011
    og = orc.Grid(bins, lo, hi)
    rng = np.random.default_rng({"foreign_prior": 1, "point_masses": 2, "prior_in_target_gap": 3}[case] + 10 * prec)
    x = rng.normal(0.0, 1.0, (1, n))
    cdf = lambda m: np.concatenate([[0.0], np.cumsum(m / m.sum())])
    if case == "foreign_prior":
        _, cp = orc.restrict(rng.normal(0.8, 0.3, (1, n)), og)
        _, ct = orc.restrict(rng.normal(-0.5, 0.7, (1, n)), og)
    elif case == "point_masses":
        mp, mt = np.zeros(bins), np.zeros(bins)
        mp[40], mt[70] = 1.0, 1.0
        cp, ct = cdf(mp)[None], cdf(mt)[None]
    else:
        mt = np.ones(bins)
        mt[30:60] = 0.0
        mp = np.zeros(bins)
        mp[35:55] = 1.0
        cp, ct = cdf(mp)[None], cdf(mt)[None]
    cp[:, -1] = 1.0
    ct[:, -1] = 1.0
    if prec == 0:
        x = x.astype(np.float32).astype(np.float64)
    dt = torch.float32 if prec == 0 else torch.float64
    out = torch.empty(1, n, dtype=dt, device=DEV)
    L.pr_match(prec, torch.tensor(x, dtype=dt, device=DEV), out, n, 1, L.Grid(bins, lo, hi), _t(cp), _t(ct))
    torch.cuda.synchronize()
    ref = orc.match(x, og, cp, ct)
    got = out.cpu().numpy().astype(np.float64)
    if prec == 1:
        np.testing.assert_array_equal(got, ref)
    else:
        assert np.all(np.abs(got - ref) <= 2e-3 * np.maximum(np.abs(ref), 1.0))


@pytest.mark.parametrize("qmode", [0, 1])
def test_quantile_iterator_degenerate_cdfs(L, orc, qmode):
    """The quantile iterator on point masses in different bins, disjoint
    supports, mass only in the two end bins, and a = b = c: bit for bit
    against the oracle, unit mass and monotone."""
    bins = 48
    og = orc.Grid(bins, -3.0, 3.0)
    def cdf(m):   # a valid CDF: non-decreasing, C_0 = 0, C_I = 1 exactly
        c = np.minimum(np.concatenate([[0.0], np.cumsum(np.asarray(m, float) / np.sum(m))]), 1.0)
        c[-1] = 1.0
        return c
    pm = lambda *idx: np.bincount(idx, minlength=bins).astype(float)
    ends = np.zeros(bins)
    ends[[0, -1]] = [0.3, 0.7]
    cases = [(pm(5), pm(20), pm(40)), (pm(0), pm(47), pm(47)), (pm(3, 4), pm(30, 31, 32), pm(10)),
             (ends, pm(24), ends), (ends, ends, ends), (pm(12), pm(12), pm(12)),
             (np.ones(bins), pm(7), np.ones(bins))]
    a, b, c = (np.stack([cdf(t[k]) for t in cases]) for k in range(3))
    V = len(cases)
    out = torch.empty(V, bins + 1, dtype=torch.float64, device=DEV)
    st = torch.zeros(1, dtype=torch.int32, device=DEV)
    L.pr_iterate(L.PR_ITER_QUANTILE, qmode, L.Grid(bins, -3.0, 3.0), V, _t(a), _t(b), _t(c), out, st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    got = out.cpu().numpy()
    for v in range(V):
        ref = orc.iterate(og, a[v], b[v], c[v], 0, qmode)
        np.testing.assert_array_equal(got[v], ref, err_msg=f"case {v}")
        assert got[v][0] == 0.0 and got[v][-1] == 1.0 and np.all(np.diff(got[v]) >= 0)
