"""The C ABI library builds, loads and exports every entry point declared in
include/pr.h; host-side argument validation rejects bad arguments before
anything is launched (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1912_09240_gb300 import build as b
    b.build()
    from paper_1912_09240_gb300 import _lib
    return _lib


def _declared():
    src = open(os.path.join(ROOT, "include", "pr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pr_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(L):
    names = _declared()
    assert len(names) >= 14
    lib = L.lib()
    for name in names:
        assert hasattr(lib, name), name
    assert set(L.EXPORTED) == set(names)


def test_status_strings_and_version(L):
    assert L.status_string(L.PR_OK) == "PR_OK"
    assert L.status_string(L.PR_ERR_INVALID_ARG) == "PR_ERR_INVALID_ARG"
    assert L.status_string(99) == "PR_ERR_UNKNOWN"
    assert re.fullmatch(r"\d+\.\d+\.\d+", L.version())


def test_invalid_arguments_rejected_on_host(L):
    lib = L.lib()
    m = L.Model(L.PR_MODEL_OU).c()
    r = L.Rng().c()
    g = L.Grid(16, -1.0, 1.0).c()
    fake = ctypes.c_void_p(0x1000)
    # NULL model / bad precision / n = 0 / bad dt / bad fast_dim for the OU family
    assert lib.pr_fine_propagate(None, 0, ctypes.byref(r), fake, fake, 0, fake, fake, 10, 0, 1, 1, 1e-3,
                                 None, None, None, None, None, None, None, None) == L.PR_ERR_INVALID_ARG
    assert lib.pr_fine_propagate(ctypes.byref(m), 7, ctypes.byref(r), fake, fake, 0, fake, fake, 10, 0, 1, 1,
                                 1e-3, None, None, None, None, None, None, None, None) == L.PR_ERR_INVALID_ARG
    assert lib.pr_fine_propagate(ctypes.byref(m), 0, ctypes.byref(r), fake, fake, 0, fake, fake, 0, 0, 1, 1,
                                 1e-3, None, None, None, None, None, None, None, None) == L.PR_ERR_INVALID_ARG
    assert lib.pr_fine_propagate(ctypes.byref(m), 0, ctypes.byref(r), fake, fake, 0, fake, fake, 10, 0, 1, 1,
                                 -1.0, None, None, None, None, None, None, None, None) == L.PR_ERR_INVALID_ARG
    m2 = L.Model(L.PR_MODEL_OU, fast_dim=3).c()
    assert lib.pr_fine_propagate(ctypes.byref(m2), 0, ctypes.byref(r), fake, fake, 0, fake, fake, 10, 0, 1, 1,
                                 1e-3, None, None, None, None, None, None, None, None) == L.PR_ERR_INVALID_ARG
    # fused outputs without a grid; cdf without counts
    assert lib.pr_fine_propagate(ctypes.byref(m), 0, ctypes.byref(r), fake, fake, 0, fake, fake, 10, 0, 1, 1,
                                 1e-3, None, None, None, fake, None, None, None, None) == L.PR_ERR_INVALID_ARG
    assert lib.pr_fine_propagate(ctypes.byref(m), 0, ctypes.byref(r), fake, fake, 0, fake, fake, 10, 0, 1, 1,
                                 1e-3, ctypes.byref(g), None, None, None, fake, None, None, None) == L.PR_ERR_INVALID_ARG
    # outputs aliasing a broadcast input
    other = ctypes.c_void_p(0x2000)
    assert lib.pr_fine_propagate(ctypes.byref(m), 0, ctypes.byref(r), fake, other, 1, fake, fake, 10, 0, 1, 1,
                                 1e-3, None, None, None, None, None, None, None, None) == L.PR_ERR_INVALID_ARG
    assert lib.pr_fine_propagate(ctypes.byref(m), 0, ctypes.byref(r), other, fake, 1, fake, fake, 10, 0, 1, 1,
                                 1e-3, None, None, None, None, None, None, None, None) == L.PR_ERR_INVALID_ARG
    bad = L.Grid(0, -1.0, 1.0).c()
    assert lib.pr_restrict(0, fake, 10, 1, ctypes.byref(bad), fake, None, None) == L.PR_ERR_INVALID_ARG
    inv = L.Grid(4, 1.0, -1.0).c()
    assert lib.pr_match(0, fake, fake, 10, 1, ctypes.byref(inv), fake, fake, None) == L.PR_ERR_INVALID_ARG
    assert lib.pr_parareal_update(None, 0, 0, 4, fake, fake, fake, fake, None, None) == L.PR_ERR_INVALID_ARG
    assert lib.pr_iterate(9, 0, ctypes.byref(g), 1, fake, fake, fake, fake, None, None) == L.PR_ERR_INVALID_ARG
    assert lib.pr_coarse_destroy(None) == L.PR_ERR_INVALID_ARG
    # misaligned counters for the raw generator
    assert lib.pr_rng_words(ctypes.byref(r), ctypes.c_void_p(0x1004), 1, fake, None) == L.PR_ERR_INVALID_ARG


def test_chemical_and_transfer_arguments_rejected_on_host(L):
    """Host-side checks of the chemical kinds, the L2 distance and the
    transfer calls: they return before any CUDA call."""
    lib = L.lib()
    r = L.Rng().c()
    g = L.Grid(16, 0.0, 16.0).c()
    fake = ctypes.c_void_p(0x1000)
    rates = (60.0, 1.0, 4.8e-3, 0.666e-5, 0.833, 1.0)
    for bad in [L.Model(L.PR_MODEL_CHEM, 2, rates=rates),                                   # one fast variable only
                L.Model(L.PR_MODEL_CHEM, 1, rates=(60.0, -1.0, 4.8e-3, 0.666e-5, 0.833, 1.0)),   # negative rate
                L.Model(L.PR_MODEL_CHEM, 1, rates=(60.0, 1.0, float("inf"), 0.666e-5, 0.833, 1.0)),
                L.Model(L.PR_MODEL_CHEM_PRINTED, 1, eps=0.0, rates=rates)]:
        m = bad.c()
        assert lib.pr_fine_propagate(ctypes.byref(m), 0, ctypes.byref(r), fake, fake, 0, fake, fake, 10, 0, 1, 1,
                                     1e-3, None, None, None, None, None, None, None, None) == L.PR_ERR_INVALID_ARG
    h = ctypes.c_void_p()
    for bad, grid in [(L.Model(L.PR_MODEL_CHEM, 1, rates=(60.0, 1.0, 4.8e-3, 0.666e-5, 0.0, 1.0)), g),   # k4 = 0
                      (L.Model(L.PR_MODEL_CHEM, 1, rates=rates), L.Grid(16, -1.0, 15.0).c())]:       # x_lo < 0
        m = bad.c()
        assert lib.pr_coarse_create(ctypes.byref(m), ctypes.byref(grid), 2.0, ctypes.byref(h), None) == \
            L.PR_ERR_INVALID_ARG
    assert lib.pr_l2_density(ctypes.byref(g), 0, fake, fake, fake, None) == L.PR_ERR_INVALID_ARG
    assert lib.pr_l2_density(ctypes.byref(g), 1, ctypes.c_void_p(0x1004), fake, fake, None) == L.PR_ERR_INVALID_ARG
    assert lib.pr_copy_to_device(None, fake, 8, None) == L.PR_ERR_INVALID_ARG
    assert lib.pr_copy_to_host(fake, None, 8, None) == L.PR_ERR_INVALID_ARG
    assert lib.pr_copy_to_device(None, None, 0, None) == L.PR_OK    # nothing to copy


def test_python_binding_raises(L):
    with pytest.raises(L.PrError) as e:
        L._check("pr_x", L.PR_ERR_NUMERIC)
    assert "PR_ERR_NUMERIC" in str(e.value)


def test_invalid_arguments_rejected_on_host_conditional_and_advection(L):
    """Section 5.2 entry points, the advection model and the workspace sizes:
    rejected before any CUDA call."""
    lib = L.lib()
    r = L.Rng().c()
    g = L.Grid(16, -1.0, 1.0).c()
    fake = ctypes.c_void_p(0x1000)
    # reweight: n = 0, missing CDF, bad precision, bad grid
    assert lib.pr_reweight(0, fake, 0, None, 0, 1, ctypes.byref(g), fake, fake, fake, None) == L.PR_ERR_INVALID_ARG
    assert lib.pr_reweight(0, fake, 0, None, 10, 1, ctypes.byref(g), None, fake, fake, None) == L.PR_ERR_INVALID_ARG
    assert lib.pr_reweight(5, fake, 0, None, 10, 1, ctypes.byref(g), fake, fake, fake, None) == L.PR_ERR_INVALID_ARG
    bad = L.Grid(0, -1.0, 1.0).c()
    assert lib.pr_reweight(0, fake, 0, None, 10, 1, ctypes.byref(bad), fake, fake, fake, None) == L.PR_ERR_INVALID_ARG
    # resample: workspace sizes grow with n and slices; bad mode; small, misaligned
    # workspace; gather in place; n too large for 32-bit indices; fast_dim out of range
    n = 5000
    need = lib.pr_resample_workspace(n, 3)
    assert need >= 3 * n * 8 and lib.pr_resample_workspace(0, 1) == 0
    ws = ctypes.c_void_p(0x10000)
    args = lambda mode, x_in, x_out, nn, wsb, d=1, wsp=ws: (0, d, x_in, fake, 0, fake, nn, 3, 0, mode, ctypes.byref(r),
                                                            None, x_out, None, wsp, wsb, None)
    assert lib.pr_resample(*args(7, fake, None, n, need)) == L.PR_ERR_INVALID_ARG
    assert lib.pr_resample(*args(0, fake, None, n, need - 1)) == L.PR_ERR_INVALID_ARG
    assert lib.pr_resample(*args(0, fake, None, n, need, wsp=ctypes.c_void_p(0x10008))) == L.PR_ERR_INVALID_ARG
    assert lib.pr_resample(*args(0, fake, fake, n, need)) == L.PR_ERR_INVALID_ARG
    assert lib.pr_resample(*args(0, fake, None, 1 << 33, 1 << 60)) == L.PR_ERR_INVALID_ARG
    assert lib.pr_resample(0, 17, fake, fake, 0, fake, n, 3, 0, 0, ctypes.byref(r), None, None, fake, ws, need,
                           None) == L.PR_ERR_INVALID_ARG
    # weighted restriction: too small a workspace
    wneed = lib.pr_restrict_weighted_workspace(3, 16)
    assert wneed >= 3 * 16 * 8
    assert lib.pr_restrict_weighted(0, fake, 0, fake, 10, 3, ctypes.byref(g), fake, ws, wneed - 8,
                                    None) == L.PR_ERR_INVALID_ARG
    # the advection model has no microscopic dynamics and needs eps > 0
    adv = L.Model(L.PR_MODEL_ADVECTION, 1, 0.0, 1.0, 1.0).c()
    assert lib.pr_fine_propagate(ctypes.byref(adv), 0, ctypes.byref(r), fake, fake, 0, fake, fake, 10, 0, 1, 1,
                                 1e-3, None, None, None, None, None, None, None, None) == L.PR_ERR_INVALID_ARG
    adv0 = L.Model(L.PR_MODEL_ADVECTION, 1, 0.0, 1.0, 0.0).c()
    h = ctypes.c_void_p()
    assert lib.pr_coarse_create(ctypes.byref(adv0), ctypes.byref(g), 0.1, ctypes.byref(h), None) == L.PR_ERR_INVALID_ARG
    # the update cluster knob accepts any value (unknown ones select 8)
    lib.pr_set_update_cluster(3)
    lib.pr_set_update_cluster(8)


def test_affine_adjoint_rejects_non_finite_seeds(L):
    lib = L.lib()
    m = L.Model(L.PR_MODEL_OU).c()
    r = L.Rng().c()
    fake = ctypes.c_void_p(0x1000)
    ws = ctypes.c_void_p(0x100000)
    need = lib.pr_fine_adjoint_workspace(100, 2, 10, 12)
    for sc, sh in ((float("nan"), 0.0), (1.0, float("inf"))):
        assert lib.pr_fine_adjoint_affine(ctypes.byref(m), ctypes.byref(r), fake, fake, 100, 0, 2, 10, 1e-3, 12, sc, sh,
                                          None, None, fake, None, None, ws, need, None) == L.PR_ERR_INVALID_ARG
    assert lib.pr_fine_adjoint_affine(ctypes.byref(m), ctypes.byref(r), fake, fake, 100, 0, 2, 10, 1e-3, 12, 1.0, 0.0,
                                      None, None, None, None, None, ws, need, None) == L.PR_ERR_INVALID_ARG
    assert lib.pr_fine_adjoint_affine(ctypes.byref(m), ctypes.byref(r), fake, fake, 100, 0, 2, 10, 1e-3, 12, 1.0, 0.0,
                                      None, None, fake, None, None, ws, need - 1, None) == L.PR_ERR_INVALID_ARG


def test_moments_rejects_bad_arguments(L):
    lib = L.lib()
    fake = ctypes.c_void_p(0x10000)
    need = lib.pr_moments_workspace(1000, 2, 3)
    assert need >= 2 * 3 * 8
    assert lib.pr_moments_workspace(1000, 2, 0) == 0 and lib.pr_moments_workspace(1000, 2, 5) == 0
    ok = dict(prec=0, v=fake, stride=1000, w=None, n=1000, s=2, q=3, out=fake, ws=fake, nb=need)

    def call(**kw):
        a = dict(ok, **kw)
        return lib.pr_moments(a["prec"], a["v"], a["stride"], a["w"], a["n"], a["s"], a["q"], a["out"], a["ws"],
                              a["nb"], None)
    assert call(prec=3) == L.PR_ERR_INVALID_ARG
    assert call(q=0) == L.PR_ERR_INVALID_ARG
    assert call(q=5) == L.PR_ERR_INVALID_ARG
    assert call(stride=999) == L.PR_ERR_INVALID_ARG          # slices would overlap
    assert call(nb=need - 1) == L.PR_ERR_INVALID_ARG
    assert call(ws=ctypes.c_void_p(0x10004)) == L.PR_ERR_INVALID_ARG
    assert call(v=None) == L.PR_ERR_INVALID_ARG
    assert call(n=0) == L.PR_ERR_INVALID_ARG


def test_misaligned_element_pointers_rejected(L):
    """Device pointers not aligned to their element size are refused on the
    host before any launch."""
    lib = L.lib()
    ok4, ok8 = ctypes.c_void_p(0x10000), ctypes.c_void_p(0x10008)
    bad4, bad8 = ctypes.c_void_p(0x10002), ctypes.c_void_p(0x10004)
    g = L.Grid(64, -3.0, 3.0).c()
    assert lib.pr_restrict(0, bad4, 10, 1, ctypes.byref(g), ok4, None, None) == L.PR_ERR_INVALID_ARG
    assert lib.pr_restrict(1, bad8, 10, 1, ctypes.byref(g), ok4, None, None) == L.PR_ERR_INVALID_ARG
    assert lib.pr_restrict(0, ok4, 10, 1, ctypes.byref(g), ok4, bad8, None) == L.PR_ERR_INVALID_ARG
    assert lib.pr_match(0, ok4, bad4, 10, 1, ctypes.byref(g), ok8, ok8, None) == L.PR_ERR_INVALID_ARG
    assert lib.pr_match(0, ok4, ok4, 10, 1, ctypes.byref(g), bad8, ok8, None) == L.PR_ERR_INVALID_ARG
    assert lib.pr_counts_to_cdf(bad4, 10, 1, 64, ok8, None) == L.PR_ERR_INVALID_ARG
    assert lib.pr_w1(ctypes.byref(g), 1, ok8, bad8, ok8, None) == L.PR_ERR_INVALID_ARG
    assert lib.pr_iterate(0, 0, ctypes.byref(g), 1, ok8, ok8, ok8, bad8, None, None) == L.PR_ERR_INVALID_ARG
    assert lib.pr_reweight(0, ok4, 0, None, 10, 1, ctypes.byref(g), ok8, ok8, bad8, None) == L.PR_ERR_INVALID_ARG
    need = lib.pr_restrict_weighted_workspace(1, 64)
    assert lib.pr_restrict_weighted(0, ok4, 0, bad8, 10, 1, ctypes.byref(g), ok8, ok8, need,
                                    None) == L.PR_ERR_INVALID_ARG
    mw = lib.pr_moments_workspace(10, 1, 2)
    assert lib.pr_moments(1, bad8, 10, None, 10, 1, 2, ok8, ok8, mw, None) == L.PR_ERR_INVALID_ARG
    r = L.Rng(1, 0).c()
    m = L.Model(0, 1, 1.0, 1.0, 0.1).c()
    assert lib.pr_fine_propagate(ctypes.byref(m), 0, ctypes.byref(r), bad4, ok4, 0, ok4, ok4, 10, 0, 1, 10,
                                 1e-3, None, None, None, None, None, None, None, None) == L.PR_ERR_INVALID_ARG
    assert lib.pr_order_statistics(ok4, 10, bad8, 1, ok8, ok8, 1 << 20, None) == L.PR_ERR_INVALID_ARG
