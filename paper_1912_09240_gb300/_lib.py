"""ctypes binding of libpr.so (include/pr.h): argument marshalling only.

Every function here has the name of the C entry point it calls and passes
plain device pointers (torch tensors' ``data_ptr()``), sizes and a stream.
No computation happens in Python; a missing library raises instead of
falling back to anything.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpr.so")

PR_OK, PR_ERR_INVALID_ARG, PR_ERR_CUDA, PR_ERR_TIMEOUT, PR_ERR_UNSUPPORTED, PR_ERR_NOMEM, PR_ERR_NUMERIC = range(7)
PR_F32, PR_F64 = 0, 1
PR_MODEL_OU, PR_MODEL_DOUBLE_WELL, PR_MODEL_DW_MULTI, PR_MODEL_ADVECTION = 0, 1, 2, 3
PR_MODEL_CHEM, PR_MODEL_CHEM_PRINTED = 4, 5
PR_ITER_QUANTILE, PR_ITER_ADD, PR_ITER_MULT, PR_ITER_ROT, PR_ITER_NONE = 0, 1, 2, 3, 4
PR_QMODE_TWO_SIDED, PR_QMODE_MIDPOINT = 0, 1
PR_RESAMPLE_STRATIFIED, PR_RESAMPLE_DETERMINISTIC = 0, 1

EXPORTED = (
    "pr_status_string", "pr_version", "pr_rng_words", "pr_fine_propagate", "pr_set_particles_per_thread",
    "pr_set_tiles_per_cta", "pr_set_update_cluster", "pr_restrict", "pr_counts_to_cdf", "pr_match", "pr_coarse_create", "pr_coarse_destroy",
    "pr_coarse_matrix", "pr_coarse_fp", "pr_parareal_update", "pr_iterate", "pr_w1",
    "pr_fine_adjoint_workspace", "pr_fine_adjoint", "pr_fine_adjoint_affine", "pr_order_statistics_workspace", "pr_order_statistics",
    "pr_fine_adjoint_noalloc_capacity", "pr_fine_adjoint_noalloc",
    "pr_batch_create", "pr_batch_destroy", "pr_batch_particle_steps", "pr_batch_set_initial", "pr_batch_iterate",
    "pr_batch_rho", "pr_batch_fine_state", "pr_batch_status", "pr_batch_set_config", "pr_batch_get_config",
    "pr_batch_tune", "pr_reweight", "pr_resample_workspace", "pr_resample", "pr_restrict_weighted_workspace",
    "pr_restrict_weighted", "pr_moments_workspace", "pr_moments", "pr_copy_to_device", "pr_copy_to_host",
    "pr_stream_synchronize", "pr_l2_density",
)


class PrError(RuntimeError):
    def __init__(self, fn: str, code: int):
        self.code = code
        super().__init__(f"{fn} failed: {status_string(code)}")


class _Model(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("fast_dim", ctypes.c_int32), ("lambda_", ctypes.c_double),
                ("beta", ctypes.c_double), ("eps", ctypes.c_double), ("tau_x", ctypes.c_double),
                ("rate", ctypes.c_double * 6)]


class _Grid(ctypes.Structure):
    _fields_ = [("bins", ctypes.c_int32), ("x_lo", ctypes.c_double), ("x_hi", ctypes.c_double)]


class _Rng(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("problem_id", ctypes.c_uint32)]


class _Problem(ctypes.Structure):
    _fields_ = [("model", _Model), ("grid", _Grid), ("n", ctypes.c_int64), ("n_slices", ctypes.c_int32),
                ("steps", ctypes.c_int32), ("dt", ctypes.c_double), ("seed", ctypes.c_uint64)]


@dataclass(frozen=True)
class Model:
    kind: int
    fast_dim: int = 1
    lam: float = 1.0
    beta: float = 1.0
    eps: float = 0.1
    tau_x: float = 1.0
    rates: tuple = ()     # k0..k5 (chemical system)

    def c(self) -> _Model:
        r = tuple(float(v) for v in self.rates) + (0.0,) * (6 - len(self.rates))
        return _Model(self.kind, self.fast_dim, self.lam, self.beta, self.eps, self.tau_x, (ctypes.c_double * 6)(*r))


@dataclass(frozen=True)
class Grid:
    bins: int
    lo: float
    hi: float

    def c(self) -> _Grid:
        return _Grid(self.bins, self.lo, self.hi)


@dataclass(frozen=True)
class Rng:
    seed: int = 0
    problem_id: int = 0

    def c(self) -> _Rng:
        return _Rng(self.seed, self.problem_id)


@dataclass(frozen=True)
class Problem:
    """One problem of a batch (include/pr.h, pr_problem)."""
    model: Model
    grid: Grid
    n: int
    n_slices: int
    steps: int
    dt: float
    seed: int = 0

    def c(self) -> _Problem:
        return _Problem(self.model.c(), self.grid.c(), self.n, self.n_slices, self.steps, self.dt, self.seed)


_lib = None


def lib() -> ctypes.CDLL:
    """Load libpr.so; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, u32, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_double
    P = ctypes.POINTER
    L.pr_status_string.argtypes = [i32]
    L.pr_status_string.restype = ctypes.c_char_p
    L.pr_version.restype = ctypes.c_char_p
    L.pr_fine_propagate.argtypes = [P(_Model), i32, P(_Rng), vp, vp, i32, vp, vp, i64, i32, i32, i32, d,
                                    P(_Grid), vp, vp, vp, vp, vp, vp, vp]
    L.pr_rng_words.argtypes = [P(_Rng), vp, i64, vp, vp]
    L.pr_set_particles_per_thread.argtypes = [i32]
    L.pr_set_particles_per_thread.restype = None
    L.pr_set_tiles_per_cta.argtypes = [i32]
    L.pr_set_tiles_per_cta.restype = None
    L.pr_set_update_cluster.argtypes = [i32]
    L.pr_set_update_cluster.restype = None
    L.pr_restrict.argtypes = [i32, vp, i64, i32, P(_Grid), vp, vp, vp]
    L.pr_counts_to_cdf.argtypes = [vp, i64, i32, i32, vp, vp]
    L.pr_match.argtypes = [i32, vp, vp, i64, i32, P(_Grid), vp, vp, vp]
    L.pr_coarse_create.argtypes = [P(_Model), P(_Grid), d, P(vp), vp]
    L.pr_coarse_destroy.argtypes = [vp]
    L.pr_coarse_matrix.argtypes = [vp, vp, vp]
    L.pr_coarse_fp.argtypes = [vp, vp, vp, i32, vp]
    L.pr_parareal_update.argtypes = [vp, i32, i32, i32, vp, vp, vp, vp, vp, vp]
    L.pr_iterate.argtypes = [i32, i32, P(_Grid), i32, vp, vp, vp, vp, vp, vp]
    L.pr_w1.argtypes = [P(_Grid), i32, vp, vp, vp, vp]
    L.pr_l2_density.argtypes = [P(_Grid), i32, vp, vp, vp, vp]
    L.pr_fine_adjoint_workspace.argtypes = [i64, i32, i32, i32]
    L.pr_fine_adjoint_workspace.restype = ctypes.c_size_t
    L.pr_fine_adjoint.argtypes = [P(_Model), P(_Rng), vp, vp, i64, i32, i32, i32, d, i32, vp, vp, vp, vp, vp,
                                  vp, vp, vp, ctypes.c_size_t, vp]
    L.pr_fine_adjoint_affine.argtypes = [P(_Model), P(_Rng), vp, vp, i64, i32, i32, i32, d, i32, d, d, vp, vp, vp,
                                         vp, vp, vp, ctypes.c_size_t, vp]
    L.pr_order_statistics_workspace.argtypes = [i64]
    L.pr_order_statistics_workspace.restype = ctypes.c_size_t
    L.pr_order_statistics.argtypes = [vp, i64, vp, i32, vp, vp, ctypes.c_size_t, vp]
    L.pr_fine_adjoint_noalloc_capacity.argtypes = []
    L.pr_fine_adjoint_noalloc_capacity.restype = ctypes.c_size_t
    L.pr_fine_adjoint_noalloc.argtypes = [P(_Model), P(_Rng), vp, vp, i64, i32, i32, i32, d, i32, vp, vp, vp, vp,
                                          vp, vp, vp, vp]
    L.pr_batch_create.argtypes = [P(_Problem), i32, i32, i32, P(vp), vp]
    L.pr_batch_destroy.argtypes = [vp]
    L.pr_batch_particle_steps.argtypes = [vp]
    L.pr_batch_particle_steps.restype = i64
    L.pr_batch_set_initial.argtypes = [vp, vp, vp, vp]
    L.pr_batch_iterate.argtypes = [vp, vp]
    L.pr_batch_rho.argtypes = [vp, i32, vp, vp]
    L.pr_batch_fine_state.argtypes = [vp, i32, vp, vp, vp]
    L.pr_batch_status.argtypes = [vp, P(i32), vp]
    L.pr_batch_set_config.argtypes = [vp, i32, d]
    L.pr_batch_get_config.argtypes = [vp, P(i32), P(d), P(i32)]
    L.pr_batch_tune.argtypes = [vp, i32, P(d), vp]
    L.pr_reweight.argtypes = [i32, vp, i32, vp, i64, i32, P(_Grid), vp, vp, vp, vp]
    L.pr_resample_workspace.argtypes = [i64, i32]
    L.pr_resample_workspace.restype = ctypes.c_size_t
    L.pr_resample.argtypes = [i32, i32, vp, vp, i32, vp, i64, i32, i32, i32, P(_Rng), vp, vp, vp, vp,
                              ctypes.c_size_t, vp]
    L.pr_restrict_weighted_workspace.argtypes = [i32, i32]
    L.pr_restrict_weighted_workspace.restype = ctypes.c_size_t
    L.pr_restrict_weighted.argtypes = [i32, vp, i32, vp, i64, i32, P(_Grid), vp, vp, ctypes.c_size_t, vp]
    L.pr_moments_workspace.argtypes = [i64, i32, i32]
    L.pr_moments_workspace.restype = ctypes.c_size_t
    L.pr_moments.argtypes = [i32, vp, i64, vp, i64, i32, i32, vp, vp, ctypes.c_size_t, vp]
    L.pr_copy_to_device.argtypes = [vp, vp, ctypes.c_size_t, vp]
    L.pr_copy_to_host.argtypes = [vp, vp, ctypes.c_size_t, vp]
    L.pr_stream_synchronize.argtypes = [vp]
    for name in EXPORTED:
        if name not in ("pr_status_string", "pr_version", "pr_set_particles_per_thread",
                        "pr_set_tiles_per_cta", "pr_set_update_cluster", "pr_fine_adjoint_workspace",
                        "pr_order_statistics_workspace", "pr_fine_adjoint_noalloc_capacity",
                        "pr_batch_particle_steps", "pr_resample_workspace", "pr_restrict_weighted_workspace",
                        "pr_moments_workspace"):
            getattr(L, name).restype = i32
    _lib = L
    return L


def status_string(code: int) -> str:
    return lib().pr_status_string(code).decode()


def version() -> str:
    return lib().pr_version().decode()


def _ptr(t) -> int | None:
    if t is None:
        return None
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _check(fn: str, rc: int):
    if rc != PR_OK:
        raise PrError(fn, rc)


def pr_fine_propagate(model: Model, precision: int, rng: Rng, x_in, y_in, broadcast_input: bool,
                      x_out, y_out, n: int, slice_begin: int, n_slices: int, steps: int, dt: float,
                      grid: Grid | None = None, cdf_prior=None, cdf_target=None, counts_start=None,
                      cdf_start=None, counts_end=None, cdf_end=None, stream=None):
    m, r = model.c(), rng.c()
    g = grid.c() if grid is not None else None
    rc = lib().pr_fine_propagate(ctypes.byref(m), precision, ctypes.byref(r), _ptr(x_in), _ptr(y_in),
                                 1 if broadcast_input else 0, _ptr(x_out), _ptr(y_out), n, slice_begin,
                                 n_slices, steps, dt, ctypes.byref(g) if g is not None else None,
                                 _ptr(cdf_prior), _ptr(cdf_target), _ptr(counts_start), _ptr(cdf_start),
                                 _ptr(counts_end), _ptr(cdf_end), _stream(stream))
    _check("pr_fine_propagate", rc)


def pr_rng_words(rng: Rng, ctr, n: int, out, stream=None):
    r = rng.c()
    _check("pr_rng_words", lib().pr_rng_words(ctypes.byref(r), _ptr(ctr), n, _ptr(out), _stream(stream)))


def pr_set_particles_per_thread(ppt: int):
    lib().pr_set_particles_per_thread(ppt)


def pr_set_tiles_per_cta(tiles: int):
    lib().pr_set_tiles_per_cta(tiles)


def pr_set_update_cluster(ctas: int):
    lib().pr_set_update_cluster(ctas)


def pr_restrict(precision: int, x, n: int, n_slices: int, grid: Grid, counts, cdf=None, stream=None):
    g = grid.c()
    _check("pr_restrict", lib().pr_restrict(precision, _ptr(x), n, n_slices, ctypes.byref(g), _ptr(counts),
                                            _ptr(cdf), _stream(stream)))


def pr_counts_to_cdf(counts, n: int, n_slices: int, bins: int, cdf, stream=None):
    _check("pr_counts_to_cdf", lib().pr_counts_to_cdf(_ptr(counts), n, n_slices, bins, _ptr(cdf),
                                                      _stream(stream)))


def pr_match(precision: int, x_prior, x_out, n: int, n_slices: int, grid: Grid, cdf_prior, cdf_target,
             stream=None):
    g = grid.c()
    _check("pr_match", lib().pr_match(precision, _ptr(x_prior), _ptr(x_out), n, n_slices, ctypes.byref(g),
                                      _ptr(cdf_prior), _ptr(cdf_target), _stream(stream)))


def pr_coarse_create(model: Model, grid: Grid, slice_dt: float, stream=None) -> int:
    m, g = model.c(), grid.c()
    h = ctypes.c_void_p()
    _check("pr_coarse_create", lib().pr_coarse_create(ctypes.byref(m), ctypes.byref(g), slice_dt,
                                                      ctypes.byref(h), _stream(stream)))
    return h.value


def pr_coarse_destroy(handle: int):
    _check("pr_coarse_destroy", lib().pr_coarse_destroy(handle))


def pr_coarse_matrix(handle: int, out, stream=None):
    _check("pr_coarse_matrix", lib().pr_coarse_matrix(handle, _ptr(out), _stream(stream)))


def pr_coarse_fp(handle: int, cdf_in, cdf_out, n_vec: int, stream=None):
    _check("pr_coarse_fp", lib().pr_coarse_fp(handle, _ptr(cdf_in), _ptr(cdf_out), n_vec, _stream(stream)))


def pr_parareal_update(coarse: int, iterator: int, qmode: int, n_slices: int, cdf0, cdf_f_star, cdf_c_star,
                       cdf_next, status=None, stream=None):
    _check("pr_parareal_update", lib().pr_parareal_update(coarse, iterator, qmode, n_slices, _ptr(cdf0),
                                                          _ptr(cdf_f_star), _ptr(cdf_c_star), _ptr(cdf_next),
                                                          _ptr(status), _stream(stream)))


def pr_iterate(iterator: int, qmode: int, grid: Grid, n_vec: int, a, b, c, out, status=None, stream=None):
    g = grid.c()
    _check("pr_iterate", lib().pr_iterate(iterator, qmode, ctypes.byref(g), n_vec, _ptr(a), _ptr(b), _ptr(c),
                                          _ptr(out), _ptr(status), _stream(stream)))


def pr_w1(grid: Grid, n_vec: int, c1, c2, w1, stream=None):
    g = grid.c()
    _check("pr_w1", lib().pr_w1(ctypes.byref(g), n_vec, _ptr(c1), _ptr(c2), _ptr(w1), _stream(stream)))


def pr_l2_density(grid: Grid, n_vec: int, c1, c2, l2, stream=None):
    g = grid.c()
    _check("pr_l2_density", lib().pr_l2_density(ctypes.byref(g), n_vec, _ptr(c1), _ptr(c2), _ptr(l2),
                                                _stream(stream)))


def pr_fine_adjoint_workspace(n: int, n_slices: int, steps: int, ckpt_every: int) -> int:
    return lib().pr_fine_adjoint_workspace(n, n_slices, steps, ckpt_every)


def pr_fine_adjoint(model: Model, rng: Rng, x0, y0, n: int, slice_begin: int, n_slices: int, steps: int,
                    dt: float, ckpt_every: int, x_T, y_T, xbar_T, ybar_T, grad, xbar_0, ybar_0, workspace,
                    stream=None):
    m, r = model.c(), rng.c()
    wbytes = workspace.numel() * workspace.element_size()
    _check("pr_fine_adjoint", lib().pr_fine_adjoint(ctypes.byref(m), ctypes.byref(r), _ptr(x0), _ptr(y0), n,
                                                    slice_begin, n_slices, steps, dt, ckpt_every, _ptr(x_T),
                                                    _ptr(y_T), _ptr(xbar_T), _ptr(ybar_T), _ptr(grad),
                                                    _ptr(xbar_0), _ptr(ybar_0), _ptr(workspace), wbytes,
                                                    _stream(stream)))


def pr_fine_adjoint_affine(model: Model, rng: Rng, x0, y0, n: int, slice_begin: int, n_slices: int, steps: int,
                           dt: float, ckpt_every: int, seed_scale: float, seed_shift: float, x_T, y_T, grad, xbar_0,
                           ybar_0, workspace, stream=None):
    m, r = model.c(), rng.c()
    wbytes = workspace.numel() * workspace.element_size()
    _check("pr_fine_adjoint_affine",
           lib().pr_fine_adjoint_affine(ctypes.byref(m), ctypes.byref(r), _ptr(x0), _ptr(y0), n, slice_begin, n_slices,
                                        steps, dt, ckpt_every, float(seed_scale), float(seed_shift), _ptr(x_T),
                                        _ptr(y_T), _ptr(grad), _ptr(xbar_0), _ptr(ybar_0), _ptr(workspace), wbytes,
                                        _stream(stream)))


def pr_order_statistics_workspace(n: int) -> int:
    return lib().pr_order_statistics_workspace(n)


def pr_reweight(precision: int, x_prior, broadcast_input: bool, w_prior, n: int, n_slices: int, grid: Grid,
                cdf_prior, cdf_target, w_out, stream=None):
    g = grid.c()
    _check("pr_reweight", lib().pr_reweight(precision, _ptr(x_prior), int(bool(broadcast_input)), _ptr(w_prior), n,
                                            n_slices, ctypes.byref(g), _ptr(cdf_prior), _ptr(cdf_target),
                                            _ptr(w_out), _stream(stream)))


def pr_resample_workspace(n: int, n_slices: int) -> int:
    return lib().pr_resample_workspace(n, n_slices)


def pr_resample(precision: int, fast_dim: int, x_in, y_in, broadcast_input: bool, w, n: int, n_slices: int,
                slice_begin: int, mode: int, rng: Rng, index_out, x_out, y_out, workspace, stream=None):
    r = rng.c()
    wbytes = workspace.numel() * workspace.element_size()
    _check("pr_resample", lib().pr_resample(precision, fast_dim, _ptr(x_in), _ptr(y_in), int(bool(broadcast_input)),
                                            _ptr(w), n, n_slices, slice_begin, mode, ctypes.byref(r),
                                            _ptr(index_out), _ptr(x_out), _ptr(y_out), _ptr(workspace), wbytes,
                                            _stream(stream)))


def pr_restrict_weighted_workspace(n_slices: int, bins: int) -> int:
    return lib().pr_restrict_weighted_workspace(n_slices, bins)


def pr_restrict_weighted(precision: int, x, broadcast_input: bool, w, n: int, n_slices: int, grid: Grid, cdf,
                         workspace, stream=None):
    g = grid.c()
    wbytes = workspace.numel() * workspace.element_size()
    _check("pr_restrict_weighted", lib().pr_restrict_weighted(precision, _ptr(x), int(bool(broadcast_input)),
                                                              _ptr(w), n, n_slices,
                                                              ctypes.byref(g), _ptr(cdf), _ptr(workspace), wbytes,
                                                              _stream(stream)))


def pr_moments_workspace(n: int, n_slices: int, max_order: int) -> int:
    return lib().pr_moments_workspace(n, n_slices, max_order)


def pr_moments(precision: int, v, slice_stride: int, w, n: int, n_slices: int, max_order: int, out, workspace,
               stream=None):
    wbytes = workspace.numel() * workspace.element_size()
    _check("pr_moments", lib().pr_moments(precision, _ptr(v), slice_stride, _ptr(w), n, n_slices, max_order,
                                          _ptr(out), _ptr(workspace), wbytes, _stream(stream)))


def pr_order_statistics(x, n: int, ranks, n_ranks: int, index_out, workspace, stream=None):
    wbytes = workspace.numel() * workspace.element_size()
    _check("pr_order_statistics", lib().pr_order_statistics(_ptr(x), n, _ptr(ranks), n_ranks, _ptr(index_out),
                                                            _ptr(workspace), wbytes, _stream(stream)))


def pr_fine_adjoint_noalloc_capacity() -> int:
    return lib().pr_fine_adjoint_noalloc_capacity()


def pr_fine_adjoint_noalloc(model: Model, rng: Rng, x0, y0, n: int, slice_begin: int, n_slices: int, steps: int,
                            dt: float, ckpt_every: int, x_T, y_T, xbar_T, ybar_T, grad, xbar_0, ybar_0,
                            stream=None):
    """pr_fine_adjoint with its scratch in the library's fixed device array
    (for callers that must not allocate device memory while they run)."""
    m, r = model.c(), rng.c()
    _check("pr_fine_adjoint_noalloc",
           lib().pr_fine_adjoint_noalloc(ctypes.byref(m), ctypes.byref(r), _ptr(x0), _ptr(y0), n, slice_begin,
                                         n_slices, steps, dt, ckpt_every, _ptr(x_T), _ptr(y_T), _ptr(xbar_T),
                                         _ptr(ybar_T), _ptr(grad), _ptr(xbar_0), _ptr(ybar_0), _stream(stream)))


def pr_batch_create(problems, iterator: int = PR_ITER_QUANTILE, qmode: int = PR_QMODE_TWO_SIDED,
                    stream=None) -> int:
    arr = (_Problem * len(problems))(*[p.c() for p in problems])
    h = ctypes.c_void_p()
    _check("pr_batch_create", lib().pr_batch_create(arr, len(problems), iterator, qmode, ctypes.byref(h),
                                                    _stream(stream)))
    return h.value


def pr_batch_destroy(plan: int):
    _check("pr_batch_destroy", lib().pr_batch_destroy(plan))


def pr_batch_particle_steps(plan: int) -> int:
    return lib().pr_batch_particle_steps(plan)


def pr_batch_set_initial(plan: int, x0, y0, stream=None):
    _check("pr_batch_set_initial", lib().pr_batch_set_initial(plan, _ptr(x0), _ptr(y0), _stream(stream)))


def pr_batch_iterate(plan: int, stream=None):
    _check("pr_batch_iterate", lib().pr_batch_iterate(plan, _stream(stream)))


def pr_batch_rho(plan: int, problem: int, out, stream=None):
    _check("pr_batch_rho", lib().pr_batch_rho(plan, problem, _ptr(out), _stream(stream)))


def pr_batch_fine_state(plan: int, problem: int, x_out, y_out, stream=None):
    _check("pr_batch_fine_state", lib().pr_batch_fine_state(plan, problem, _ptr(x_out), _ptr(y_out),
                                                            _stream(stream)))


def pr_batch_status(plan: int, stream=None) -> int:
    w = ctypes.c_int32()
    _check("pr_batch_status", lib().pr_batch_status(plan, ctypes.byref(w), _stream(stream)))
    return w.value


def pr_batch_set_config(plan: int, ppt: int, item_work: float):
    _check("pr_batch_set_config", lib().pr_batch_set_config(plan, ppt, item_work))


def pr_batch_get_config(plan: int):
    ppt, work, items = ctypes.c_int32(), ctypes.c_double(), ctypes.c_int32()
    _check("pr_batch_get_config", lib().pr_batch_get_config(plan, ctypes.byref(ppt), ctypes.byref(work),
                                                            ctypes.byref(items)))
    return ppt.value, work.value, items.value


def pr_batch_tune(plan: int, steps_div: int = 8, stream=None) -> float:
    best = ctypes.c_double()
    _check("pr_batch_tune", lib().pr_batch_tune(plan, steps_div, ctypes.byref(best), _stream(stream)))
    return best.value


def _nbytes(t) -> int:
    return t.numel() * t.element_size()


def pr_copy_to_device(dst, src, stream=None):
    """Copy the host tensor `src` into the device tensor `dst` (same size in bytes)."""
    if _nbytes(dst) != _nbytes(src):
        raise ValueError("pr_copy_to_device: sizes differ")
    _check("pr_copy_to_device", lib().pr_copy_to_device(_ptr(dst), _ptr(src), _nbytes(src), _stream(stream)))


def pr_copy_to_host(dst, src, stream=None):
    """Copy the device tensor `src` into the host tensor `dst` (same size in bytes)."""
    if _nbytes(dst) != _nbytes(src):
        raise ValueError("pr_copy_to_host: sizes differ")
    _check("pr_copy_to_host", lib().pr_copy_to_host(_ptr(dst), _ptr(src), _nbytes(src), _stream(stream)))


def pr_stream_synchronize(stream=None):
    _check("pr_stream_synchronize", lib().pr_stream_synchronize(_stream(stream)))
