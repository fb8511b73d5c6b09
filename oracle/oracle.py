"""Plain FP64 CPU oracle of the micro-macro parareal hot path.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  It shares no code with the CUDA library and never imports it.

The per-particle and per-bin work is plain C in ``oracle.c`` (loaded through
ctypes); the coarse Fokker-Planck propagator is assembled here entry by entry
from the finite-volume fluxes of Section 2.2.2 and exponentiated with
``scipy.linalg.expm`` (a library primitive).  The parareal driver follows
Sections 3.2.3-3.2.4 step by step.

Parity pins live in ``tests/test_oracle_*.py``; every function below is pinned
(no "parity unpinned" function remains in this module).
"""
from __future__ import annotations

import ctypes
import functools
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")

MODEL_OU, MODEL_DOUBLE_WELL, MODEL_DW_MULTI, MODEL_ADVECTION = 0, 1, 2, 3
MODEL_CHEM, MODEL_CHEM_PRINTED = 4, 5


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc, FP64, no contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call([
            "gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
            "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d, i64, i32, u32, u64 = (ctypes.c_double, ctypes.c_int64, ctypes.c_int,
                                 ctypes.c_uint32, ctypes.c_uint64)
        vp = ctypes.c_void_p
        _lib.or_num_threads.restype = i32
        _lib.or_set_num_threads.argtypes = [i32]
        _lib.or_philox_batch.argtypes = [vp, i64, u64, vp]
        _lib.or_uniform.argtypes = [u32]
        _lib.or_uniform.restype = d
        _lib.or_step_normals.argtypes = [u64, u32, u32, u32, u32, i32, vp]
        _lib.or_normals_block.argtypes = [u64, u32, u32, i64, u32, u32, i32, i32, vp]
        _lib.or_fine_propagate_chem.argtypes = [i32, vp, d, d, u64, u32, vp, vp, i64, vp, i32, i32, i32, d]
        _lib.or_chem_coefficients.argtypes = [i32, vp, d, d, vp]
        _lib.or_l2_density.argtypes = [i32, d, d, vp, vp]
        _lib.or_l2_density.restype = d
        _lib.or_fine_propagate.argtypes = [i32, i32, d, d, d, d, u64, u32, vp, vp, i64,
                                           i32, i32, i32, d]
        _lib.or_fine_propagate_ids.argtypes = [i32, i32, d, d, d, d, u64, u32, vp, vp, i64, vp,
                                               i32, i32, i32, d]
        _lib.or_fine_tangent.argtypes = [i32, d, d, d, d, u64, u32, vp, vp, i64, vp, i32, i32, i32, d,
                                          vp, vp, vp, vp]
        _lib.or_edge.argtypes = [i32, i32, d, d]
        _lib.or_edge.restype = d
        _lib.or_bin.argtypes = [d, i32, d, d]
        _lib.or_bin.restype = i32
        _lib.or_restrict.argtypes = [vp, i64, i32, i32, d, d, vp, vp]
        _lib.or_match.argtypes = [vp, vp, i64, i32, i32, d, d, vp, vp]
        _lib.or_quantile_update.argtypes = [i32, d, d, i32, vp, vp, vp, vp]
        _lib.or_quantile_update.restype = i32
        _lib.or_iterator_mass.argtypes = [i32, i32, vp, vp, vp, vp]
        _lib.or_w1.argtypes = [i32, d, d, vp, vp]
        _lib.or_w1.restype = d
        _lib.or_reweight_factors.argtypes = [i32, vp, vp, vp]
        _lib.or_reweight.argtypes = [vp, vp, i64, i32, i32, d, d, vp, vp, vp]
        _lib.or_weight_fixed.argtypes = [d]
        _lib.or_weight_fixed.restype = u64
        _lib.or_resample.argtypes = [vp, i64, i32, i32, u64, u32, u32, vp]
        _lib.or_restrict_weighted.argtypes = [vp, vp, i64, i32, i32, d, d, vp]
        _lib.or_moments.argtypes = [vp, i64, vp, i64, i32, i32, vp]
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------
# Model and grid descriptions
# --------------------------------------------------------------------------

@dataclass(frozen=True)
class Model:
    """Slow-fast SDE of Section 2.1.1 with tau_x = 1 unless given.

    kind 0: d_x F = x - lambda*y           (linear OU family)
    kind 1: d_x F = x^3 - x + lambda*y     (double well)
    kind 2: d_x F = x^3 - x + lambda*mean(y), y in R^d
    kind 3: no microscopic model; the coarse potential Fbar(x) = x/eps (the
            linear advection test of Section 6), diffusion 1/beta
    fast:   d_y G = y - x per component, E = 1; slow diffusion D = 1/beta.
    kind 4: the chemically reacting system of Section 2.1.2 with rates
            k0..k5 (`rates`), drifts read as the net reaction rates
            (chemical Langevin form; see oracle.c); kind 5: the same with
            the drifts of the potentials as printed.  fast_dim = 1; lam and
            beta unused.
    """
    kind: int
    fast_dim: int = 1
    lam: float = 1.0
    beta: float = 1.0
    eps: float = 0.1
    tau_x: float = 1.0
    rates: tuple = ()

    @property
    def chem(self) -> bool:
        return self.kind in (MODEL_CHEM, MODEL_CHEM_PRINTED)

    def rates_array(self) -> np.ndarray:
        k = np.ascontiguousarray(self.rates, dtype=np.float64)
        assert k.shape == (6,), "the chemical system needs six rates k0..k5"
        return k


@dataclass(frozen=True)
class Grid:
    bins: int
    lo: float
    hi: float

    @property
    def h(self) -> float:
        return (self.hi - self.lo) / self.bins

    def edges(self) -> np.ndarray:
        return np.array([lib().or_edge(i, self.bins, self.lo, self.hi)
                         for i in range(self.bins + 1)])


# --------------------------------------------------------------------------
# RNG
# --------------------------------------------------------------------------

def num_threads() -> int:
    return lib().or_num_threads()


def set_num_threads(n: int) -> None:
    """Cap the oracle's OpenMP threads (n >= 1); timing only, results do not depend on it."""
    lib().or_set_num_threads(int(n))


def philox(ctr: np.ndarray, seed: int) -> np.ndarray:
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.empty_like(ctr)
    lib().or_philox_batch(_p(ctr), ctr.shape[0], seed, _p(out))
    return out


def uniform(w: int) -> float:
    return lib().or_uniform(w)


def step_normals(seed: int, problem: int, p: int, n: int, m: int, Q: int) -> np.ndarray:
    z = np.empty(Q, dtype=np.float64)
    lib().or_step_normals(seed, problem, p, n, m, Q, _p(z))
    return z


def normals_block(seed: int, problem: int, p0: int, n_part: int, n: int, m0: int,
                  n_steps: int, Q: int) -> np.ndarray:
    out = np.empty((n_part, n_steps, Q), dtype=np.float64)
    lib().or_normals_block(seed, problem, p0, n_part, n, m0, n_steps, Q, _p(out))
    return out


# --------------------------------------------------------------------------
# Fine propagator (Section 2.1.3, Eqs. EMx/EMy)
# --------------------------------------------------------------------------

def fine_propagate(model: Model, seed: int, x: np.ndarray, y: np.ndarray, slice_begin: int,
                   steps: int, dt: float, problem: int = 0, ids: np.ndarray | None = None):
    """Advance x[n_slices][N], y[n_slices][d][N] (copies) by `steps` EM steps per slice.
    ids[N]: particle indices keying the random numbers of each column (default 0..N-1)."""
    x = np.array(x, dtype=np.float64, order="C", copy=True)
    y = np.array(y, dtype=np.float64, order="C", copy=True)
    n_slices, N = x.shape
    assert y.shape == (n_slices, model.fast_dim, N)
    if model.chem:
        assert model.fast_dim == 1
        k = model.rates_array()
        idp = None
        if ids is not None:
            ids = np.ascontiguousarray(ids, dtype=np.uint32)
            assert ids.shape == (N,)
            idp = _p(ids)
        lib().or_fine_propagate_chem(model.kind - MODEL_CHEM, _p(k), model.eps, model.tau_x, seed, problem,
                                     _p(x), _p(y), N, idp, slice_begin, n_slices, steps, dt)
        return x, y
    if ids is None:
        lib().or_fine_propagate(model.kind, model.fast_dim, model.lam, model.beta, model.eps,
                                model.tau_x, seed, problem, _p(x), _p(y), N, slice_begin,
                                n_slices, steps, dt)
    else:
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        assert ids.shape == (N,)
        lib().or_fine_propagate_ids(model.kind, model.fast_dim, model.lam, model.beta, model.eps,
                                    model.tau_x, seed, problem, _p(x), _p(y), N, _p(ids),
                                    slice_begin, n_slices, steps, dt)
    return x, y


def fine_tangent(model: Model, seed: int, x0: np.ndarray, y0: np.ndarray, slice_begin: int,
                 n_slices: int, steps: int, dt: float, problem: int = 0, ids: np.ndarray | None = None):
    """Forward-mode pathwise derivatives with fixed noise (d = 1 families).

    Returns X_T, Y_T [N] and dX_T, dY_T [N][5] with respect to
    (lambda, beta, eps, x0, y0)."""
    assert model.fast_dim == 1 and model.kind in (MODEL_OU, MODEL_DOUBLE_WELL)
    x0 = np.ascontiguousarray(x0, dtype=np.float64).reshape(-1)
    y0 = np.ascontiguousarray(y0, dtype=np.float64).reshape(-1)
    N = x0.shape[0]
    xo, yo = np.empty(N), np.empty(N)
    dx, dy = np.empty((N, 5)), np.empty((N, 5))
    idp = None
    if ids is not None:
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        assert ids.shape == (N,)
        idp = _p(ids)
    lib().or_fine_tangent(model.kind, model.lam, model.beta, model.eps, model.tau_x, seed, problem,
                          _p(x0), _p(y0), N, idp, slice_begin, n_slices, steps, dt, _p(xo), _p(yo), _p(dx), _p(dy))
    return xo, yo, dx, dy


# --------------------------------------------------------------------------
# Restriction, matching, iterators, W1
# --------------------------------------------------------------------------

def bin_index(x: float, grid: Grid) -> int:
    return lib().or_bin(float(x), grid.bins, grid.lo, grid.hi)


def restrict(x: np.ndarray, grid: Grid):
    """x[n_slices][N] -> (counts[n_slices][I] uint32, cdf[n_slices][I+1])."""
    x = np.ascontiguousarray(np.atleast_2d(x), dtype=np.float64)
    n_slices, N = x.shape
    counts = np.empty((n_slices, grid.bins), dtype=np.uint32)
    cdf = np.empty((n_slices, grid.bins + 1), dtype=np.float64)
    lib().or_restrict(_p(x), N, n_slices, grid.bins, grid.lo, grid.hi, _p(counts), _p(cdf))
    return counts, cdf


def match(x_prior: np.ndarray, grid: Grid, cdf_prior: np.ndarray, cdf_target: np.ndarray):
    x_prior = np.ascontiguousarray(np.atleast_2d(x_prior), dtype=np.float64)
    n_slices, N = x_prior.shape
    cp = np.ascontiguousarray(np.atleast_2d(cdf_prior), dtype=np.float64)
    ct = np.ascontiguousarray(np.atleast_2d(cdf_target), dtype=np.float64)
    assert cp.shape == ct.shape == (n_slices, grid.bins + 1)
    out = np.empty_like(x_prior)
    lib().or_match(_p(x_prior), _p(out), N, n_slices, grid.bins, grid.lo, grid.hi, _p(cp), _p(ct))
    return out


# --------------------------------------------------------------------------
# Matching preserving the conditional distribution (Section 5.2)
# --------------------------------------------------------------------------

RESAMPLE_STRATIFIED, RESAMPLE_DETERMINISTIC = 0, 1


def reweight_factors(grid: Grid, cdf_prior: np.ndarray, cdf_target: np.ndarray) -> np.ndarray:
    """r_i = rho'_i / rhobar_i for one prior/target pair (mass of target bins
    the prior does not support moved half left, half right)."""
    cp = np.ascontiguousarray(cdf_prior, dtype=np.float64)
    ct = np.ascontiguousarray(cdf_target, dtype=np.float64)
    r = np.empty(grid.bins)
    lib().or_reweight_factors(grid.bins, _p(cp), _p(ct), _p(r))
    return r


def reweight(x: np.ndarray, grid: Grid, cdf_prior: np.ndarray, cdf_target: np.ndarray,
             wbar: np.ndarray | None = None) -> np.ndarray:
    """W^p = Wbar^p rho'_i / rhobar_i; x, wbar: [n_slices][N] (wbar None: 1/N)."""
    x = np.ascontiguousarray(np.atleast_2d(x), dtype=np.float64)
    n_slices, N = x.shape
    cp = np.ascontiguousarray(np.atleast_2d(cdf_prior), dtype=np.float64)
    ct = np.ascontiguousarray(np.atleast_2d(cdf_target), dtype=np.float64)
    assert cp.shape == ct.shape == (n_slices, grid.bins + 1)
    wb = None if wbar is None else np.ascontiguousarray(np.atleast_2d(wbar), dtype=np.float64)
    w = np.empty_like(x)
    lib().or_reweight(_p(x), None if wb is None else _p(wb), N, n_slices, grid.bins, grid.lo, grid.hi,
                      _p(cp), _p(ct), _p(w))
    return w


def weight_fixed(w) -> int:
    """round(w 2^61) as an integer (the fixed point of the cumulative weights)."""
    return int(lib().or_weight_fixed(float(w)))


def resample(w: np.ndarray, mode: int, seed: int, slice_begin: int, problem: int = 0) -> np.ndarray:
    """Stratified (mode 0) or deterministic (mode 1) resampling: index[n_slices][N]
    of the particle each output takes."""
    w = np.ascontiguousarray(np.atleast_2d(w), dtype=np.float64)
    n_slices, N = w.shape
    idx = np.empty((n_slices, N), dtype=np.uint32)
    lib().or_resample(_p(w), N, n_slices, mode, seed, problem, slice_begin, _p(idx))
    return idx


def restrict_weighted(x: np.ndarray, w: np.ndarray, grid: Grid) -> np.ndarray:
    """Weighted restriction: CDFs [n_slices][I+1] of the bin sums of the weights."""
    x = np.ascontiguousarray(np.atleast_2d(x), dtype=np.float64)
    w = np.ascontiguousarray(np.atleast_2d(w), dtype=np.float64)
    n_slices, N = x.shape
    assert w.shape == x.shape
    cdf = np.empty((n_slices, grid.bins + 1))
    lib().or_restrict_weighted(_p(x), _p(w), N, n_slices, grid.bins, grid.lo, grid.hi, _p(cdf))
    return cdf


def moments(v: np.ndarray, Q: int, w: np.ndarray | None = None) -> np.ndarray:
    """Monte Carlo estimator (Eq. MCestimator) of v^q, q = 1..Q, per slice:
    [n_slices][Q], weights w [n_slices][n] or uniform 1/n."""
    v = np.ascontiguousarray(np.atleast_2d(v), dtype=np.float64)
    n_slices, n = v.shape
    if w is not None:
        w = np.ascontiguousarray(np.atleast_2d(w), dtype=np.float64)
        assert w.shape == v.shape
    out = np.empty((n_slices, Q))
    lib().or_moments(_p(v), n, None if w is None else _p(w), n, n_slices, Q, _p(out))
    return out


QMODE_TWO_SIDED, QMODE_MIDPOINT = 0, 1
ITER_QUANTILE, ITER_ADD, ITER_MULT, ITER_ROT = 0, 1, 2, 3


def iterate(grid: Grid, a: np.ndarray, b: np.ndarray, c: np.ndarray,
            iterator: int = ITER_QUANTILE, qmode: int = QMODE_TWO_SIDED) -> np.ndarray:
    """J(a = rho_c^{n+1}, b = rho_f^*, c = rho_c^*) on CDFs; returns the new CDF."""
    a, b, c = (np.ascontiguousarray(v, dtype=np.float64) for v in (a, b, c))
    out = np.empty(grid.bins + 1, dtype=np.float64)
    if iterator == ITER_QUANTILE:
        lib().or_quantile_update(grid.bins, grid.lo, grid.hi, qmode, _p(a), _p(b), _p(c), _p(out))
    else:
        lib().or_iterator_mass(iterator, grid.bins, _p(a), _p(b), _p(c), _p(out))
    return out


def w1(grid: Grid, c1: np.ndarray, c2: np.ndarray) -> float:
    c1 = np.ascontiguousarray(c1, dtype=np.float64)
    c2 = np.ascontiguousarray(c2, dtype=np.float64)
    return lib().or_w1(grid.bins, grid.lo, grid.hi, _p(c1), _p(c2))


def l2_density(grid: Grid, c1: np.ndarray, c2: np.ndarray) -> float:
    """L2 distance of the piecewise-constant densities of two CDFs (the
    histogram error of the experiments of Section 6)."""
    c1 = np.ascontiguousarray(c1, dtype=np.float64)
    c2 = np.ascontiguousarray(c2, dtype=np.float64)
    return lib().or_l2_density(grid.bins, grid.lo, grid.hi, _p(c1), _p(c2))


# --------------------------------------------------------------------------
# Coarse propagator (Section 2.2.2): finite volumes on the detailed-balance
# form of Eq. FPz_rewritten, exact in time through the matrix exponential.
# --------------------------------------------------------------------------

# Equilibrium of the chemical system's fast variable (Section 2.2.3): the mean
# ybar of phi(y) ~ exp(-int_0^y G'(s)/E(s) ds) / E(y) by the trapezoidal
# rule.  The paper does not give the quadrature grid; the reading is
# y_j = j * CHEM_DY, j = 0 .. CHEM_J (y in [0, 2000], far beyond both wells,
# where phi has decayed by many orders), the inner integral by the
# cumulative trapezoidal rule on the same grid.
CHEM_DY = 0.5
CHEM_J = 4000


def _chem_coefficients(reading: int, k: np.ndarray, x: float, y: float):
    out = np.empty(4)
    lib().or_chem_coefficients(reading, _p(k), x, y, _p(out))
    return out


def chem_coefficients(model: Model, x: float, y: float):
    """(d_x F, d_y G, D, E) of the chemical system at (x, y) (Section 2.1.2)."""
    return _chem_coefficients(model.kind - MODEL_CHEM, model.rates_array(), x, y)


def chem_ybar(model: Model) -> float:
    return _chem_ybar(model.kind, tuple(float(v) for v in model.rates_array()))


@functools.lru_cache(maxsize=64)
def _chem_ybar(kind: int, rates: tuple) -> float:
    k = np.ascontiguousarray(rates, dtype=np.float64)
    reading = kind - MODEL_CHEM
    y = np.array([j * CHEM_DY for j in range(CHEM_J + 1)])
    ratio = np.empty(CHEM_J + 1)            # G'(y) / E(y)
    log_e = np.empty(CHEM_J + 1)
    for j in range(CHEM_J + 1):
        _, dg, _, e = _chem_coefficients(reading, k, 0.0, y[j])
        ratio[j] = dg / e
        log_e[j] = np.log(e)
    integral = 0.0                           # int_0^{y_j} G'/E, cumulative trapezoid
    log_phi = np.empty(CHEM_J + 1)
    for j in range(CHEM_J + 1):
        if j:
            integral += 0.5 * CHEM_DY * (ratio[j - 1] + ratio[j])
        log_phi[j] = -integral - log_e[j]
    top = max(log_phi)
    num = den = 0.0
    for j in range(CHEM_J + 1):              # trapezoid weights 1/2 at the ends (dy cancels)
        wgt = 0.5 if j in (0, CHEM_J) else 1.0
        phi = np.exp(log_phi[j] - top)
        num += wgt * y[j] * phi
        den += wgt * phi
    return num / den


def effective_potential(model: Model, x):
    """Fbar(x) with Fbar(0) = 0, by averaging d_x F over phi(y; x) (Eq. Fbar).
    The fast OU has E[y | x] = x in every component; the chemical system's
    F is linear in y, so Fbar needs only ybar (Section 2.2.3)."""
    x = np.asarray(x, dtype=np.float64)
    if model.kind == MODEL_ADVECTION:     # given directly (Section 6, linear advection case)
        return x / model.eps
    if model.chem:
        k, yb = model.rates_array(), chem_ybar(model)
        if model.kind == MODEL_CHEM:      # F = -k4 x y + k5 x^2 / 2 (the net rates' potential)
            return -k[4] * x * yb + 0.5 * k[5] * x * x
        return -k[4] * x * yb - 0.5 * k[5] * x * x      # as printed
    if model.kind == MODEL_OU:
        return 0.5 * (1.0 - model.lam) * x * x
    return 0.25 * x ** 4 - 0.5 * (1.0 - model.lam) * x * x


def effective_diffusion(model: Model, x):
    """Dbar(x) (Eq. Dbar): 1/beta, or (k4 ybar + k5 x)/2 for the chemical system."""
    x = np.asarray(x, dtype=np.float64)
    if model.chem:
        k = model.rates_array()
        return 0.5 * (k[4] * chem_ybar(model) + k[5] * x)
    return np.full_like(x, 1.0 / model.beta)


def log_rho_inf(model: Model, x):
    """log rho_inf(x) = log(1/Dbar(x)) - int_0^x Fbar'(s)/Dbar(s) ds (Eq. FPz_rewritten).

    Constant Dbar: the integral is Fbar(x)/Dbar.  The chemical system, with
    a = k4 ybar, Dbar(s) = (a + k5 s)/2: Fbar'(s) = k5 s - a (net rates)
    gives int_0^x 2 (k5 s - a)/(a + k5 s) ds = 2x - (4a/k5) log(1 + k5 x/a);
    Fbar'(s) = -(a + k5 s) (as printed) gives -2x."""
    x = np.asarray(x, dtype=np.float64)
    if model.chem:
        k = model.rates_array()
        a = k[4] * chem_ybar(model)
        Dbar = 0.5 * (a + k[5] * x)
        if model.kind == MODEL_CHEM:
            integral = 2.0 * x - (4.0 * a / k[5]) * np.log1p(k[5] * x / a)
        else:
            integral = -2.0 * x
        return np.log(1.0 / Dbar) - integral
    Dbar = 1.0 / model.beta
    return np.log(1.0 / Dbar) - effective_potential(model, x) / Dbar


def coarse_generator(model: Model, grid: Grid) -> np.ndarray:
    """A with d m/dt = A m for the cell masses m_c (zero flux at both ends).

    Flux at interior edge e between cells e-1 and e:
      phi_e = Dbar(x_e) rho_inf(x_e) / h_e * ( m_e / (h_{e+1/2} rho_inf(xi_e))
                                       - m_{e-1} / (h_{e-1/2} rho_inf(xi_{e-1})) )
    with h_e the distance between the two centres; dm_c/dt = (phi_{c+1} - phi_c)/tau_x.
    """
    I = grid.bins
    x = grid.edges()
    xi = 0.5 * (x[:-1] + x[1:])
    width = x[1:] - x[:-1]
    A = np.zeros((I, I), dtype=np.float64)
    for e in range(1, I):
        h_e = xi[e] - xi[e - 1]
        coef = float(effective_diffusion(model, x[e])) / h_e
        r_right = np.exp(log_rho_inf(model, x[e]) - log_rho_inf(model, xi[e])) / width[e]
        r_left = np.exp(log_rho_inf(model, x[e]) - log_rho_inf(model, xi[e - 1])) / width[e - 1]
        # phi_e = coef * (r_right * m_e - r_left * m_{e-1})
        # cell e-1 gains +phi_e (its right edge), cell e loses phi_e (its left edge)
        A[e - 1, e] += coef * r_right / model.tau_x
        A[e - 1, e - 1] -= coef * r_left / model.tau_x
        A[e, e] -= coef * r_right / model.tau_x
        A[e, e - 1] += coef * r_left / model.tau_x
    return A


def coarse_propagator(model: Model, grid: Grid, slice_dt: float) -> np.ndarray:
    import scipy.linalg
    return scipy.linalg.expm(coarse_generator(model, grid) * slice_dt)


TAIL_MASS = 1e-10


def coarse_apply(P: np.ndarray, cdf: np.ndarray) -> np.ndarray:
    """C(rho) on a CDF: masses, P @ masses (masses <= TAIL_MASS dropped),
    cumulative sum normalised to 1."""
    cdf = np.atleast_2d(np.asarray(cdf, dtype=np.float64))
    out = np.empty_like(cdf)
    for r in range(cdf.shape[0]):
        m = cdf[r, 1:] - cdf[r, :-1]
        # bin masses at or below TAIL_MASS are set to 0: below that level the
        # entries of P @ m are rounding noise of the matrix exponential
        # (absolute error ~1e-15), which would otherwise decide where the
        # support of the result ends (and so the quantile iterator's q(0) and
        # q(1)); this also clips negative round-off, keeping the CDF monotone
        mp = P @ m
        mp = np.where(mp > TAIL_MASS, mp, 0.0)
        s = np.cumsum(mp)
        out[r, 0] = 0.0
        out[r, 1:] = s / s[-1]
        out[r, -1] = 1.0
    return out


# --------------------------------------------------------------------------
# Micro-macro parareal driver (Sections 3.2.3-3.2.4), viewpoint (i)
# --------------------------------------------------------------------------

@dataclass
class PararealResult:
    x: list           # x[k] = array [K+1][N], X_k^n (slow)
    y: list           # y[k] = array [K+1][d][N]
    rho: list         # rho[k] = CDFs [K+1][I+1], rho_k^n
    serial_x: np.ndarray | None = None
    serial_rho: np.ndarray | None = None
    w: list | None = None   # w[k] = weights [K+1][N] (uniform 1/N except in "reweight" mode)


def serial_fine(model: Model, seed: int, x0, y0, K: int, steps: int, dt: float, problem: int = 0):
    """X^{n+1} = F_n(X^n), n = 0..K-1 -> x[K+1][N], y[K+1][d][N]."""
    N = x0.shape[-1]
    d = model.fast_dim
    xs = np.empty((K + 1, N))
    ys = np.empty((K + 1, d, N))
    xs[0] = x0
    ys[0] = y0
    for n in range(K):
        xn, yn = fine_propagate(model, seed, xs[n][None], ys[n][None], n, steps, dt, problem)
        xs[n + 1] = xn[0]
        ys[n + 1] = yn[0]
    return xs, ys


MATCHINGS = ("quantile", "resample", "resample_det", "reweight")


def _conditional_match(grid: Grid, xp, yp, cdf_prior, cdf_target, matching: str, seed: int, problem: int,
                       slice_begin: int, wbar=None):
    """Section 5.2 on slices slice_begin..: reweight the priors xp[S][N] (weights
    wbar, None: 1/N) to the targets, then resample (stratified or u~ = 1/2) or
    keep the weights.  Returns (x, y, w) with w None after resampling."""
    w = reweight(xp, grid, cdf_prior, cdf_target, wbar)
    if matching == "reweight":
        return xp.copy(), yp.copy(), w
    mode = RESAMPLE_STRATIFIED if matching == "resample" else RESAMPLE_DETERMINISTIC
    idx = resample(w, mode, seed, slice_begin, problem).astype(np.int64)
    x = np.take_along_axis(xp, idx, axis=1)
    y = np.stack([yp[s][:, idx[s]] for s in range(xp.shape[0])])
    return x, y, None


def parareal(model: Model, grid: Grid, seed: int, x0, y0, K: int, steps: int, dt: float,
             iters: int, qmode: int = QMODE_TWO_SIDED, iterator: int = ITER_QUANTILE,
             problem: int = 0, matching: str = "quantile") -> PararealResult:
    """Sections 3.2.3-3.2.4 with the matching of Section 5.1 ("quantile") or
    of Section 5.2 ("resample": reweighting and stratified resampling,
    "resample_det": u~ = 1/2, "reweight": weights carried by the ensembles,
    restrictions weighted).  res.w[k] holds the weights in "reweight" mode."""
    assert matching in MATCHINGS
    x0 = np.asarray(x0, dtype=np.float64)
    y0 = np.asarray(y0, dtype=np.float64).reshape(model.fast_dim, -1)
    N = x0.shape[0]
    weighted = matching == "reweight"
    uni = np.full(N, 1.0 / N)
    R = (lambda x, w: restrict_weighted(x, w, grid)) if weighted else (lambda x, w: restrict(x, grid)[1])
    P = coarse_propagator(model, grid, steps * dt)
    cdf0 = R(x0[None], uni[None])[0]

    # iteration 0: coarse sweep, then matching against the initial ensemble
    rho = np.empty((K + 1, grid.bins + 1))
    rho[0] = cdf0
    for n in range(K):
        rho[n + 1] = coarse_apply(P, rho[n])[0]
    X = np.empty((K + 1, N))
    Y = np.empty((K + 1, model.fast_dim, N))
    W = np.tile(uni, (K + 1, 1))
    X[0] = x0
    Y[0] = y0
    if matching == "quantile":
        for n in range(1, K + 1):
            X[n] = match(x0[None], grid, cdf0[None], rho[n][None])[0]
            Y[n] = y0
    else:
        xs, ys, ws = _conditional_match(grid, np.tile(x0, (K, 1)), np.tile(y0, (K, 1, 1)),
                                        np.tile(cdf0, (K, 1)), rho[1:], matching, seed, problem, 1)
        X[1:], Y[1:] = xs, ys
        if ws is not None:
            W[1:] = ws
    res = PararealResult(x=[X.copy()], y=[Y.copy()], rho=[rho.copy()])
    res.w = [W.copy()]

    for _k in range(iters):
        # parallel phase
        Xbar, Ybar = fine_propagate(model, seed, X[:K], Y[:K], 0, steps, dt, problem)
        f_star = R(Xbar, W[:K])
        start = R(X[:K], W[:K])
        c_star = coarse_apply(P, start)
        # serial phase
        new_rho = np.empty_like(rho)
        new_rho[0] = cdf0
        for n in range(K):
            a = coarse_apply(P, new_rho[n])[0]
            new_rho[n + 1] = iterate(grid, a, f_star[n], c_star[n], iterator, qmode)
        # matching with the fine results as priors
        Xn = np.empty_like(X)
        Yn = np.empty_like(Y)
        Wn = np.tile(uni, (K + 1, 1))
        Xn[0] = x0
        Yn[0] = y0
        if matching == "quantile":
            Xn[1:] = match(Xbar, grid, f_star, new_rho[1:])
            Yn[1:] = Ybar
        else:
            xs, ys, ws = _conditional_match(grid, Xbar, Ybar, f_star, new_rho[1:], matching, seed, problem, 1,
                                            W[:K] if weighted else None)
            Xn[1:], Yn[1:] = xs, ys
            if ws is not None:
                Wn[1:] = ws
        X, Y, W, rho = Xn, Yn, Wn, new_rho
        res.x.append(X.copy())
        res.y.append(Y.copy())
        res.rho.append(rho.copy())
        res.w.append(W.copy())
    return res


# --------------------------------------------------------------------------
# Parareal with the discretised Fokker-Planck equation as both propagators
# (Section 6, linear advection case): restriction and matching are the
# identity, the iterator is not.
# --------------------------------------------------------------------------

def fp_parareal(grid: Grid, fine: Model, coarse: Model, rho0: np.ndarray, K: int, dT: float, iters: int,
                iterator: int = ITER_QUANTILE, qmode: int = QMODE_TWO_SIDED) -> list:
    """rho[k] = CDFs [K+1][I+1] of iterations k = 0..iters, with
    rho_0^{n+1} = C rho_0^n and rho_{k+1}^{n+1} = J(C rho_{k+1}^n, F rho_k^n, C rho_k^n),
    F = exp(A_fine dT), C = exp(A_coarse dT)."""
    PF = coarse_propagator(fine, grid, dT)
    PC = coarse_propagator(coarse, grid, dT)
    rho = np.empty((K + 1, grid.bins + 1))
    rho[0] = rho0
    for n in range(K):
        rho[n + 1] = coarse_apply(PC, rho[n])[0]
    out = [rho.copy()]
    for _k in range(iters):
        f_star = coarse_apply(PF, rho[:K])
        c_star = coarse_apply(PC, rho[:K])
        new = np.empty_like(rho)
        new[0] = rho0
        for n in range(K):
            a = coarse_apply(PC, new[n])[0]
            new[n + 1] = iterate(grid, a, f_star[n], c_star[n], iterator, qmode)
        rho = new
        out.append(rho.copy())
    return out


def fp_serial(grid: Grid, fine: Model, rho0: np.ndarray, K: int, dT: float) -> np.ndarray:
    """rho^n = F^n rho0, n = 0..K (the reference the parareal iterates reach)."""
    PF = coarse_propagator(fine, grid, dT)
    rho = np.empty((K + 1, grid.bins + 1))
    rho[0] = rho0
    for n in range(K):
        rho[n + 1] = coarse_apply(PF, rho[n])[0]
    return rho
