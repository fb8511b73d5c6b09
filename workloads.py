"""Seeded synthetic workloads of the paper's shape.

This module holds the problem descriptions (model parameters, grid, slice
count, step size) and the seeded generators of the initial ensembles.  It
contains none of the method's arithmetic: both the CUDA path and the FP64
oracle receive the arrays generated here as inputs.

The paper uses no public dataset; its workloads are synthetic SDE ensembles
(Section 6).  The workloads below are synthetic ensembles; the first five are of the same
kind: a 1-D slow variable coupled to a fast Ornstein-Uhlenbeck variable, with
Gaussian initial conditions, uniform bin grids and uniform weights 1/N; the
chemical-reaction workload has the paper's own system, parameters and
lognormal initial conditions (Section 6, Table 1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MODEL_OU, MODEL_DOUBLE_WELL, MODEL_DW_MULTI = 0, 1, 2
MODEL_CHEM, MODEL_CHEM_PRINTED = 4, 5


@dataclass(frozen=True)
class Workload:
    name: str
    kind: int                 # drift family (see MODEL_*)
    fast_dim: int
    lam: float
    beta: float
    eps: float
    N: int                    # particles
    T: float                  # horizon
    K: int                    # parareal slices
    dt: float                 # fine EM step
    bins: int
    lo: float
    hi: float
    iters: int
    x0_mean: float
    x0_std: float
    y0: str                   # "normal01" (Y0 ~ N(0,1)), "x0" (Y0 = X0) or "lognormal" (see x0_dist)
    precision: str            # "f64" or "f32"
    seed: int = 0
    tau_x: float = 1.0
    rates: tuple = ()         # k0..k5 of the chemical system
    x0_dist: str = "normal"   # "normal", or "lognormal": X0 and Y0 independent lognormal of mean x0_mean, sd x0_std

    @property
    def slice_dt(self) -> float:
        return self.T / self.K

    @property
    def steps(self) -> int:
        """EM steps per slice; the smallest S with T/(K S) <= dt."""
        s = self.slice_dt / self.dt
        r = round(s)
        return int(r) if abs(s - r) < 1e-9 * max(1.0, s) else int(math.ceil(s))

    @property
    def step_dt(self) -> float:
        return self.slice_dt / self.steps

    @property
    def particle_steps_per_iteration(self) -> int:
        return self.N * self.K * self.steps

    def scaled(self, **kw) -> "Workload":
        d = dict(self.__dict__)
        d.update(kw)
        return Workload(**d)


# Plain method in FP64: linear OU, eps = 0.1.
OU_SMALL = Workload(
    name="ou_n4096_k8_fp64", kind=MODEL_OU, fast_dim=1, lam=1.0, beta=1.0, eps=0.1,
    N=4096, T=1.0, K=8, dt=1e-3, bins=256, lo=-4.0, hi=4.0, iters=4,
    x0_mean=1.0, x0_std=0.1, y0="normal01", precision="f64")

# Double-well slow variable, FP32 state (the throughput workload).
DOUBLE_WELL = Workload(
    name="double_well_n2^20_k50_s1000_fp32", kind=MODEL_DOUBLE_WELL, fast_dim=1, lam=0.5,
    beta=3.0, eps=1e-2, N=1 << 20, T=5.0, K=50, dt=1e-4, bins=512, lo=-3.0, hi=3.0,
    iters=10, x0_mean=-1.0, x0_std=0.2, y0="x0", precision="f32")

# Adjoint workload: the linear OU family of the first workload at N = 2^20.
ADJOINT = Workload(
    name="adjoint_ou_n2^20_k20_s1000", kind=MODEL_OU, fast_dim=1, lam=1.0, beta=1.0, eps=0.1,
    N=1 << 20, T=2.0, K=20, dt=1e-4, bins=512, lo=-4.0, hi=4.0, iters=0,
    x0_mean=1.0, x0_std=0.1, y0="normal01", precision="f32")

# Large fast space: 16-dim fast OU, coupling lambda * mean(y).
LARGE_FAST = Workload(
    name="dw_fast16_n4e6_k100_s1000_fp32", kind=MODEL_DW_MULTI, fast_dim=16, lam=0.5,
    beta=3.0, eps=1e-3, N=4_000_000, T=1.0, K=100, dt=1e-5, bins=1024, lo=-3.0, hi=3.0,
    iters=8, x0_mean=-1.0, x0_std=0.2, y0="x0", precision="f32")


@dataclass(frozen=True)
class BatchedWorkload:
    """64 independent OU problems with uneven eps, lambda and particle counts."""
    problems: tuple
    name: str = "batched64_ou_k32_fp32"


def batched_problems(n_problems: int = 64, seed: int = 0, K: int = 32, T: float = 2.0,
                     bins: int = 256, n_min: float = 1e4, n_max: float = 1e6,
                     eps_min: float = 1e-3, eps_max: float = 1e-1) -> BatchedWorkload:
    rng = np.random.default_rng(np.random.PCG64(seed + 1000))
    eps = np.exp(rng.uniform(np.log(eps_min), np.log(eps_max), n_problems))
    lam = rng.uniform(0.0, 1.0, n_problems)
    N = np.rint(np.exp(rng.uniform(np.log(n_min), np.log(n_max), n_problems))).astype(int)
    probs = tuple(
        Workload(name=f"batch{i}", kind=MODEL_OU, fast_dim=1, lam=float(lam[i]), beta=1.0,
                 eps=float(eps[i]), N=int(N[i]), T=T, K=K, dt=float(eps[i]) / 50.0, bins=bins,
                 lo=-4.0, hi=4.0, iters=4, x0_mean=1.0, x0_std=0.1, y0="normal01",
                 precision="f32", seed=seed)
        for i in range(n_problems))
    return BatchedWorkload(problems=probs)


def _lognormal_params(mean: float, sd: float):
    """(mu, sigma) of the lognormal with the given mean and standard deviation."""
    s2 = math.log1p((sd / mean) ** 2)
    return math.log(mean) - 0.5 * s2, math.sqrt(s2)


def _draw_slow(rng, w: Workload) -> np.ndarray:
    if w.x0_dist == "lognormal":
        mu, sig = _lognormal_params(w.x0_mean, w.x0_std)
        return rng.lognormal(mu, sig, w.N)
    return rng.normal(w.x0_mean, w.x0_std, w.N)


def initial_slow(w: Workload, seed: int | None = None) -> np.ndarray:
    """X0 [N] alone (the first draws of the stream of `initial_ensemble`);
    for workloads with Y0 = X0 the fast start is its broadcast."""
    rng = np.random.default_rng(np.random.PCG64(w.seed if seed is None else seed))
    return _draw_slow(rng, w)


def initial_ensemble(w: Workload, seed: int | None = None):
    """X0 [N] and Y0 [d][N] in float64, from a PCG64 stream keyed by `seed`."""
    rng = np.random.default_rng(np.random.PCG64(w.seed if seed is None else seed))
    x0 = _draw_slow(rng, w)
    if w.y0 == "normal01":
        y0 = rng.normal(0.0, 1.0, (w.fast_dim, w.N))
    elif w.y0 == "lognormal":
        mu, sig = _lognormal_params(w.x0_mean, w.x0_std)
        y0 = rng.lognormal(mu, sig, (w.fast_dim, w.N))
    else:
        y0 = np.repeat(x0[None, :], w.fast_dim, axis=0)
    return x0, y0


# The chemically reacting system of Section 2.1.2 with the defaults of
# Table 1 (Section 6): P = 1e5 particles, tau_x = 25, eps = 2.5e-2, 20 slices
# of 2 (T = 40), fine step 1e-3, 600 cells on [0, 600], 20 iterations;
# X0 and Y0 independent lognormal with mean 100 and standard deviation 20.
# Rates k0..k5 = 60, 1, 4.8e-3, k3, 0.833, 1: the printed k3 = 0.666e-6
# leaves the fast variable one equilibrium far outside the grid, so the
# workload takes k3 = 0.666e-5, which makes it bistable (wells near 105 and
# 410) as the paper describes it.
CHEM_RATES = (60.0, 1.0, 4.8e-3, 0.666e-5, 0.833, 1.0)
CHEM_RATES_PRINTED = (60.0, 1.0, 4.8e-3, 0.666e-6, 0.833, 1.0)
CHEM = Workload(
    name="chem_n1e5_k20_s2000_fp32", kind=MODEL_CHEM, fast_dim=1, lam=0.0, beta=1.0, eps=2.5e-2,
    N=100_000, T=40.0, K=20, dt=1e-3, bins=600, lo=0.0, hi=600.0, iters=20, x0_mean=100.0,
    x0_std=20.0, y0="lognormal", precision="f32", tau_x=25.0, rates=CHEM_RATES, x0_dist="lognormal")

WORKLOADS = {w.name: w for w in (OU_SMALL, DOUBLE_WELL, ADJOINT, LARGE_FAST, CHEM)}
