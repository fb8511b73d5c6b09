"""Convergence studies of Section 6 (varying the time-scale separation;
scaling with the number of intervals) over the C ABI.

For one problem, a reference is the serial fine solution with `ref_factor`
times the particles (the paper uses ten), whose first N particles are the
parareal ensemble's (same initial states, same random numbers); the error of
parareal iterate k is measured at every slice against the reference's
restriction, as the L2 distance of the piecewise-constant densities
(``pr_l2_density``, the paper's histogram error) and as W1 (``pr_w1``).  The
harness launches the library's kernels only; the per-iteration errors stay
on the device until the run ends.
"""
from __future__ import annotations

import torch

from . import _lib as L
from .parareal import PararealSolver


class ConvergenceStudy:
    def __init__(self, model: L.Model, grid: L.Grid, K: int, steps: int, dt: float, x0, y0, x0_ref, y0_ref,
                 seed: int = 0, precision: int = L.PR_F32, device: str = "cuda", chunk: int = 0):
        """x0 [N], y0 [d][N]: the parareal ensemble; x0_ref [M], y0_ref [d][M]
        (M >= N, its first N columns equal to x0, y0): the reference's."""
        self.model, self.grid, self.K, self.steps, self.dt = model, grid, K, steps, dt
        self.seed, self.precision, self.chunk = seed, precision, chunk
        self.device = torch.device(device)
        dty = torch.float32 if precision == L.PR_F32 else torch.float64
        self.x0 = torch.as_tensor(x0, dtype=dty).to(self.device).reshape(-1)
        self.y0 = torch.as_tensor(y0, dtype=dty).to(self.device).reshape(model.fast_dim, -1)
        xr = torch.as_tensor(x0_ref, dtype=dty).to(self.device).reshape(-1)
        yr = torch.as_tensor(y0_ref, dtype=dty).to(self.device).reshape(model.fast_dim, -1)
        self.N, self.M = self.x0.numel(), xr.numel()
        if self.M < self.N:
            raise ValueError("the reference needs at least as many particles as the parareal ensemble")
        self.ref = self._reference(xr, yr)

    def _reference(self, x, y) -> torch.Tensor:
        """CDFs [K+1][bins+1] of the serial fine solution from (x, y)."""
        M, K, g = self.M, self.K, self.grid
        x = x.clone().reshape(1, M)
        y = y.clone().reshape(1, self.model.fast_dim, M)
        counts = torch.empty(1, g.bins, dtype=torch.int32, device=self.device)
        cdf = torch.empty(K + 1, g.bins + 1, dtype=torch.float64, device=self.device)
        L.pr_restrict(self.precision, x, M, 1, g, counts, cdf[0:1])
        for n in range(K):
            L.pr_fine_propagate(self.model, self.precision, L.Rng(self.seed), x, y, False, x, y, M, n, 1,
                                self.steps, self.dt, g, None, None, None, None, counts, cdf[n + 1:n + 2])
        return cdf

    def run(self, iters: int, iterator: int = L.PR_ITER_QUANTILE, matching: str = "quantile",
            keep_states: bool = False) -> dict:
        """Iterations 0..iters: per iteration and slice, the L2 and W1 errors
        against the reference ([iters+1][K+1] each, on the host at the end);
        with keep_states, the macroscopic states [iters+1][K+1][bins+1] too."""
        K, g = self.K, self.grid
        sv = PararealSolver(self.model, g, self.N, K, self.steps, self.dt, precision=self.precision,
                            rng=L.Rng(self.seed), iterator=iterator, device=str(self.device), chunk=self.chunk,
                            matching=matching)
        sv.set_initial(self.x0, self.y0)
        l2 = torch.empty(iters + 1, K + 1, dtype=torch.float64, device=self.device)
        w1 = torch.empty_like(l2)
        states = [] if keep_states else None
        for k in range(iters + 1):
            if k:
                sv.iterate()
            rho = sv.rho
            L.pr_l2_density(g, K + 1, rho, self.ref, l2[k])
            L.pr_w1(g, K + 1, rho, self.ref, w1[k])
            if keep_states:
                states.append(rho.clone())
        status = int(sv.status.item())
        sv.close()
        out = {"l2": l2.cpu(), "w1": w1.cpu(), "status": status}
        if keep_states:
            out["states"] = torch.stack(states).cpu()
        return out
