"""Micro-macro parareal driver (Sections 3.2.3-3.2.4) over the C ABI.

The driver owns the device buffers (torch tensors: memory only) and sequences
the library's kernels; it performs no arithmetic of its own.  One parareal
iteration k -> k+1 is, in order:

1. fine propagation of all slices at once (``pr_fine_propagate``), slice 0
   from X_0 and slice n >= 1 from the matched state
   X_k^n = M(rho_k^n, Xbar_{k-1}^n), with the matching fused into the kernel's
   prologue and the restrictions R X_k^n and R Xbar_k^{n+1} into it;
2. the coarse propagator on every start state, rho_c* = C(R X_k^n)
   (``pr_coarse_fp``);
3. the serial update rho_{k+1}^{n+1} = J(C(rho_{k+1}^n), rho_f*, rho_c*)
   (``pr_parareal_update``).

Iteration 0 is the serial coarse sweep from R X_0 (``PR_ITER_NONE``); its
matching against X_0 happens in the prologue of the first fine launch.
"""
from __future__ import annotations

import torch

from . import _lib as L


class PararealSolver:
    def __init__(self, model: L.Model, grid: L.Grid, n: int, K: int, steps: int, dt: float,
                 precision: int = L.PR_F32, rng: L.Rng = L.Rng(), iterator: int = L.PR_ITER_QUANTILE,
                 qmode: int = L.PR_QMODE_TWO_SIDED, device: str = "cuda", stream=None):
        self.model, self.grid, self.n, self.K, self.steps, self.dt = model, grid, n, K, steps, dt
        self.precision, self.rng, self.iterator, self.qmode = precision, rng, iterator, qmode
        self.device = torch.device(device)
        self.stream = stream
        dt_ = torch.float32 if precision == L.PR_F32 else torch.float64
        d, I = model.fast_dim, grid.bins
        z = lambda *s, dtype=dt_: torch.zeros(*s, dtype=dtype, device=self.device)
        self.x0, self.y0 = z(n), z(d, n)
        self.xa, self.ya = z(K, n), z(K, d, n)    # Xbar of the previous iteration
        self.xb, self.yb = z(K, n), z(K, d, n)    # start states -> Xbar of this iteration
        f64 = torch.float64
        self.cdf0 = z(I + 1, dtype=f64)
        self.counts0 = z(I, dtype=torch.int32)
        self.rho = z(K + 1, I + 1, dtype=f64)
        self.prior0 = z(K, I + 1, dtype=f64)
        self.f_star = z(K, I + 1, dtype=f64)        # R Xbar_k^{n+1} of this iteration
        self.f_star_prev = z(K, I + 1, dtype=f64)   # ... of the previous iteration
        self.start = z(K, I + 1, dtype=f64)
        self.c_star = z(K, I + 1, dtype=f64)
        self.counts_s = z(K, I, dtype=torch.int32)
        self.counts_e = z(K, I, dtype=torch.int32)
        self.status = z(1, dtype=torch.int32)
        self.coarse = L.pr_coarse_create(model, grid, steps * dt, stream=self._s())
        self.k = 0
        # when a list, (start, end) CUDA events around the main fine launch of
        # every iteration are appended to it
        self.fine_events = None

    def _s(self):
        return self.stream if self.stream is not None else torch.cuda.current_stream(self.device)

    def close(self):
        if getattr(self, "coarse", None):
            L.pr_coarse_destroy(self.coarse)
            self.coarse = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- setup and iteration 0 -------------------------------------------------
    def set_initial(self, x0: torch.Tensor, y0: torch.Tensor):
        self.x0.copy_(x0.reshape(self.n))
        self.y0.copy_(y0.reshape(self.model.fast_dim, self.n))
        s = self._s()
        L.pr_restrict(self.precision, self.x0, self.n, 1, self.grid, self.counts0, self.cdf0, stream=s)
        self.prior0.copy_(self.cdf0.expand(self.K, -1))
        L.pr_parareal_update(self.coarse, L.PR_ITER_NONE, self.qmode, self.K, self.cdf0, None, None,
                             self.rho, self.status, stream=s)
        self.k = 0

    # -- one generic iteration ---------------------------------------------------
    def iterate(self):
        K, n, s = self.K, self.n, self._s()
        first = self.k == 0
        # slice 0 starts from X_0 (no matching)
        L.pr_fine_propagate(self.model, self.precision, self.rng, self.x0, self.y0, True,
                            self.xb[0], self.yb[0], n, 0, 1, self.steps, self.dt, self.grid,
                            None, None, self.counts_s[0], self.start[0], self.counts_e[0],
                            self.f_star[0], stream=s)
        if K > 1:
            if first:   # X_0^n = M(rho_0^n, X_0)
                src_x, src_y, bcast, prior = self.x0, self.y0, True, self.prior0[: K - 1]
            else:       # X_k^n = M(rho_k^n, Xbar_{k-1}^n)
                src_x, src_y, bcast, prior = self.xa[: K - 1], self.ya[: K - 1], False, self.f_star_prev[: K - 1]
            ev = None
            if self.fine_events is not None:
                ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                ev[0].record(s)
            L.pr_fine_propagate(self.model, self.precision, self.rng, src_x, src_y, bcast,
                                self.xb[1:], self.yb[1:], n, 1, K - 1, self.steps, self.dt, self.grid,
                                prior, self.rho[1:K], self.counts_s[1:], self.start[1:], self.counts_e[1:],
                                self.f_star[1:], stream=s)
            if ev is not None:
                ev[1].record(s)
                self.fine_events.append(ev)
        L.pr_coarse_fp(self.coarse, self.start, self.c_star, K, stream=s)
        L.pr_parareal_update(self.coarse, self.iterator, self.qmode, K, self.cdf0, self.f_star, self.c_star,
                             self.rho, self.status, stream=s)
        # the fine results become the priors of the next matching
        self.xa, self.xb = self.xb, self.xa
        self.ya, self.yb = self.yb, self.ya
        self.f_star, self.f_star_prev = self.f_star_prev, self.f_star
        self.k += 1

    # -- the serial fine solution with the same random numbers -----------------
    def serial_reference(self):
        """x[K+1][n], y[K+1][d][n] and their restrictions rho[K+1][I+1]."""
        K, n, s = self.K, self.n, self._s()
        d = self.model.fast_dim
        xs = torch.empty(K + 1, n, dtype=self.x0.dtype, device=self.device)
        ys = torch.empty(K + 1, d, n, dtype=self.x0.dtype, device=self.device)
        xs[0].copy_(self.x0)
        ys[0].copy_(self.y0)
        for m in range(K):
            L.pr_fine_propagate(self.model, self.precision, self.rng, xs[m], ys[m], False, xs[m + 1], ys[m + 1],
                                n, m, 1, self.steps, self.dt, stream=s)
        counts = torch.empty(K + 1, self.grid.bins, dtype=torch.int32, device=self.device)
        rho = torch.empty(K + 1, self.grid.bins + 1, dtype=torch.float64, device=self.device)
        L.pr_restrict(self.precision, xs, n, K + 1, self.grid, counts, rho, stream=s)
        return xs, ys, rho

    def w1_to(self, rho_ref: torch.Tensor) -> torch.Tensor:
        out = torch.empty(self.K + 1, dtype=torch.float64, device=self.device)
        L.pr_w1(self.grid, self.K + 1, self.rho, rho_ref, out, stream=self._s())
        return out

    def state(self):
        """Current iterate X_k^n for n = 1..K is held implicitly (Xbar + matching);
        this returns the fine end states Xbar_{k-1}^{n} and rho_k."""
        return self.xa, self.ya, self.rho
