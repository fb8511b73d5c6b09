"""Micro-macro parareal driver (Sections 3.2.3-3.2.4) over the C ABI.

The driver owns the device buffers (torch tensors: memory only) and sequences
the library's kernels; it performs no arithmetic of its own.  One parareal
iteration k -> k+1 is:

1. fine propagation of all slices (``pr_fine_propagate``), slice 0 from X_0
   and slice n >= 1 from the matched state X_k^n = M(rho_k^n, Xbar_{k-1}^n),
   the matching fused into the kernel's prologue and the restrictions
   R X_k^n and R Xbar_k^{n+1} into it;
2. the coarse propagator on every start state, rho_c* = C(R X_k^n)
   (``pr_coarse_fp``);
3. the serial update rho_{k+1}^{n+1} = J(C(rho_{k+1}^n), rho_f*, rho_c*)
   (``pr_parareal_update``).

Iteration 0 is the serial coarse sweep from R X_0 (``PR_ITER_NONE``); its
matching against X_0 happens in the prologue of the first fine launch.

Pipelined mode (``chunk > 0``): the slices are cut into chunks; the fine
launches of chunk c run on two alternating streams and the coarse step and
serial sweep of chunk c on a high-priority stream as soon as that chunk's
fine results exist.  Slice n of iteration k+1 only needs the sweep of
iteration k up to slice n, so the serial sweep hides behind the fine work.
The macroscopic states are double-buffered; every cross-stream hazard is
ordered by an event (fine(k+1, c) waits for the sweep of chunk c and for
fine(k, c+1), which reads the slice fine(k+1, c) overwrites).  Results are
bit for bit those of the sequential mode.  ``join()`` (called by every
accessor) makes the caller's stream wait for the outstanding work.

Matching (``matching``): "quantile" (Section 5.1, fused into the fine
launch), "resample" / "resample_det" (Section 5.2: reweighting of the prior
ensemble to the target histogram, stratified resampling with uniform or
u~ = 1/2 points, gather of the start states, then the fine launch in place),
"reweight" (Section 5.2 without resampling: positions kept, weights carried
by the ensembles, every restriction weighted).

Graph mode (``graph=True``): iterations k >= 1 are replayed as one CUDA graph
each (two graphs, one per binding of the double buffers), which removes the
per-launch host cost that dominates small workloads.  In pipelined graph mode
the chunks still overlap within an iteration; consecutive iterations are
ordered by the graph launches themselves.

Skipping converged slices (``skip_converged=True``, exactness property of
Section 3.2.4): iterate k is the serial fine solution on slices n <= k, so
iteration k >= 1 need not propagate slices n < k again -- their start states
are those of iteration k - 1, and so are their fine results.  Iteration k
launches the fine work of slices k..K-1 only (K(K-1)/2 slice propagations
fewer over K iterations) and takes slice k - 1's results, the last ones not
yet in both halves of the double buffers, from the previous iteration's
half.  The results are those of the full iteration bit for bit wherever the
iterator meets J(a, b, a) = b bit for bit (the quantile iterator); with the
other iterators the skipped slices keep the serial fine result exactly,
where recomputing them would reproduce it within rounding.  Not combined
with graph mode (the work changes from one iteration to the next).
"""
from __future__ import annotations

import torch

from . import _lib as L


MATCHINGS = ("quantile", "resample", "resample_det", "reweight")


class PararealSolver:
    def __init__(self, model: L.Model, grid: L.Grid, n: int, K: int, steps: int, dt: float,
                 precision: int = L.PR_F32, rng: L.Rng = L.Rng(), iterator: int = L.PR_ITER_QUANTILE,
                 qmode: int = L.PR_QMODE_TWO_SIDED, device: str = "cuda", stream=None, chunk: int = 0,
                 graph: bool = False, matching: str = "quantile", skip_converged: bool = False):
        if matching not in MATCHINGS:
            raise ValueError(f"matching must be one of {MATCHINGS}")
        if skip_converged and graph:
            raise ValueError("skip_converged changes the work of every iteration: it cannot be graph-replayed")
        self.matching = matching
        self.skip_converged = bool(skip_converged)
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
        self._rho = z(K + 1, I + 1, dtype=f64)       # rho_k (read by the fine launches)
        self._rho_next = z(K + 1, I + 1, dtype=f64)  # rho_{k+1} (written by the sweep)
        self.prior0 = z(K, I + 1, dtype=f64)
        self.f_star = z(K, I + 1, dtype=f64)        # R Xbar_k^{n+1} of this iteration
        self.f_star_prev = z(K, I + 1, dtype=f64)   # ... of the previous iteration
        self.start = z(K, I + 1, dtype=f64)
        self.c_star = z(K, I + 1, dtype=f64)
        self.counts_s = z(K, I, dtype=torch.int32)
        self.counts_e = z(K, I, dtype=torch.int32)
        self.chunk = int(chunk) if chunk and chunk < K else 0
        nch = (K + self.chunk - 1) // self.chunk if self.chunk else 1
        # Section 5.2 matchings: weights of the start states (and of the
        # priors, which carry them in "reweight" mode), per-stream scratch
        self._ws = {}
        if matching != "quantile":
            self.w = z(K, n, dtype=f64)
            self.w_uni = torch.full((n,), 1.0 / n, dtype=f64, device=self.device)
            if matching == "reweight":
                self.w_prev = z(K, n, dtype=f64)
                self.w[0].copy_(self.w_uni)
                self.w_prev[0].copy_(self.w_uni)
        self._status = z(nch, dtype=torch.int32)
        self.coarse = L.pr_coarse_create(model, grid, steps * dt, stream=self._s())
        self.k = 0
        # when a list, (start, end) CUDA events around the main fine launch of
        # every sequential iteration are appended to it
        self.fine_events = None
        # kernels of libpr.so enqueued by iterate() so far (the fine call with
        # both fused restrictions is 3: the fine kernel and two counts->CDF)
        self.launches = 0
        if self.chunk:
            self._sf = [torch.cuda.Stream(self.device), torch.cuda.Stream(self.device)]
            self._su = torch.cuda.Stream(self.device, priority=-1)
            self._ev_fine = [None] * nch     # fine(k, c) of the latest enqueued iteration
            self._ev_upd = [None] * nch      # sweep(k, c) of the latest enqueued iteration
        self._ev_zero = []                   # zeroth sweep, chunk by chunk (pipelined mode)
        self._pending = False
        self.graph = bool(graph)
        self._swaps = 0                  # iterations since construction (buffer binding parity)
        self._graphs = [None, None]
        self._graph_launches = [0, 0]

    # -- plumbing ----------------------------------------------------------------
    def _s(self):
        return self.stream if self.stream is not None else torch.cuda.current_stream(self.device)

    def close(self):
        if getattr(self, "coarse", None):
            self.join()
            L.pr_coarse_destroy(self.coarse)
            self.coarse = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def join(self):
        """Make the caller's stream wait for every enqueued kernel of the solver."""
        if self.chunk and self._pending:
            s = self._s()
            for ev in self._ev_upd + self._ev_fine + self._ev_zero:
                if ev is not None:
                    s.wait_event(ev)
            self._pending = False

    @property
    def rho(self) -> torch.Tensor:
        """rho_k^n, n = 0..K, as CDFs at the edges (after the latest iteration)."""
        self.join()
        return self._rho

    @property
    def status(self) -> torch.Tensor:
        self.join()
        return self._status.max().reshape(1)

    # -- setup and iteration 0 -------------------------------------------------
    def set_initial(self, x0: torch.Tensor, y0: torch.Tensor):
        self.join()
        s = self._s()
        self.x0.copy_(x0.reshape(self.n))
        self.y0.copy_(y0.reshape(self.model.fast_dim, self.n))
        self._initial_states(s)

    def set_initial_host(self, x0: torch.Tensor, y0: torch.Tensor):
        """set_initial() from X_0 and Y_0 in host memory (page-locked for an
        asynchronous copy), copied into the solver by the library."""
        self.join()
        s = self._s()
        L.pr_copy_to_device(self.x0, x0.reshape(self.n), stream=s)
        L.pr_copy_to_device(self.y0, y0.reshape(self.model.fast_dim, self.n), stream=s)
        self._initial_states(s)

    def rho_to_host(self, out: torch.Tensor):
        """Copy rho_k^n, n = 0..K, into the host tensor `out` [K+1][bins+1]
        (asynchronous on the solver's stream when `out` is page-locked)."""
        L.pr_copy_to_host(out, self.rho, stream=self._s())

    def _initial_states(self, s):
        """R X_0 and the zeroth iteration (serial coarse sweep), on stream s."""
        if self.matching == "reweight":   # every restriction carries the weights (here 1/N)
            L.pr_restrict_weighted(self.precision, self.x0, False, self.w_uni, self.n, 1, self.grid, self.cdf0,
                                   self._scratch("wr", 0, L.pr_restrict_weighted_workspace(1, self.grid.bins)),
                                   stream=s)
        else:
            L.pr_restrict(self.precision, self.x0, self.n, 1, self.grid, self.counts0, self.cdf0, stream=s)
        self.prior0.copy_(self.cdf0.expand(self.K, -1))
        self.k = 0
        if self.chunk:
            # the zeroth sweep chunk by chunk on the sweep stream: the first
            # iteration's fine chunk c waits only for the sweep up to its
            # slices, so the rest of the sweep runs beside the fine work
            K, C = self.K, self.chunk
            ready = torch.cuda.Event()
            ready.record(s)
            self._su.wait_event(ready)
            self._ev_zero = []
            for c in range(len(self._ev_upd)):
                a, b = c * C, min(K, (c + 1) * C)
                state = self.cdf0 if a == 0 else self._rho[a]
                L.pr_parareal_update(self.coarse, L.PR_ITER_NONE, self.qmode, b - a, state, None, None,
                                     self._rho[a:b + 1], self._status[c], stream=self._su)
                ev = torch.cuda.Event()
                ev.record(self._su)
                self._ev_zero.append(ev)
            self._pending = True
        else:
            L.pr_parareal_update(self.coarse, L.PR_ITER_NONE, self.qmode, self.K, self.cdf0, None, None,
                                 self._rho, self._status[0], stream=s)
        if self.chunk:
            self._ev_fine = [None] * len(self._ev_fine)
            self._ev_upd = [None] * len(self._ev_upd)

    # -- one generic iteration ---------------------------------------------------
    def _scratch(self, kind: str, role: int, nbytes: int) -> torch.Tensor:
        """Device scratch of a library call, one per kind and per stream role
        (0: sequential; chunk parity in the pipelined schedule), kept."""
        t = self._ws.get((kind, role))
        if t is None or t.numel() < nbytes:
            t = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=self.device)
            self._ws[(kind, role)] = t
        return t

    def _fine(self, a: int, b: int, first: bool, stream, role: int = 0):
        """Matching and fine launches for slices [a, b) of this iteration on `stream`."""
        n, grid, prec = self.n, self.grid, self.precision
        weighted = self.matching == "reweight"
        span = self.chunk or self.K
        if a == 0:
            if weighted:   # X_0 with its uniform weights; restrictions with the weights
                wr = self._scratch("wr", role, L.pr_restrict_weighted_workspace(span, grid.bins))
                L.pr_restrict_weighted(prec, self.x0, False, self.w_uni, n, 1, grid, self.start[0], wr, stream=stream)
                L.pr_fine_propagate(self.model, prec, self.rng, self.x0, self.y0, True, self.xb[0], self.yb[0], n,
                                    0, 1, self.steps, self.dt, stream=stream)
                L.pr_restrict_weighted(prec, self.xb[0], False, self.w_uni, n, 1, grid, self.f_star[0], wr,
                                       stream=stream)
                self.launches += 5
            else:
                L.pr_fine_propagate(self.model, prec, self.rng, self.x0, self.y0, True,
                                    self.xb[0], self.yb[0], n, 0, 1, self.steps, self.dt, grid,
                                    None, None, self.counts_s[0], self.start[0], self.counts_e[0],
                                    self.f_star[0], stream=stream)
                self.launches += 3
            a = 1
        if b <= a:
            return
        if first:   # X_0^n = M(rho_0^n, X_0)
            src_x, src_y, bcast, prior = self.x0, self.y0, True, self.prior0[a - 1:b - 1]
            w_prior = None
        else:       # X_k^n = M(rho_k^n, Xbar_{k-1}^n)
            src_x, src_y, bcast = self.xa[a - 1:b - 1], self.ya[a - 1:b - 1], False
            prior = self.f_star_prev[a - 1:b - 1]
            w_prior = self.w_prev[a - 1:b - 1] if weighted else None
        ev = None
        if self.fine_events is not None and not self.chunk:
            ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            ev[0].record(stream)
        S = b - a
        if self.matching == "quantile":
            # Section 5.1: the matching is fused into the fine launch's prologue
            L.pr_fine_propagate(self.model, prec, self.rng, src_x, src_y, bcast,
                                self.xb[a:b], self.yb[a:b], n, a, S, self.steps, self.dt, grid,
                                prior, self._rho[a:b], self.counts_s[a:b], self.start[a:b], self.counts_e[a:b],
                                self.f_star[a:b], stream=stream)
            self.launches += 3
        elif weighted:
            # Section 5.2, reweighting only: positions unchanged, weights carried
            wr = self._scratch("wr", role, L.pr_restrict_weighted_workspace(span, grid.bins))
            L.pr_reweight(prec, src_x, bcast, w_prior, n, S, grid, prior, self._rho[a:b], self.w[a:b],
                          stream=stream)
            L.pr_restrict_weighted(prec, src_x, bcast, self.w[a:b], n, S, grid, self.start[a:b], wr, stream=stream)
            L.pr_fine_propagate(self.model, prec, self.rng, src_x, src_y, bcast, self.xb[a:b], self.yb[a:b], n, a,
                                S, self.steps, self.dt, stream=stream)
            L.pr_restrict_weighted(prec, self.xb[a:b], False, self.w[a:b], n, S, grid, self.f_star[a:b], wr,
                                   stream=stream)
            self.launches += 7
        else:
            # Section 5.2 with resampling: reweight, resample into the start
            # states (gather of x and y), then the fine launch in place
            mode = L.PR_RESAMPLE_STRATIFIED if self.matching == "resample" else L.PR_RESAMPLE_DETERMINISTIC
            rs = self._scratch("rs", role, L.pr_resample_workspace(n, span))
            L.pr_reweight(prec, src_x, bcast, None, n, S, grid, prior, self._rho[a:b], self.w[a:b], stream=stream)
            L.pr_resample(prec, self.model.fast_dim, src_x, src_y, bcast, self.w[a:b], n, S, a, mode, self.rng, None,
                          self.xb[a:b], self.yb[a:b], rs, stream=stream)
            L.pr_fine_propagate(self.model, prec, self.rng, self.xb[a:b], self.yb[a:b], False, self.xb[a:b],
                                self.yb[a:b], n, a, S, self.steps, self.dt, grid, None, None, self.counts_s[a:b],
                                self.start[a:b], self.counts_e[a:b], self.f_star[a:b], stream=stream)
            self.launches += 8
        if ev is not None:
            ev[1].record(stream)
            self.fine_events.append(ev)

    def iterate(self):
        if self.graph and self.k >= 1:
            self._replay()
        else:
            self._enqueue(self._s(), self.k == 0, in_graph=False)
        self._advance()

    def _advance(self):
        # the fine results become the priors of the next matching
        self.xa, self.xb = self.xb, self.xa
        self.ya, self.yb = self.yb, self.ya
        self.f_star, self.f_star_prev = self.f_star_prev, self.f_star
        self._rho, self._rho_next = self._rho_next, self._rho
        if self.matching == "reweight":
            self.w, self.w_prev = self.w_prev, self.w
        self._swaps += 1
        self.k += 1

    def _carry(self, stream):
        """Slice k - 1 of this iteration's outputs, taken from the previous
        iteration's (the start state of slice k - 1 is exact in both)."""
        m = self.k - 1
        with torch.cuda.stream(stream):
            self.xb[m].copy_(self.xa[m])
            self.yb[m].copy_(self.ya[m])
            self.f_star[m].copy_(self.f_star_prev[m])
            if self.matching == "reweight":
                self.w[m].copy_(self.w_prev[m])

    def _enqueue(self, s, first: bool, in_graph: bool):
        """Enqueue one iteration behind the work already on stream `s`."""
        K = self.K
        # with skip_converged, slices n < k keep the previous iteration's results
        lo = self.k if self.skip_converged else 0
        carry = self.skip_converged and 1 <= self.k <= K
        if not self.chunk:
            if carry:
                self._carry(s)
            self._fine(lo, K, first, s)
            L.pr_coarse_fp(self.coarse, self.start, self.c_star, K, stream=s)
            L.pr_parareal_update(self.coarse, self.iterator, self.qmode, K, self.cdf0, self.f_star, self.c_star,
                                 self._rho_next, self._status[0], stream=s)
            self.launches += 2
            return
        C = self.chunk
        nch = len(self._ev_upd)
        fork = torch.cuda.Event()
        fork.record(s)
        for st in (*self._sf, self._su):
            st.wait_event(fork)
        new_fine, new_upd = [None] * nch, [None] * nch
        for c in range(nch):
            a, b = c * C, min(K, (c + 1) * C)
            sf = self._sf[c % 2]
            if not in_graph:   # a graph launch starts after the previous iteration has ended
                for ev in (self._ev_upd[c], self._ev_fine[c + 1] if c + 1 < nch else None,
                           self._ev_zero[c] if first and self._ev_zero else None):
                    if ev is not None:
                        sf.wait_event(ev)
            if carry and a <= self.k - 1 < b:
                self._carry(sf)
            self._fine(max(a, lo), b, first, sf, role=c % 2)
            ef = torch.cuda.Event()
            ef.record(sf)
            new_fine[c] = ef
            su = self._su
            su.wait_event(ef)
            L.pr_coarse_fp(self.coarse, self.start[a:b], self.c_star[a:b], b - a, stream=su)
            state = self.cdf0 if a == 0 else self._rho_next[a]
            L.pr_parareal_update(self.coarse, self.iterator, self.qmode, b - a, state, self.f_star[a:b],
                                 self.c_star[a:b], self._rho_next[a:b + 1], self._status[c], stream=su)
            self.launches += 2
            eu = torch.cuda.Event()
            eu.record(su)
            new_upd[c] = eu
        if in_graph:       # every forked stream rejoins the capturing stream
            for ev in new_fine + new_upd:
                s.wait_event(ev)
            self._ev_fine, self._ev_upd = [None] * nch, [None] * nch
        else:
            self._ev_fine, self._ev_upd = new_fine, new_upd
            self._pending = True

    def _replay(self):
        """Iterations k >= 1 as one CUDA graph each.  The buffers alternate
        between two bindings, so there is one graph per binding, captured on
        first use (capture enqueues nothing; the replay does the work)."""
        p = self._swaps % 2
        s = self._s()
        if self._graphs[p] is None:
            self.join()
            cs = torch.cuda.Stream(self.device)
            cs.wait_stream(s)
            g = torch.cuda.CUDAGraph()
            n0, events = self.launches, self.fine_events
            self.fine_events = None      # no timing events inside a graph
            try:
                with torch.cuda.graph(g, stream=cs):
                    self._enqueue(cs, False, in_graph=True)
            finally:
                self.fine_events = events
            self._graph_launches[p] = self.launches - n0
            self.launches = n0
            s.wait_stream(cs)
            self._graphs[p] = g
        with torch.cuda.stream(s):
            self._graphs[p].replay()
        self.launches += self._graph_launches[p]

    # -- the serial fine solution with the same random numbers -----------------
    def serial_reference(self):
        """x[K+1][n], y[K+1][d][n] and their restrictions rho[K+1][I+1]."""
        self.join()
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
        if self.matching == "reweight":
            wu = self.w_uni.expand(K + 1, n).contiguous()
            L.pr_restrict_weighted(self.precision, xs, False, wu, n, K + 1, self.grid, rho,
                                   self._scratch("wr_ref", 0, L.pr_restrict_weighted_workspace(K + 1, self.grid.bins)),
                                   stream=s)
        else:
            L.pr_restrict(self.precision, xs, n, K + 1, self.grid, counts, rho, stream=s)
        return xs, ys, rho

    def w1_to(self, rho_ref: torch.Tensor) -> torch.Tensor:
        out = torch.empty(self.K + 1, dtype=torch.float64, device=self.device)
        L.pr_w1(self.grid, self.K + 1, self.rho, rho_ref, out, stream=self._s())
        return out

    def increment(self) -> torch.Tensor:
        """W1(rho_k^n, rho_{k-1}^n) for n = 0..K on the device: the change of
        the macroscopic states in the latest iteration (k >= 1).  It needs no
        serial solution, and by the exactness theorem it is 0 from iteration
        K + 1 on."""
        if self.k < 1:
            raise RuntimeError("increment() needs at least one iteration after set_initial()")
        out = torch.empty(self.K + 1, dtype=torch.float64, device=self.device)
        L.pr_w1(self.grid, self.K + 1, self.rho, self._rho_next, out, stream=self._s())
        return out

    def run(self, tol: float, max_iters: int | None = None) -> int:
        """Iterate until max_n increment() <= tol, or until iteration
        max_iters (default K + 1, where the increment is 0); returns the
        number of iterations taken.  One host synchronisation per iteration."""
        limit = self.K + 1 if max_iters is None else max_iters
        while self.k < limit:
            self.iterate()
            if float(self.increment().max().item()) <= tol:
                break
        return self.k

    def state(self):
        """The fine end states Xbar_{k-1}^{n}, n = 1..K, and rho_k (the iterate
        X_k^n is their matching against rho_k)."""
        self.join()
        return self.xa, self.ya, self._rho

    def moments(self, max_order: int = 2, component: int = -1) -> torch.Tensor:
        """Monte Carlo estimates (Eq. MCestimator) of v^q, q = 1..max_order, over
        the fine end states Xbar_{k-1}^{n}, n = 1..K: [K][max_order], v the
        slow variable (component -1) or fast component `component`, with the
        weights those states carry (matching "reweight") or 1/N."""
        self.join()
        K, n, d = self.K, self.n, self.model.fast_dim
        if component >= 0:
            if component >= d:
                raise ValueError("component out of range")
            v, stride = self.ya.reshape(-1)[component * n:], d * n
        else:
            v, stride = self.xa, n
        w = self.w_prev if self.matching == "reweight" else None
        out = torch.empty(K, max_order, dtype=torch.float64, device=self.device)
        ws = self._scratch("mom", 0, L.pr_moments_workspace(n, K, max_order))
        L.pr_moments(self.precision, v, stride, w, n, K, max_order, out, ws, stream=self._s())
        return out

    def weights(self):
        """Weights carried by the fine end states (matching "reweight"; slice 0
        and the other matchings: uniform 1/N)."""
        self.join()
        if self.matching == "reweight":
            return self.w_prev
        return None
