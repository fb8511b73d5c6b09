"""Batched serving of many independent micro-macro parareal problems.

``BatchSolver`` wraps a plan of libpr.so (pr_batch_*): the plan owns the
device buffers and runs each parareal iteration of the whole batch as one
persistent fine launch plus three small launches, replayed as a CUDA graph
from the second iteration on.  Tensors here only carry the packed initial
ensembles in and the macroscopic states out.
"""
from __future__ import annotations

import torch

from . import _lib as L


class BatchSolver:
    def __init__(self, problems: list[L.Problem], iterator: int = L.PR_ITER_QUANTILE,
                 qmode: int = L.PR_QMODE_TWO_SIDED, device: str = "cuda", stream=None):
        self.problems = list(problems)
        self.device = torch.device(device)
        self.stream = stream
        self.plan = L.pr_batch_create(self.problems, iterator, qmode, stream=self._s())
        self.offsets = []
        off = 0
        for p in self.problems:
            self.offsets.append(off)
            off += p.n
        self.total_n = off

    def _s(self):
        return self.stream if self.stream is not None else torch.cuda.current_stream(self.device)

    def close(self):
        if getattr(self, "plan", None):
            L.pr_batch_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def particle_steps(self) -> int:
        return L.pr_batch_particle_steps(self.plan)

    def set_initial(self, x0s, y0s):
        """x0s, y0s: per-problem 1-D arrays or tensors (or already packed float32 device tensors)."""
        if torch.is_tensor(x0s) and x0s.dim() == 1 and x0s.numel() == self.total_n:
            x0, y0 = x0s.to(self.device, torch.float32).contiguous(), y0s.to(self.device, torch.float32).contiguous()
        else:
            x0 = torch.cat([torch.as_tensor(v, dtype=torch.float32).reshape(-1) for v in x0s]).to(self.device)
            y0 = torch.cat([torch.as_tensor(v, dtype=torch.float32).reshape(-1) for v in y0s]).to(self.device)
        self._x0, self._y0 = x0, y0
        L.pr_batch_set_initial(self.plan, x0, y0, stream=self._s())

    def iterate(self):
        L.pr_batch_iterate(self.plan, stream=self._s())

    def rho(self, problem: int) -> torch.Tensor:
        p = self.problems[problem]
        out = torch.empty(p.n_slices + 1, p.grid.bins + 1, dtype=torch.float64, device=self.device)
        L.pr_batch_rho(self.plan, problem, out, stream=self._s())
        return out

    def fine_state(self, problem: int):
        p = self.problems[problem]
        x = torch.empty(p.n_slices, p.n, dtype=torch.float32, device=self.device)
        y = torch.empty(p.n_slices, p.n, dtype=torch.float32, device=self.device)
        L.pr_batch_fine_state(self.plan, problem, x, y, stream=self._s())
        return x, y

    def status(self) -> int:
        return L.pr_batch_status(self.plan, stream=self._s())

    def _w1(self, problem: int, a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
        p = self.problems[problem]
        out = torch.empty(p.n_slices + 1, dtype=torch.float64, device=self.device)
        L.pr_w1(p.grid, p.n_slices + 1, a, b, out, stream=self._s())
        return out

    def snapshot(self) -> list[torch.Tensor]:
        """Copies of every problem's macroscopic states rho_k (device)."""
        return [self.rho(i) for i in range(len(self.problems))]

    def increments(self, prev: list[torch.Tensor], cur: list[torch.Tensor] | None = None) -> torch.Tensor:
        """max_n W1(cur^n, prev^n) per problem [n_problems] (device); cur
        defaults to the current states."""
        cur = self.snapshot() if cur is None else cur
        return torch.stack([self._w1(i, cur[i], prev[i]).max() for i in range(len(self.problems))])

    def run(self, tol: float, max_iters: int | None = None) -> tuple[int, torch.Tensor]:
        """Iterate until every problem's increment max_n W1(rho_k^n, rho_{k-1}^n)
        is within `tol` (no serial solution needed; by the exactness theorem it
        is 0 once k exceeds the problem's slice count), or until max_iters
        (default: the largest slice count + 1).  Returns the iterations taken
        and the last increments [n_problems] (device).  One host
        synchronisation per iteration."""
        limit = max(p.n_slices for p in self.problems) + 1 if max_iters is None else max_iters
        prev = self.snapshot()
        inc = torch.full((len(self.problems),), float("inf"), dtype=torch.float64, device=self.device)
        k = 0
        while k < limit:
            self.iterate()
            k += 1
            cur = self.snapshot()
            inc = self.increments(prev, cur)
            if float(inc.max().item()) <= tol:
                break
            prev = cur
        return k, inc

    def tune(self, steps_div: int = 8) -> float:
        return L.pr_batch_tune(self.plan, steps_div, stream=self._s())

    def config(self):
        return L.pr_batch_get_config(self.plan)

    def set_config(self, ppt: int, item_work: float):
        L.pr_batch_set_config(self.plan, ppt, item_work)
