"""Parareal on densities with the discretised Fokker-Planck equation as both
the fine and the coarse propagator (Section 6, linear advection case).

Restriction and matching are the identity here; the iterator is not.  The
fine propagator F = exp(A_fine dT) and the coarse propagator
C = exp(A_coarse dT) are two handles of ``pr_coarse_create`` (typically the
same model with biased parameters for the coarse one, e.g. the potential
x/eps and diffusion 1/beta of ``PR_MODEL_ADVECTION``); one iteration is

    rho_{k+1}^{n+1} = J(C rho_{k+1}^n, F rho_k^n, C rho_k^n),

two ``pr_coarse_fp`` calls over all slices and one ``pr_parareal_update``
(the serial sweep).  Tensors are plumbing; every step runs in libpr.so.
"""
from __future__ import annotations

import torch

from . import _lib as L


class FPParareal:
    def __init__(self, grid: L.Grid, fine: L.Model, coarse: L.Model, K: int, dT: float,
                 iterator: int = L.PR_ITER_QUANTILE, qmode: int = L.PR_QMODE_TWO_SIDED, device: str = "cuda",
                 stream=None):
        self.grid, self.K, self.dT, self.iterator, self.qmode = grid, K, dT, iterator, qmode
        self.device = torch.device(device)
        self.stream = stream
        I = grid.bins
        z = lambda *s: torch.zeros(*s, dtype=torch.float64, device=self.device)
        self.cdf0 = z(I + 1)
        self._rho, self._rho_next = z(K + 1, I + 1), z(K + 1, I + 1)
        self.f_star, self.c_star = z(K, I + 1), z(K, I + 1)
        self._status = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.fine = L.pr_coarse_create(fine, grid, dT, stream=self._s())
        self.coarse = L.pr_coarse_create(coarse, grid, dT, stream=self._s())
        self.k = 0

    def _s(self):
        return self.stream if self.stream is not None else torch.cuda.current_stream(self.device)

    @property
    def rho(self) -> torch.Tensor:
        return self._rho

    @property
    def status(self) -> torch.Tensor:
        return self._status

    def set_initial(self, cdf0: torch.Tensor):
        """rho^0 = cdf0 ([bins+1]); iteration 0 is the coarse sweep."""
        s = self._s()
        self.cdf0.copy_(cdf0.reshape(-1))
        L.pr_parareal_update(self.coarse, L.PR_ITER_NONE, self.qmode, self.K, self.cdf0, None, None, self._rho,
                             self._status, stream=s)
        self.k = 0

    def iterate(self):
        s, K = self._s(), self.K
        L.pr_coarse_fp(self.fine, self._rho[:K], self.f_star, K, stream=s)
        L.pr_coarse_fp(self.coarse, self._rho[:K], self.c_star, K, stream=s)
        L.pr_parareal_update(self.coarse, self.iterator, self.qmode, K, self.cdf0, self.f_star, self.c_star,
                             self._rho_next, self._status, stream=s)
        self._rho, self._rho_next = self._rho_next, self._rho
        self.k += 1

    def serial_reference(self) -> torch.Tensor:
        """rho^n = F^n rho^0, n = 0..K."""
        s = self._s()
        out = torch.empty(self.K + 1, self.grid.bins + 1, dtype=torch.float64, device=self.device)
        out[0].copy_(self.cdf0)
        for n in range(self.K):
            L.pr_coarse_fp(self.fine, out[n:n + 1], out[n + 1:n + 2], 1, stream=s)
        return out

    def w1_to(self, ref: torch.Tensor) -> torch.Tensor:
        out = torch.empty(self.K + 1, dtype=torch.float64, device=self.device)
        L.pr_w1(self.grid, self.K + 1, self._rho, ref, out, stream=self._s())
        return out

    def close(self):
        for h in ("fine", "coarse"):
            if getattr(self, h, None):
                L.pr_coarse_destroy(getattr(self, h))
                setattr(self, h, None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
