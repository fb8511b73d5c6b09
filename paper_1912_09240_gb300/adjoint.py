"""Pathwise gradients of the fine propagator with fixed noise.

``FineEM`` is a ``torch.autograd.Function``: its forward runs
``pr_fine_propagate`` over consecutive slices (binary32 state), its backward
runs ``pr_fine_adjoint`` seeded with the incoming gradient and returns
dL/d(lambda, beta, eps) and dL/d(X_0, Y_0).  The two helpers compute the two
observables of the adjoint workload: the second moment E[X_T^2] and the
empirical quantile function Q(p_j) = X_(ceil(p_j N)), p_j = (j + 1/2)/M, whose
pathwise derivative is that of the particle holding the rank (order
statistics), with their gradients.  The binned quantile is piecewise constant
in the particle positions (zero derivative almost everywhere), hence order
statistics.

Tensors here are plumbing (device memory, workspaces, seeds); every step of
the propagation, the adjoint and the ranking runs in libpr.so.
"""
from __future__ import annotations

import math

import torch

from . import _lib as L


def _workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(nbytes, 1), dtype=torch.uint8, device=device)


class FineEM(torch.autograd.Function):
    """(X_T, Y_T) = F(X_0, Y_0; theta) over n_slices x steps EM steps, theta = (lambda, beta, eps)."""

    @staticmethod
    def forward(ctx, theta, x0, y0, kind: int, tau_x: float, rng: L.Rng, slice_begin: int, n_slices: int,
                steps: int, dt: float, ckpt_every: int = 256):
        lam, beta, eps = (float(v) for v in theta.detach().double().cpu())
        model = L.Model(kind, 1, lam, beta, eps, tau_x)
        n = x0.numel()
        x = x0.detach().reshape(1, n).to(torch.float32).clone()
        y = y0.detach().reshape(1, 1, n).to(torch.float32).clone()
        for s in range(n_slices):
            L.pr_fine_propagate(model, L.PR_F32, rng, x, y, False, x, y, n, slice_begin + s, 1, steps, dt)
        ctx.save_for_backward(x0.detach().reshape(n).to(torch.float32).contiguous(),
                              y0.detach().reshape(n).to(torch.float32).contiguous())
        ctx.cfg = (model, rng, n, slice_begin, n_slices, steps, dt, ckpt_every, theta.dtype, theta.device,
                   x0.shape, y0.shape, x0.dtype)
        return x.reshape(n), y.reshape(n)

    @staticmethod
    def backward(ctx, gx, gy):
        x0, y0 = ctx.saved_tensors
        model, rng, n, sb, ns, steps, dt, ck, tdtype, tdev, xshape, yshape, xdtype = ctx.cfg
        dev = x0.device
        xbar = (gx if gx is not None else torch.zeros(n, device=dev)).reshape(n).to(torch.float64).contiguous()
        ybar = (gy if gy is not None else torch.zeros(n, device=dev)).reshape(n).to(torch.float64).contiguous()
        grad = torch.zeros(3, dtype=torch.float64, device=dev)
        xb0 = torch.empty(n, dtype=torch.float64, device=dev)
        yb0 = torch.empty(n, dtype=torch.float64, device=dev)
        ws = _workspace(L.pr_fine_adjoint_workspace(n, ns, steps, ck), dev)
        L.pr_fine_adjoint(model, rng, x0, y0, n, sb, ns, steps, dt, ck, None, None, xbar, ybar, grad, xb0, yb0, ws)
        return (grad.to(device=tdev, dtype=tdtype), xb0.to(xdtype).reshape(xshape), yb0.to(xdtype).reshape(yshape),
                None, None, None, None, None, None, None, None)


def fine_em(theta, x0, y0, kind, tau_x, rng, slice_begin, n_slices, steps, dt, ckpt_every=256):
    return FineEM.apply(theta, x0, y0, kind, tau_x, rng, slice_begin, n_slices, steps, dt, ckpt_every)


def second_moment_gradient(model: L.Model, rng: L.Rng, x0, y0, slice_begin: int, n_slices: int, steps: int,
                           dt: float, ckpt_every: int = 256):
    """E[X_T^2] = mean_p X_T^2 and its gradient with respect to (lambda, beta, eps), in one adjoint pass:
    the seeds 2 X_T^p / N depend only on each particle's own end state, so the adjoint takes them
    after its own forward pass (pr_fine_adjoint_affine)."""
    n = x0.numel()
    dev = x0.device
    xT = torch.empty(n, dtype=torch.float32, device=dev)
    grad = torch.zeros(3, dtype=torch.float64, device=dev)
    ws = _workspace(L.pr_fine_adjoint_workspace(n, n_slices, steps, ckpt_every), dev)
    L.pr_fine_adjoint_affine(model, rng, x0.reshape(n).to(torch.float32).contiguous(),
                             y0.reshape(n).to(torch.float32).contiguous(), n, slice_begin, n_slices, steps, dt,
                             ckpt_every, 2.0 / n, 0.0, xT, None, grad, None, None, ws)
    moments = torch.empty(2, dtype=torch.float64, device=dev)   # E[X_T], E[X_T^2] (Eq. MCestimator)
    L.pr_moments(L.PR_F32, xT, n, None, n, 1, 2, moments, _workspace(L.pr_moments_workspace(n, 1, 2), dev))
    return moments[1], grad


def quantile_gradient(model: L.Model, rng: L.Rng, x0, y0, slice_begin: int, n_slices: int, steps: int, dt: float,
                      n_points: int = 512, ckpt_every: int = 256):
    """Q(p_j) = X_(r_j), r_j = ceil(p_j N) (1-based rank), p_j = (j + 1/2)/n_points, and
    dQ(p_j)/d(lambda, beta, eps) = dX_T/dtheta of the particle holding rank r_j.
    Returns (Q [n_points] float32, dQ [n_points][3] float64, particle indices [n_points])."""
    n = x0.numel()
    dev = x0.device
    xT = torch.empty(n, dtype=torch.float32, device=dev)
    grads = torch.empty(n, 3, dtype=torch.float64, device=dev)
    ws = _workspace(L.pr_fine_adjoint_workspace(n, n_slices, steps, ckpt_every), dev)
    L.pr_fine_adjoint(model, rng, x0.reshape(n).to(torch.float32).contiguous(),
                      y0.reshape(n).to(torch.float32).contiguous(), n, slice_begin, n_slices, steps, dt,
                      ckpt_every, xT, None, None, None, grads, None, None, ws)
    ranks = torch.tensor([max(1, math.ceil((j + 0.5) / n_points * n)) - 1 for j in range(n_points)],
                         dtype=torch.int64, device=dev)
    idx = torch.empty(n_points, dtype=torch.int64, device=dev)
    ws2 = _workspace(L.pr_order_statistics_workspace(n), dev)
    L.pr_order_statistics(xT, n, ranks, n_points, idx, ws2)
    return xT[idx], grads[idx], idx
