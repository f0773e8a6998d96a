"""torch.autograd.Functions around the library's adjoint (marshalling only).

J = time average of the plate Nusselt number Nu_bar (Eq. mean_Nu) over steps
win_begin..nsteps of an FP64 2D run, as a function of its initial condition
and Ra; every step's dt is the CFL dt of the forward run, held fixed (see
cm_adj_forward in include/cm.h).  The forward and the reverse pass both run in
libcm.so; this module only moves arrays and scalars.  Gradients are written
by the library straight into tensors on the input's device (CUDA tensors
receive them device to device).

The derivative of the TVD limiter is a reading: grid["adj_limiter"] =
CM_ADJ_PHI_EXACT (default) differentiates phi exactly where it is smooth,
CM_ADJ_PHI_FROZEN holds the limiter's ratios fixed, which keeps gradients of
long windows bounded (include/cm.h states why).
"""
from __future__ import annotations

import numpy as np
import torch

from . import _binding as B


def _solver(grid, Ra):
    from . import Solver
    kw = dict(grid)
    nx, nz = kw.pop("nx"), kw.pop("nz")
    Pr, gamma = kw.pop("Pr", 1.0), kw.pop("gamma", 5.0 / 3.0)
    return Solver(nx, nz, float(Ra), Pr, gamma, precision="fp64", **kw)


def _grad_buffer(like: torch.Tensor, shape):
    """A float64 buffer for the library to fill: a CUDA tensor on the input's
    device, else a host numpy array."""
    if like.is_cuda:
        return torch.empty(shape, dtype=torch.float64, device=like.device)
    return np.empty(shape, dtype=np.float64)


def _as_tensor(buf, device):
    return buf if isinstance(buf, torch.Tensor) else torch.from_numpy(buf).to(device)


class NuObjective(torch.autograd.Function):
    """NuObjective.apply(X0, Ra, grid, nsteps, K, win_begin) -> J.

    X0: float64 tensor (4, nz, nx) in the cm_get_state layout; Ra: 0-dim
    float64 tensor; grid: dict with nx, nz and optionally Pr, gamma, aspect and
    any cm_params field; K: checkpoint interval.  The library keeps one
    context per process, so the backward of this node must run before another
    context is created."""

    @staticmethod
    def forward(ctx, X0, Ra, grid, nsteps, K, win_begin):
        s = _solver(grid, Ra)
        s.set_state(np.ascontiguousarray(X0.detach().cpu().numpy(), dtype=np.float64))
        J = B.cm_adj_forward(int(nsteps), int(K), int(win_begin))
        ctx.solver = s
        ctx.shape = tuple(X0.shape)
        ctx.like = X0
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        gX = _grad_buffer(ctx.like, ctx.shape)
        gRa = B.cm_adj_backward(gX, None)
        ctx.solver.close()
        g = gJ.to(torch.float64)
        return (_as_tensor(gX, ctx.like.device) * g.to(ctx.like.device), g * gRa, None, None, None, None)


class NuObjectiveT(torch.autograd.Function):
    """NuObjectiveT.apply(T0, Ra, grid, nsteps, K, win_begin) -> J, as a
    function of the initial temperature field.

    T0: float64 tensor (nz, nx), the temperature of the initial condition of
    cm_init (isobaric at the conduction pressure, u = 0; cm_set_temperature);
    its plate rows are ignored (the plates keep their temperatures) and get a
    zero gradient.  Ra, grid, nsteps, K, win_begin as for NuObjective.  The
    gradient is dJ/dT0 at fixed pressure and velocity (cm_adj_backward's
    grad_T0)."""

    @staticmethod
    def forward(ctx, T0, Ra, grid, nsteps, K, win_begin):
        s = _solver(grid, Ra)
        B.cm_set_temperature(np.ascontiguousarray(T0.detach().cpu().numpy(), dtype=np.float64))
        J = B.cm_adj_forward(int(nsteps), int(K), int(win_begin))
        ctx.solver = s
        ctx.shape = tuple(T0.shape)
        ctx.like = T0
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        gT = _grad_buffer(ctx.like, ctx.shape)
        gRa = B.cm_adj_backward(None, gT)
        ctx.solver.close()
        g = gJ.to(torch.float64)
        return (_as_tensor(gT, ctx.like.device) * g.to(ctx.like.device), g * gRa, None, None, None, None)
