"""torch.autograd.Function around the library's adjoint (marshalling only).

J = time average of the plate Nusselt number Nu_bar (Eq. mean_Nu) over steps
win_begin..nsteps of an FP64 2D run started from X0, as a function of X0 and
Ra; every step's dt is the CFL dt of the forward run, held fixed (see
cm_adj_forward in include/cm.h).  The forward and the reverse pass both run in
libcm.so; this module only moves arrays and scalars.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _binding as B


class NuObjective(torch.autograd.Function):
    """NuObjective.apply(X0, Ra, grid, nsteps, K, win_begin) -> J.

    X0: float64 tensor (4, nz, nx) in the cm_get_state layout; Ra: 0-dim
    float64 tensor; grid: dict with nx, nz and optionally Pr, gamma, aspect and
    any cm_params field; K: checkpoint interval.  The library keeps one
    context per process, so the backward of this node must run before another
    context is created."""

    @staticmethod
    def forward(ctx, X0, Ra, grid, nsteps, K, win_begin):
        from . import Solver
        kw = dict(grid)
        nx, nz = kw.pop("nx"), kw.pop("nz")
        Pr, gamma = kw.pop("Pr", 1.0), kw.pop("gamma", 5.0 / 3.0)
        s = Solver(nx, nz, float(Ra), Pr, gamma, precision="fp64", **kw)
        s.set_state(np.ascontiguousarray(X0.detach().cpu().numpy(), dtype=np.float64))
        J = B.cm_adj_forward(int(nsteps), int(K), int(win_begin))
        ctx.solver = s
        ctx.shape = tuple(X0.shape)
        ctx.device = X0.device
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        gX = np.empty(ctx.shape, dtype=np.float64)
        gRa = B.cm_adj_backward(gX, None)
        ctx.solver.close()
        g = gJ.to(torch.float64)
        return (torch.from_numpy(gX).to(ctx.device) * g, g * gRa, None, None, None, None)
