"""GB300-native MacCormack-TVD solver for fully compressible convection
(arXiv 2411.10372, Sec. 2 equations, Sec. 3.1 scheme).

The compute path is libcm.so (hand-written sm_103a CUDA kernels behind the C
ABI of include/cm.h); this package is its thin Python binding.  `Solver` is a
convenience wrapper that fills the C structs and moves numpy arrays; it does
no arithmetic of the method.
"""
from __future__ import annotations

import ctypes

import numpy as np

from ._binding import (cm_adj_backward, cm_adj_forward, cm_adj_get_dts, cm_adj_set_dts, CM_ADJ_PHI_EXACT,
                       CM_ADJ_PHI_FROZEN, CM_SPLIT_PRINTED, CM_SPLIT_SYMMETRIC, cm_batch_diagnostics, cm_batch_finalize, cm_batch_get_state, cm_batch_init,
                       cm_batch_launch_count, cm_batch_profile_steps, cm_batch_step, cm_batch_tuning,
                       CM_EBADCKPT, CM_ECUDA, CM_EINVAL, CM_ENAN, CM_ENOMEM, CM_ENOTINIT, CM_EUNSTABLE,
                       CM_FP32, CM_FP64, CM_OK, CM_TVD_DAVIS, CM_TVD_OFF, CM_TVD_SUM, CMError, cm_default_params,
                       cm_diag, cm_diag_noalloc, cm_diagnostics, cm_finalize, cm_get_dt, cm_get_state, cm_get_time, cm_grid,
                       cm_init, cm_last_error, cm_launch_count, cm_load, cm_profile_steps, cm_params, cm_run_host,
                       cm_profiles, cm_run_host_f32, cm_sample, cm_tuning,
                       cm_save, cm_set_state, cm_set_temperature, cm_state_bytes, cm_state_layout, cm_state_ptr, cm_step, cm_sweep,
                       cm_sync, cm_znodes, cm_ext, cm_ext_profiles, cm_extended, lib)

__all__ = [n for n in dir() if n.startswith("cm_") or n.startswith("CM")] + ["Solver", "lib"]


class Solver:
    """One solver context (the library keeps a single context per process).

    Parameters follow cm_params; `precision` is "fp64" or "fp32".  `stream`
    may be a torch.cuda.Stream (its handle is passed to the library).
    `zstretch` (beta of the tanh z-grid) or `znodes` (the nz plane heights)
    select a stretched z-grid (cm_grid)."""

    def __init__(self, nx: int, nz: int, Ra: float, Pr: float = 1.0, gamma: float = 5.0 / 3.0, *,
                 ny: int = 1, ndim: int = 2, aspect: float = 4.0, precision: str = "fp64", stream=None,
                 zstretch: float = 0.0, znodes=None, **params):
        zn = None
        if znodes is not None:
            zn = np.ascontiguousarray(znodes, dtype=np.float64)
            if zn.shape != (nz,):
                raise ValueError(f"znodes must hold nz = {nz} plane heights")
        self.grid = cm_grid(ndim, nx, ny if ndim == 3 else 1, nz, aspect, zstretch,
                            zn.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if zn is not None else None)
        p = cm_default_params()
        t_top_given = "t_top" in params
        for k, v in params.items():
            if not hasattr(p, k):
                raise TypeError(f"unknown parameter {k}")
            setattr(p, k, v)
        if not t_top_given:
            p.t_top = 1.0 - p.eps - p.D
        p.precision = CM_FP64 if precision == "fp64" else CM_FP32
        if stream is not None:
            p.stream = getattr(stream, "cuda_stream", stream)
        self.params = p
        self.Ra, self.Pr, self.gamma = Ra, Pr, gamma
        self.nf = 5 if ndim == 3 else 4
        cm_init(self.grid, Ra, Pr, gamma, p)
        self.grid.znodes = None  # read during cm_init only

    @property
    def z(self) -> np.ndarray:
        """Plane heights of the z-grid."""
        return cm_znodes(self.grid.nz)

    def ext_profiles(self) -> dict:
        """Plane means of F_n, F_p, F_b, F_v, (rho u_z)^2, T_sa^2, and the profiles T_sa, rho - rho_A, U."""
        return cm_ext_profiles(self.grid.nz)

    def extended(self, nbins: int = 64, log10_lo: float = -16.0, log10_hi: float = 0.0):
        """C(Ra), boundary layers, averaged z-momentum terms, max K_e/I_e and its histogram."""
        return cm_extended(nbins, log10_lo, log10_hi)

    @property
    def shape(self) -> tuple:
        g = self.grid
        if g.ndim == 3:
            return (5, g.nz, g.ny, g.nx)
        return (4, g.nz, g.nx)

    def state(self) -> np.ndarray:
        out = np.empty(self.shape, dtype=np.float64)
        return cm_get_state(out)

    def set_state(self, X: np.ndarray):
        cm_set_state(np.ascontiguousarray(X, dtype=np.float64).reshape(self.shape))

    def step(self, n: int = 1):
        cm_step(n)

    def sweep(self, direction: int, Delta: float):
        cm_sweep(direction, Delta)

    def sample(self) -> dict:
        cm_diagnostics(1 << 16)  # drop anything queued before
        cm_sample()
        return cm_diagnostics(1)[0]

    def diagnostics(self, max_samples: int = 1 << 16) -> list[dict]:
        return cm_diagnostics(max_samples)

    def dt(self) -> float:
        return cm_get_dt()

    def time(self) -> tuple[float, int]:
        return cm_get_time()

    def sync(self):
        cm_sync()

    def close(self):
        cm_finalize()
