"""ctypes binding of include/cm.h (argument marshalling only).

Every function here has the name of the C entry point it calls; all
arithmetic of the solver runs in the CUDA kernels of libcm.so.  There is no
fallback: if libcm.so cannot be loaded, `lib()` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcm.so")

CM_OK, CM_EINVAL, CM_ECUDA, CM_ENOTINIT, CM_ENAN = 0, -1, -2, -3, -4
CM_EUNSTABLE, CM_ENOMEM, CM_EBADCKPT = -7, -8, -9
CM_FP64, CM_FP32 = 0, 1
CM_TVD_DAVIS, CM_TVD_SUM, CM_TVD_OFF = 0, 1, 2
CM_ADJ_PHI_EXACT, CM_ADJ_PHI_FROZEN = 0, 1
CM_SPLIT_PRINTED, CM_SPLIT_SYMMETRIC = 0, 1


class cm_grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("aspect", ctypes.c_double), ("zstretch", ctypes.c_double),
                ("znodes", ctypes.POINTER(ctypes.c_double))]


class cm_params(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("D", ctypes.c_double), ("cfl", ctypes.c_double),
                ("dt_fixed", ctypes.c_double), ("gravity", ctypes.c_double), ("t_bot", ctypes.c_double),
                ("t_top", ctypes.c_double), ("pert_amp", ctypes.c_double), ("stokes", ctypes.c_double),
                ("seed", ctypes.c_ulonglong), ("precision", ctypes.c_int), ("tvd_form", ctypes.c_int),
                ("diag_every", ctypes.c_int), ("diag_capacity", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("state_buf", ctypes.c_void_p), ("adj_limiter", ctypes.c_int), ("layout_exact", ctypes.c_int),
                ("split", ctypes.c_int), ("reserved_", ctypes.c_int)]


class cm_diag(ctypes.Structure):
    _fields_ = [("step", ctypes.c_longlong), ("t", ctypes.c_double), ("dt", ctypes.c_double),
                ("Nu", ctypes.c_double), ("Nu_conv", ctypes.c_double), ("Nu_K", ctypes.c_double),
                ("Nu_bot", ctypes.c_double), ("Nu_top", ctypes.c_double), ("Nu_bar", ctypes.c_double),
                ("Re", ctypes.c_double), ("KE", ctypes.c_double), ("mass", ctypes.c_double),
                ("energy", ctypes.c_double), ("mach_max", ctypes.c_double), ("status", ctypes.c_int),
                ("pad_", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "pad_"}


class cm_ext(ctypes.Structure):
    _fields_ = [(f, ctypes.c_double) for f in ("C", "rho_uz_sq", "Tsa_sq", "lambda_b", "lambda_top", "F_n", "F_p",
                                               "F_b", "F_v", "r_max", "lambda_b_slope", "lambda_top_slope")]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class CMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (status {code})")
        self.code = code


_SIGS = {
    "cm_default_params": (ctypes.c_int, [ctypes.POINTER(cm_params)]),
    "cm_state_bytes": (ctypes.c_int, [ctypes.POINTER(cm_grid), ctypes.c_int, ctypes.POINTER(ctypes.c_ulonglong)]),
    "cm_init": (ctypes.c_int, [ctypes.POINTER(cm_grid), ctypes.c_double, ctypes.c_double, ctypes.c_double,
                               ctypes.POINTER(cm_params)]),
    "cm_step": (ctypes.c_int, [ctypes.c_int]),
    "cm_sample": (ctypes.c_int, []),
    "cm_diagnostics": (ctypes.c_int, [ctypes.POINTER(cm_diag), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "cm_state_ptr": (ctypes.c_void_p, [ctypes.c_int]),
    "cm_state_layout": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int)] * 3),
    "cm_get_state": (ctypes.c_int, [ctypes.c_void_p]),
    "cm_set_state": (ctypes.c_int, [ctypes.c_void_p]),
    "cm_set_temperature": (ctypes.c_int, [ctypes.c_void_p]),
    "cm_run_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(cm_diag)]),
    "cm_sweep": (ctypes.c_int, [ctypes.c_int, ctypes.c_double]),
    "cm_get_dt": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double)]),
    "cm_get_time": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]),
    "cm_profile_steps": (ctypes.c_int, [ctypes.c_int, ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double)]),
    "cm_launch_count": (ctypes.c_longlong, []),
    "cm_sync": (ctypes.c_int, []),
    "cm_save": (ctypes.c_int, [ctypes.c_char_p]),
    "cm_load": (ctypes.c_int, [ctypes.c_char_p]),
    "cm_profiles": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double)]),
    "cm_tuning": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "cm_znodes": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double)]),
    "cm_ext_profiles": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double)]),
    "cm_extended": (ctypes.c_int, [ctypes.POINTER(cm_ext), ctypes.POINTER(ctypes.c_longlong), ctypes.c_int,
                                   ctypes.c_double, ctypes.c_double]),
    "cm_run_host_f32": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(cm_diag)]),
    "cm_adj_forward": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "cm_adj_backward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "cm_adj_set_dts": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
    "cm_adj_get_dts": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
    "cm_diag_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(cm_grid), ctypes.c_int,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.POINTER(cm_params),
                                       ctypes.c_double, ctypes.c_double, ctypes.c_longlong, ctypes.c_void_p,
                                       ctypes.POINTER(cm_diag)]),
    "cm_batch_init": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(cm_grid), ctypes.POINTER(ctypes.c_double),
                                     ctypes.c_double, ctypes.c_double, ctypes.POINTER(cm_params)]),
    "cm_batch_step": (ctypes.c_int, [ctypes.c_int]),
    "cm_batch_diagnostics": (ctypes.c_int, [ctypes.POINTER(cm_diag)]),
    "cm_batch_get_state": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p]),
    "cm_batch_tuning": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "cm_batch_profile_steps": (ctypes.c_int, [ctypes.c_int, ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_double)]),
    "cm_batch_launch_count": (ctypes.c_longlong, []),
    "cm_batch_finalize": (ctypes.c_int, []),
    "cm_finalize": (ctypes.c_int, []),
    "cm_last_error": (ctypes.c_char_p, []),
}

_lib = None


def lib(build_if_missing: bool = True):
    """Load libcm.so (building it with nvcc if it is missing or stale)."""
    global _lib
    if _lib is None:
        if build_if_missing:
            from . import build as _build
            _build.build()
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library {LIB_PATH} is missing: run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc: int):
    if rc != CM_OK:
        raise CMError(rc, lib().cm_last_error().decode())
    return rc


def _dp(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return ctypes.c_void_p(a.ctypes.data)


# ---- the C entry points, same names -----------------------------------------

def cm_default_params() -> cm_params:
    p = cm_params()
    _check(lib().cm_default_params(ctypes.byref(p)))
    return p


def cm_state_bytes(grid: cm_grid, precision: int) -> int:
    b = ctypes.c_ulonglong()
    _check(lib().cm_state_bytes(ctypes.byref(grid), precision, ctypes.byref(b)))
    return b.value


def cm_init(grid: cm_grid, Ra: float, Pr: float, gamma: float, params: cm_params | None = None):
    _check(lib().cm_init(ctypes.byref(grid), Ra, Pr, gamma, ctypes.byref(params) if params is not None else None))


def cm_step(n: int):
    _check(lib().cm_step(int(n)))


def cm_sample():
    _check(lib().cm_sample())


def cm_diagnostics(max_samples: int = 4096) -> list[dict]:
    buf = (cm_diag * max(max_samples, 1))()
    n = ctypes.c_int()
    rc = lib().cm_diagnostics(buf, max_samples, ctypes.byref(n))
    out = [buf[i].as_dict() for i in range(n.value)]
    _check(rc)
    return out


def cm_state_ptr(field: int) -> int:
    return lib().cm_state_ptr(field) or 0


def cm_state_layout() -> tuple[int, int, int]:
    p, n, e = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().cm_state_layout(ctypes.byref(p), ctypes.byref(n), ctypes.byref(e)))
    return p.value, n.value, e.value


def cm_get_state(out: np.ndarray) -> np.ndarray:
    _check(lib().cm_get_state(_dp(out)))
    return out


def cm_set_state(state: np.ndarray):
    _check(lib().cm_set_state(_dp(np.ascontiguousarray(state, dtype=np.float64))))


def cm_set_temperature(T: np.ndarray):
    """The initial condition of cm_init built on the temperature field T (nz x nx, or nz x ny x nx)."""
    _check(lib().cm_set_temperature(_dp(np.ascontiguousarray(T, dtype=np.float64))))


def cm_run_host(state_in: np.ndarray | None, nsteps: int, state_out: np.ndarray | None = None,
                want_diag: bool = True):
    d = cm_diag()
    _check(lib().cm_run_host(_dp(state_in), int(nsteps), _dp(state_out), ctypes.byref(d) if want_diag else None))
    return d.as_dict() if want_diag else None


def cm_sweep(direction: int, Delta: float):
    _check(lib().cm_sweep(int(direction), float(Delta)))


def cm_get_dt() -> float:
    v = ctypes.c_double()
    _check(lib().cm_get_dt(ctypes.byref(v)))
    return v.value


def cm_get_time() -> tuple[float, int]:
    t, s = ctypes.c_double(), ctypes.c_longlong()
    _check(lib().cm_get_time(ctypes.byref(t), ctypes.byref(s)))
    return t.value, s.value


def cm_profile_steps(n: int, flush_bytes: int = 0, per_sweep: bool = True) -> tuple[list[float], list[float]]:
    """(mean ms per sweep position, ms of each step) of n profiled steps; with
    per_sweep=False only the steps are bracketed (the sweep list is empty)."""
    ms = (ctypes.c_double * 6)()
    steps = (ctypes.c_double * n)()
    _check(lib().cm_profile_steps(int(n), int(flush_bytes), ms if per_sweep else None, steps))
    if not per_sweep:
        return [], list(steps)
    _, nf, _ = cm_state_layout()
    return list(ms)[: 6 if nf == 5 else 4], list(steps)


PROFILE_KEYS = ("rho", "E", "conv_flux", "kin_flux", "u2", "KE", "T", "mach_max")


def cm_profiles(nz: int) -> dict:
    """Plane means of the current state (include/cm.h): name -> array of nz values."""
    out = np.empty((nz, 8), dtype=np.float64)
    _check(lib().cm_profiles(out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return {k: out[:, q].copy() for q, k in enumerate(PROFILE_KEYS)}


EXT_PROFILE_KEYS = ("F_n", "F_p", "F_b", "F_v", "rho_uz_sq", "Tsa_sq", "Tsa", "rho_minus_rhoA", "U")


def cm_ext_profiles(nz: int) -> dict:
    """Plane means of the z-momentum terms, (rho u_z)^2, T_sa^2, and the profiles T_sa,
    rho - rho_A, U (include/cm.h): name -> nz values."""
    out = np.empty((nz, 9), dtype=np.float64)
    _check(lib().cm_ext_profiles(out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return {k: out[:, q].copy() for q, k in enumerate(EXT_PROFILE_KEYS)}


def cm_extended(nbins: int = 64, log10_lo: float = -16.0, log10_hi: float = 0.0):
    """(cm_ext as a dict, histogram of log10 K_e/I_e as int64 array; None if nbins == 0)."""
    e = cm_ext()
    hist = np.zeros(max(nbins, 1), dtype=np.int64)
    hp = hist.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)) if nbins > 0 else None
    _check(lib().cm_extended(ctypes.byref(e), hp, int(nbins), float(log10_lo), float(log10_hi)))
    return e.as_dict(), (hist if nbins > 0 else None)


def cm_znodes(nz: int) -> np.ndarray:
    """The nz plane heights of the context's z-grid (include/cm.h)."""
    z = np.empty(nz, dtype=np.float64)
    _check(lib().cm_znodes(z.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return z


def cm_tuning() -> tuple[int, int]:
    """(rows per segment of the z sweep, of the x sweep) chosen at cm_init (0 = model)."""
    z, x = ctypes.c_int(), ctypes.c_int()
    _check(lib().cm_tuning(ctypes.byref(z), ctypes.byref(x)))
    return z.value, x.value


def cm_launch_count() -> int:
    return int(lib().cm_launch_count())


def cm_sync():
    _check(lib().cm_sync())


def cm_save(path: str):
    _check(lib().cm_save(path.encode()))


def cm_load(path: str):
    _check(lib().cm_load(path.encode()))


def cm_diag_noalloc(state_ptr: int, precision: int, grid: cm_grid, pitch: int, Ra: float, Pr: float,
                    gamma: float, params: cm_params, t: float = 0.0, dt: float = 0.0, step: int = 0,
                    stream: int | None = None) -> dict:
    """Diagnostics of a device state without allocating (see include/cm.h)."""
    d = cm_diag()
    _check(lib().cm_diag_noalloc(ctypes.c_void_p(state_ptr), int(precision), ctypes.byref(grid), int(pitch),
                                 float(Ra), float(Pr), float(gamma), ctypes.byref(params), float(t), float(dt),
                                 int(step), ctypes.c_void_p(stream) if stream else None, ctypes.byref(d)))
    return d.as_dict()


def _any_ptr(a):
    """Host numpy float64 array, a CUDA tensor (its data pointer) or None."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return _dp(a)
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous() and str(a.dtype) == "torch.float64"
        return ctypes.c_void_p(a.data_ptr())
    raise TypeError("expected a float64 numpy array or torch tensor")


def _fp(a):
    if a is None:
        return None
    assert a.dtype == np.float32 and a.flags.c_contiguous
    return ctypes.c_void_p(a.ctypes.data)


def cm_run_host_f32(state_in: np.ndarray | None, nsteps: int, state_out: np.ndarray | None = None,
                    want_diag: bool = True):
    """cm_run_host with float32 host arrays (FP32 contexts)."""
    d = cm_diag()
    _check(lib().cm_run_host_f32(_fp(state_in), int(nsteps), _fp(state_out), ctypes.byref(d) if want_diag else None))
    return d.as_dict() if want_diag else None


def cm_adj_forward(nsteps: int, K: int, win_begin: int) -> float:
    """Forward run for the adjoint; returns J (see include/cm.h)."""
    J = ctypes.c_double()
    _check(lib().cm_adj_forward(int(nsteps), int(K), int(win_begin), ctypes.byref(J)))
    return J.value


def cm_adj_backward(grad_X0=None, grad_T0=None) -> float:
    """Reverse pass; fills grad_X0 / grad_T0 (host arrays or CUDA tensors) and returns dJ/dRa."""
    g = ctypes.c_double()
    _check(lib().cm_adj_backward(_any_ptr(grad_X0), _any_ptr(grad_T0), ctypes.byref(g)))
    return g.value


def cm_adj_set_dts(dts) -> None:
    """Replay these per-step dts in the next cm_adj_forward of len(dts) steps (None or [] clears)."""
    a = np.ascontiguousarray([] if dts is None else dts, dtype=np.float64)
    _check(lib().cm_adj_set_dts(a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a.size else None, int(a.size)))


def cm_adj_get_dts(nsteps: int) -> np.ndarray:
    """The dt of each step of the last cm_adj_forward (nsteps of them)."""
    out = np.empty(int(nsteps), dtype=np.float64)
    _check(lib().cm_adj_get_dts(out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(nsteps)))
    return out


_batch_n = 0


def cm_batch_init(grids: list, Ra: list, Pr: float, gamma: float, params: cm_params | None = None):
    global _batch_n
    n = len(grids)
    g = (cm_grid * n)(*grids)
    ra = (ctypes.c_double * n)(*[float(r) for r in Ra])
    _check(lib().cm_batch_init(n, g, ra, Pr, gamma, ctypes.byref(params) if params is not None else None))
    _batch_n = n


def cm_batch_step(n: int):
    _check(lib().cm_batch_step(int(n)))


def cm_batch_diagnostics() -> list[dict]:
    out = (cm_diag * max(_batch_n, 1))()
    _check(lib().cm_batch_diagnostics(out))
    return [out[i].as_dict() for i in range(_batch_n)]


def cm_batch_get_state(box: int, out: np.ndarray) -> np.ndarray:
    _check(lib().cm_batch_get_state(int(box), _dp(out)))
    return out


def cm_batch_tuning() -> tuple[list[int], list[int]]:
    z = (ctypes.c_int * max(_batch_n, 1))()
    x = (ctypes.c_int * max(_batch_n, 1))()
    _check(lib().cm_batch_tuning(z, x))
    return list(z)[:_batch_n], list(x)[:_batch_n]


def cm_batch_profile_steps(n: int, flush_bytes: int = 0) -> float:
    ms = ctypes.c_double()
    _check(lib().cm_batch_profile_steps(int(n), int(flush_bytes), ctypes.byref(ms)))
    return ms.value


def cm_batch_launch_count() -> int:
    return int(lib().cm_batch_launch_count())


def cm_batch_finalize():
    _check(lib().cm_batch_finalize())


def cm_finalize():
    _check(lib().cm_finalize())


def cm_last_error() -> str:
    return lib().cm_last_error().decode()
