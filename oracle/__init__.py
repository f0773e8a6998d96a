"""FP64 CPU oracle for the MacCormack-TVD compressible-convection step.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and bench.py's
CPU-baseline / reference leg may import this package; the product package
``paper_2411_10372_gb300`` never does.  It is a ctypes wrapper around
``cm_oracle.c`` (plain C, FP64, compiled with ``-O2 -ffp-contract=off``),
which follows Sec. 2 (equations, closures, Nu/Re definitions) and Sec. 3.1
(vector form, operator splitting, predictor / corrector / TVD) of
arXiv 2411.10372.  The C file's header lists the readings taken where the
paper is silent or garbled.

State arrays are float64 numpy arrays of shape (nf, nz, nx) in 2D
(fields rho, m_x, m_z, E) or (nf, nz, ny, nx) in 3D (rho, m_x, m_y, m_z, E).

Parity status of each function (what pins it, see tests/test_oracle_*.py):
  init / profile ... closed-form hydrostatic balance, isobaric perturbation
  sweep / step ..... mass conservation, hydrostatic rest, acoustic speed,
                     shear / thermal / sound decay rates, Sod shock tube
  dt ............... closed form on the conduction state
  diag ............. Nu = 1 on the conduction state, analytic fields
  stretched z-grid . exact mass conservation, steady linear conduction without
                     gravity, exact trapezoid / plate-derivative rules, second-
                     order self-convergence on nested tanh grids
  advect1d ......... total-variation test of the TVD reading
  ext_profiles /
  extended ......... closed forms of the force terms on polynomial and
                     trigonometric fields (uniform and stretched planes), C of
                     trigonometric fields, boundary layers of a built profile,
                     exact histogram counts
  torch_ref.py ..... PyTorch restatement of the 2D step for autograd (the
                     adjoint's reference): equal to this oracle state by
                     state and in Nu_bar; its gradient equals central
                     differences of this oracle (tests/test_torch_ref_pins.py)
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile cm_oracle.c into liboracle.so next to it (gcc, FP64, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
             "-shared", "-o", tmp, _SRC, "-lm"],
            check=True,
        )
        os.replace(tmp, _LIB)
    return _LIB


_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")


def build_omp(force: bool = False) -> str | None:
    """The same source with -fopenmp (liboracle_omp.so): the sweeps' per-node
    loops run on all host cores, with the same values bit for bit.  None if
    the compiler has no OpenMP."""
    if force or not os.path.exists(_LIB_OMP) or os.path.getmtime(_LIB_OMP) < os.path.getmtime(_SRC):
        tmp = _LIB_OMP + f".tmp{os.getpid()}"
        r = subprocess.run(
            ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
             "-shared", "-o", tmp, _SRC, "-lm"], capture_output=True)
        if r.returncode != 0:
            return None
        os.replace(tmp, _LIB_OMP)
    return _LIB_OMP


class _Cfg(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("tvd_form", ctypes.c_int), ("split", ctypes.c_int),
        ("aspect", ctypes.c_double), ("Ra", ctypes.c_double), ("Pr", ctypes.c_double),
        ("gamma", ctypes.c_double), ("eps", ctypes.c_double), ("D", ctypes.c_double),
        ("cfl", ctypes.c_double), ("dt_fixed", ctypes.c_double), ("gravity", ctypes.c_double),
        ("t_bot", ctypes.c_double), ("t_top", ctypes.c_double), ("pert_amp", ctypes.c_double),
        ("stokes", ctypes.c_double), ("seed", ctypes.c_uint64),
        ("zstretch", ctypes.c_double), ("znodes", ctypes.POINTER(ctypes.c_double)),
    ]


TVD_SPLIT, TVD_SUM, TVD_OFF = 0, 1, 2


@dataclass
class Config:
    """Problem definition.  Defaults: eps = 0.1, D = 0.5 (the paper's production
    values), Gamma = 4, CFL 0.5, Stokes stress, Davis-form TVD term."""
    nx: int = 256
    nz: int = 64
    ny: int = 1
    ndim: int = 2
    Ra: float = 1e6
    Pr: float = 1.0
    gamma: float = 5.0 / 3.0
    eps: float = 0.1
    D: float = 0.5
    aspect: float = 4.0
    cfl: float = 0.5
    dt_fixed: float = 0.0
    gravity: float = 1.0
    t_bot: float = 1.0
    t_top: float | None = None        # None: 1 - eps - D
    pert_amp: float = 1e-3
    seed: int = 12345
    tvd_form: int = TVD_SPLIT
    split: int = 0                    # 0: Eq. time_step as printed; 1: palindrome x, (y), z, z, (y), x
    stokes: float = -2.0 / 3.0
    zstretch: float = 0.0             # beta of the tanh z-grid (Sec. 3); 0 = uniform
    znodes: "np.ndarray | None" = None  # explicit plane heights, overriding zstretch

    @property
    def nf(self) -> int:
        return 5 if self.ndim == 3 else 4

    @property
    def shape(self) -> tuple:
        if self.ndim == 3:
            return (5, self.nz, self.ny, self.nx)
        return (4, self.nz, self.nx)

    def c(self) -> _Cfg:
        t_top = (1.0 - self.eps - self.D) if self.t_top is None else self.t_top
        zn = None
        if self.znodes is not None:
            zn = np.ascontiguousarray(self.znodes, dtype=np.float64)
            assert zn.shape == (self.nz,)
        c = _Cfg(self.ndim, self.nx, self.ny if self.ndim == 3 else 1, self.nz,
                 self.tvd_form, self.split, self.aspect, self.Ra, self.Pr, self.gamma, self.eps,
                 self.D, self.cfl, self.dt_fixed, self.gravity, self.t_bot, t_top,
                 self.pert_amp, self.stokes, self.seed & 0xFFFFFFFFFFFFFFFF, self.zstretch,
                 zn.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if zn is not None else None)
        c._keep = zn  # the C side reads znodes through the pointer
        return c


_lib = None


class library:
    """Context manager that points this wrapper at another build of the oracle
    (used by the mutation test, which plants mistakes in copies of cm_oracle.c)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        self._saved = _lib
        _lib = None
        lib(self.path)
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved
        return False


def lib(path: str | None = None):
    global _lib
    if _lib is None:
        L = ctypes.CDLL(path or build())
        dp = ctypes.POINTER(ctypes.c_double)
        cp = ctypes.POINTER(_Cfg)
        L.orc_init.argtypes = [cp, dp]
        L.orc_profile.argtypes = [cp, dp, dp, dp]
        L.orc_znodes.argtypes = [cp, dp]
        L.orc_ext_profiles.argtypes = [cp, dp, dp]
        L.orc_extended.argtypes = [cp, dp, dp, ctypes.POINTER(ctypes.c_longlong), ctypes.c_int, ctypes.c_double,
                                   ctypes.c_double]
        L.orc_sweep.argtypes = [cp, ctypes.c_int, ctypes.c_double, dp]
        L.orc_dt.argtypes = [cp, dp]
        L.orc_dt.restype = ctypes.c_double
        L.orc_step.argtypes = [cp, dp, ctypes.c_int, dp, dp]
        L.orc_diag.argtypes = [cp, dp, dp]
        L.orc_advect1d.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_int, ctypes.c_int, dp]
        L.orc_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.orc_splitmix64.restype = ctypes.c_uint64
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def init(cfg: Config) -> np.ndarray:
    """Initial state: conduction profile + isobaric seeded temperature perturbation."""
    X = np.zeros(cfg.shape, dtype=np.float64)
    c = cfg.c()
    lib().orc_init(ctypes.byref(c), _ptr(X))
    return X


def profile(cfg: Config):
    """(T_c, p_c, rho_c) per z-plane of the conduction / hydrostatic state."""
    T = np.zeros(cfg.nz); p = np.zeros(cfg.nz); r = np.zeros(cfg.nz)
    c = cfg.c()
    lib().orc_profile(ctypes.byref(c), _ptr(T), _ptr(p), _ptr(r))
    return T, p, r


def znodes(cfg: Config) -> np.ndarray:
    """The nz plane heights of cfg's z-grid (uniform, tanh of cfg.zstretch, or cfg.znodes)."""
    z = np.zeros(cfg.nz)
    c = cfg.c()
    lib().orc_znodes(ctypes.byref(c), _ptr(z))
    return z


def sweep(cfg: Config, X: np.ndarray, direction: int, Delta: float) -> np.ndarray:
    """One directional operator L_dir(Delta); direction 0 = x, 1 = y, 2 = z."""
    Y = np.ascontiguousarray(X, dtype=np.float64).copy()
    c = cfg.c()
    lib().orc_sweep(ctypes.byref(c), int(direction), float(Delta), _ptr(Y))
    return Y


def dt(cfg: Config, X: np.ndarray) -> float:
    Xc = np.ascontiguousarray(X, dtype=np.float64)
    c = cfg.c()
    return float(lib().orc_dt(ctypes.byref(c), _ptr(Xc)))


def step(cfg: Config, X: np.ndarray, nsteps: int, t0: float = 0.0):
    """Advance nsteps full steps.  Returns (X_new, t_new, dts)."""
    Y = np.ascontiguousarray(X, dtype=np.float64).copy()
    t = ctypes.c_double(t0)
    dts = np.zeros(max(nsteps, 1))
    c = cfg.c()
    lib().orc_step(ctypes.byref(c), _ptr(Y), int(nsteps), ctypes.byref(t), _ptr(dts))
    return Y, t.value, dts[:nsteps]


DIAG_KEYS = ("Nu", "Nu_conv", "Nu_K", "Nu_bot", "Nu_top", "Nu_bar", "Re", "KE", "mass",
             "energy", "Mach_max")


def diag(cfg: Config, X: np.ndarray) -> dict:
    Xc = np.ascontiguousarray(X, dtype=np.float64)
    out = np.zeros(len(DIAG_KEYS))
    c = cfg.c()
    lib().orc_diag(ctypes.byref(c), _ptr(Xc), _ptr(out))
    return dict(zip(DIAG_KEYS, out.tolist()))


EXT_PROFILE_KEYS = ("F_n", "F_p", "F_b", "F_v", "rho_uz_sq", "Tsa_sq", "Tsa", "rho_minus_rhoA", "U")
EXT_KEYS = ("C", "rho_uz_sq", "Tsa_sq", "lambda_b", "lambda_t", "F_n", "F_p", "F_b", "F_v", "r_max",
            "lambda_b_slope", "lambda_t_slope")


def ext_profiles(cfg: Config, X: np.ndarray) -> dict:
    """Plane means of the z-momentum terms, of (rho u_z)^2, T_sa^2, T_sa, rho - rho_A and
    the rms velocity U (name -> nz values)."""
    Xc = np.ascontiguousarray(X, dtype=np.float64)
    out = np.zeros((cfg.nz, 9))
    c = cfg.c()
    lib().orc_ext_profiles(ctypes.byref(c), _ptr(Xc), _ptr(out))
    return {k: out[:, q].copy() for q, k in enumerate(EXT_PROFILE_KEYS)}


def extended(cfg: Config, X: np.ndarray, nbins: int = 64, lo: float = -16.0, hi: float = 0.0):
    """(dict of C, boundary-layer thicknesses, volume-averaged forces, r_max;
    histogram of log10 K_e/I_e)."""
    Xc = np.ascontiguousarray(X, dtype=np.float64)
    out = np.zeros(len(EXT_KEYS))
    hist = np.zeros(nbins, dtype=np.int64)
    c = cfg.c()
    lib().orc_extended(ctypes.byref(c), _ptr(Xc), _ptr(out), hist.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                       int(nbins), float(lo), float(hi))
    return dict(zip(EXT_KEYS, out.tolist())), hist


def advect1d(u0: np.ndarray, a: float, dt: float, h: float, nsteps: int, tvd_form: int) -> np.ndarray:
    u = np.ascontiguousarray(u0, dtype=np.float64).copy()
    lib().orc_advect1d(len(u), a, dt, h, nsteps, tvd_form, _ptr(u))
    return u


def splitmix64(seed: int, idx: int) -> int:
    return int(lib().orc_splitmix64(seed & 0xFFFFFFFFFFFFFFFF, idx & 0xFFFFFFFFFFFFFFFF))
