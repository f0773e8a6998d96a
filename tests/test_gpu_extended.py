"""Parity of the extended diagnostics (plane means of the z-momentum terms,
C(Ra), boundary layers by the tangent construction and by the slope
criterion, K_e/I_e histogram; the analyses of Secs. 4-6) with
the FP64 oracle, through the C ABI.

Both sides evaluate every quantity in FP64 from the same state (FP32 states
widened), in the same order of operations per node; only the order of the
sums over nodes differs.  Bars: plane means and derived quantities <= 1e-12
relative (1e-12 of the largest plane value for profiles that cross zero);
boundary layers 1e-9 relative (a plate derivative amplifies the rounding of
the plane means, as for the plate Nusselt numbers); histogram counts exactly
equal.
"""
import math

import numpy as np
import pytest

import oracle as O
from test_gpu_stretched import solver_for, stirred_on, stirred_3d_on, solver3_for
from test_oracle_pins import random_planes

pytestmark = pytest.mark.gpu

NB, LO, HI = 96, -14.0, 0.0


def compare(got_prof, want_prof, got_ext, want_ext, got_hist, want_hist):
    for key, w in want_prof.items():
        g = got_prof[key]
        scale = max(np.max(np.abs(w)), 1e-300)
        assert np.max(np.abs(g - w)) <= 1e-12 * scale, (key, np.max(np.abs(g - w)) / scale)
    m = {"lambda_top": "lambda_t", "lambda_top_slope": "lambda_t_slope"}
    for key, g in got_ext.items():
        w = want_ext[m.get(key, key)]
        if key.startswith("lambda"):
            assert (math.isnan(g) and math.isnan(w)) or abs(g - w) <= 1e-9 * abs(w), (key, g, w)
        else:
            assert abs(g - w) <= 1e-12 * max(abs(w), 1e-300), (key, g, w)
    assert np.array_equal(got_hist, want_hist)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("kind", ["uniform", "tanh", "random"])
def test_extended_2d_matches_oracle(precision, kind):
    kw = {"uniform": {}, "tanh": {"zstretch": 2.0}, "random": {"znodes": random_planes(41, 5)}}[kind]
    cfg = O.Config(nx=100, nz=41, Ra=1e7, dt_fixed=1e-5, **kw)
    z = O.znodes(cfg)
    X = stirred_on(cfg, z, seed=3, u_amp=0.2)
    if precision == "fp32":
        X = X.astype(np.float32).astype(np.float64)
    s = solver_for(cfg, precision)
    try:
        s.set_state(X)
        if precision == "fp32":  # the state the kernels see is exactly X
            assert np.array_equal(s.state(), X)
        prof = s.ext_profiles()
        ext, hist = s.extended(NB, LO, HI)
    finally:
        s.close()
    want_ext, want_hist = O.extended(cfg, X, NB, LO, HI)
    compare(prof, O.ext_profiles(cfg, X), ext, want_ext, hist, want_hist)


@pytest.mark.parametrize("kind", ["uniform", "tanh"])
def test_extended_3d_matches_oracle(kind):
    kw = {"uniform": {}, "tanh": {"zstretch": 1.5}}[kind]
    cfg = O.Config(nx=36, ny=20, nz=17, ndim=3, Ra=1e6, dt_fixed=1e-5, **kw)
    X = stirred_3d_on(cfg, O.znodes(cfg), seed=9, u_amp=0.2)
    s = solver3_for(cfg, "fp64")
    try:
        s.set_state(X)
        prof = s.ext_profiles()
        ext, hist = s.extended(NB, LO, HI)
    finally:
        s.close()
    want_ext, want_hist = O.extended(cfg, X, NB, LO, HI)
    compare(prof, O.ext_profiles(cfg, X), ext, want_ext, hist, want_hist)


def test_conduction_state_has_no_flow_terms():
    """At rest: F_n = F_v = 0 exactly, every node at r = 0 (bin 0), C undefined
    (0/0); T_sa = -eps z is linear, so the tangent construction gives 1/2."""
    cfg = O.Config(nx=64, nz=33, Ra=1e6, pert_amp=0.0)
    s = solver_for(cfg)
    try:
        prof = s.ext_profiles()
        ext, hist = s.extended(NB, LO, HI)
    finally:
        s.close()
    assert np.all(prof["F_n"] == 0) and np.all(prof["F_v"] == 0)
    assert math.isnan(ext["C"]) and ext["r_max"] == 0.0
    assert abs(ext["lambda_b"] - 0.5) < 1e-9 and abs(ext["lambda_top"] - 0.5) < 1e-9
    assert hist[0] == cfg.nx * cfg.nz and hist[1:].sum() == 0


def test_full_size_extended_fp32():
    """The 4096 x 1024, Ra = 1e10 FP32 workload after 300 steps: every
    extended quantity and the histogram against the oracle on the same state."""
    import paper_2411_10372_gb300 as cm
    cfg = O.Config(nx=4096, nz=1024, Ra=1e10)
    s = cm.Solver(cfg.nx, cfg.nz, cfg.Ra, precision="fp32")
    try:
        s.step(300)
        X = s.state()
        prof = s.ext_profiles()
        ext, hist = s.extended(NB, LO, HI)
    finally:
        s.close()
    want_ext, want_hist = O.extended(cfg, X, NB, LO, HI)
    compare(prof, O.ext_profiles(cfg, X), ext, want_ext, hist, want_hist)
    assert hist.sum() == cfg.nx * cfg.nz
