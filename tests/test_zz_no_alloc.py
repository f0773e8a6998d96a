"""cm_diag_noalloc: diagnostics for callers that must not allocate device memory.

Such callers are analysis hooks embedded in another application's time loop:
the host's memory pool owns the device memory, so a cudaMalloc there could
fail or synchronise the device under the host's own streams.  The entry point
uses only a fixed scratch array inside libcm.so.  Here it is called through
the C ABI on the solver's own state and must reproduce the record of the
context entry point (cm_sample + cm_diagnostics) within the diagnostics
tolerance of the parity tests (1e-12 relative), on two calls in a row, for
FP64 and FP32 states on uniform and stretched z-grids.  This file is
collected last on purpose.
"""
import ctypes

import pytest

pytestmark = pytest.mark.gpu

KEYS = ("Nu", "Nu_conv", "Nu_K", "Nu_bot", "Nu_top", "Nu_bar", "Re", "KE", "mass", "energy", "mach_max", "t", "dt")


def _close(a, b, tol=1e-12):
    return abs(a - b) <= tol * max(abs(b), 1.0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("zgrid", ["uniform", "tanh", "given"])
def test_noalloc_diagnostics_match_context_entry_point(precision, zgrid):
    """Uniform planes, the tanh grid (beta = 2) and given planes: on the
    stretched grids the plate Nusselt numbers and the volume averages use the
    plane table copied into the scratch array."""
    import numpy as np
    import paper_2411_10372_gb300 as cm
    code = cm.CM_FP64 if precision == "fp64" else cm.CM_FP32
    Ra, Pr, gamma = 1e6, 1.0, 5.0 / 3.0
    z = np.linspace(0.0, 1.0, 64)
    z = z - 0.5 * np.sin(2 * np.pi * z) / (2 * np.pi)
    z[0], z[-1] = 0.0, 1.0
    kw = {"uniform": {}, "tanh": {"zstretch": 2.0}, "given": {"znodes": z}}[zgrid]
    s = cm.Solver(256, 64, Ra, Pr, gamma, precision=precision, **kw)
    grid = s.grid
    if zgrid == "given":  # the solver's grid drops znodes after cm_init
        grid = cm.cm_grid(2, 256, 1, 64, s.grid.aspect, 0.0, z.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    try:
        for n_more in (40, 7):  # two states: the second call sees the first call's scratch
            s.step(n_more)
            pitch, nf, elem = cm.cm_state_layout()
            t, steps = cm.cm_get_time()
            dt = cm.cm_get_dt()
            ref = s.sample()
            for _ in range(2):  # two calls in a row on the same state
                got = cm.cm_diag_noalloc(cm.cm_state_ptr(0), code, grid, pitch, Ra, Pr, gamma, s.params,
                                         t, dt, steps)
                assert got["status"] == 0 and got["step"] == ref["step"] == steps
                for k in KEYS:
                    assert _close(got[k], ref[k]), (k, got[k], ref[k])
    finally:
        s.close()


@pytest.mark.parametrize("zgrid", ["uniform", "tanh"])
def test_noalloc_on_a_3d_state(zgrid):
    """A 3D state (5 fields, ny rows per plane) gives the record of cm_sample."""
    import paper_2411_10372_gb300 as cm
    Ra, Pr, gamma = 1e6, 1.0, 5.0 / 3.0
    s = cm.Solver(40, 17, Ra, Pr, gamma, ny=24, ndim=3, precision="fp32", pert_amp=1e-2,
                  zstretch=2.0 if zgrid == "tanh" else 0.0)
    try:
        s.step(6)
        pitch, nf, elem = cm.cm_state_layout()
        assert nf == 5
        t, steps = cm.cm_get_time()
        dt = cm.cm_get_dt()
        ref = s.sample()
        for _ in range(2):
            got = cm.cm_diag_noalloc(cm.cm_state_ptr(0), cm.CM_FP32, s.grid, pitch, Ra, Pr, gamma, s.params, t, dt,
                                     steps)
            for k in KEYS:
                assert _close(got[k], ref[k]), (k, got[k], ref[k])
    finally:
        s.close()


def test_noalloc_takes_no_device_memory():
    """After a first call (which loads the module holding the scratch array),
    further calls leave the device's free memory exactly as it was."""
    torch = pytest.importorskip("torch")
    import paper_2411_10372_gb300 as cm
    Ra, Pr, gamma = 1e6, 1.0, 5.0 / 3.0
    s = cm.Solver(256, 64, Ra, Pr, gamma, precision="fp64", zstretch=2.0)
    try:
        s.step(5)
        pitch, _, _ = cm.cm_state_layout()
        t, steps = cm.cm_get_time()
        dt = cm.cm_get_dt()
        args = (cm.cm_state_ptr(0), cm.CM_FP64, s.grid, pitch, Ra, Pr, gamma, s.params, t, dt, steps)
        first = cm.cm_diag_noalloc(*args)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(5):
            got = cm.cm_diag_noalloc(*args)
            assert got["Nu_bar"] == first["Nu_bar"]
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
    finally:
        s.close()


def test_noalloc_rejects_grid_beyond_scratch():
    import paper_2411_10372_gb300 as cm
    g = cm.cm_grid(2, 64, 1, 16385, 4.0)
    p = cm.cm_default_params()
    with pytest.raises(cm.CMError) as e:
        cm.cm_diag_noalloc(1 << 20, cm.CM_FP32, g, 64, 1e6, 1.0, 5.0 / 3.0, p)
    assert e.value.code == cm.CM_EINVAL and "16384" in str(e.value)
