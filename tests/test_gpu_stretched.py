"""Parity of the CUDA path with the FP64 oracle on stretched z-grids (the tanh
grid of Sec. 3 and seeded uneven planes), through the C ABI.

Bars: FP64 single sweeps <= 1e-13 relative L2 per field, FP64 steps <= 1e-12
after 200 steps, diagnostics <= 1e-12; FP32 as on the uniform grid (single
sweeps 2e-6, 100 steps 1e-5, momentum against rho c).  Inputs are seeded and
synthetic; the plane heights are inputs given to both sides (or beta, from
which each side computes its own tanh planes).
"""
import math

import numpy as np
import pytest

import oracle as O
from physics import closures
from test_gpu_parity import rel_l2
from test_oracle_pins import random_planes, stirred_on

pytestmark = pytest.mark.gpu


def solver_for(cfg: O.Config, precision="fp64", **extra):
    import paper_2411_10372_gb300 as cm
    t_top = (1.0 - cfg.eps - cfg.D) if cfg.t_top is None else cfg.t_top
    return cm.Solver(cfg.nx, cfg.nz, cfg.Ra, cfg.Pr, cfg.gamma, aspect=cfg.aspect, precision=precision,
                     eps=cfg.eps, D=cfg.D, cfl=cfg.cfl, dt_fixed=cfg.dt_fixed, gravity=cfg.gravity,
                     t_bot=cfg.t_bot, t_top=t_top, pert_amp=cfg.pert_amp, stokes=cfg.stokes, seed=cfg.seed,
                     tvd_form=cfg.tvd_form, zstretch=cfg.zstretch, znodes=cfg.znodes, **extra)


GRIDS = [("tanh2", dict(zstretch=2.0)), ("tanh1", dict(zstretch=1.0)), ("random", "random")]
SHAPES = [(8, 9), (29, 17), (64, 33), (100, 41), (256, 65)]


def cfg_for(nx, nz, grid, **kw):
    if grid == "random":
        return O.Config(nx=nx, nz=nz, znodes=random_planes(nz, seed=nx + nz), **kw)
    return O.Config(nx=nx, nz=nz, **grid, **kw)


@pytest.mark.parametrize("nx,nz", SHAPES)
@pytest.mark.parametrize("name,grid", GRIDS, ids=[g[0] for g in GRIDS])
def test_planes_match_oracle(nx, nz, name, grid):
    cfg = cfg_for(nx, nz, grid)
    s = solver_for(cfg)
    z = s.z
    want = O.znodes(cfg)
    if cfg.znodes is not None:
        assert np.array_equal(z, want)
    else:
        assert np.max(np.abs(z - want)) <= 2e-16
    s.close()


@pytest.mark.parametrize("nx,nz", SHAPES)
@pytest.mark.parametrize("name,grid", GRIDS, ids=[g[0] for g in GRIDS])
@pytest.mark.parametrize("tvd", [O.TVD_SPLIT, O.TVD_SUM, O.TVD_OFF])
def test_single_sweeps_fp64(nx, nz, name, grid, tvd):
    """One L_z and one L_x on a stirred state, every node, FP64."""
    cfg = cfg_for(nx, nz, grid, Ra=1e5, tvd_form=tvd, dt_fixed=1e-5)
    z = O.znodes(cfg)
    X = stirred_on(cfg, z, seed=nx * 31 + nz)
    s = solver_for(cfg)
    for direction in (2, 0):
        Delta = 0.2 * min(cfg.aspect / nx, float(np.min(np.diff(z)))) / 4.0
        s.set_state(X)
        s.sweep(direction, Delta)
        got = s.state()
        want = O.sweep(cfg, X, direction, Delta)
        for f in range(4):
            assert rel_l2(got[f], want[f]) <= 1e-13, (direction, f, rel_l2(got[f], want[f]))
    s.close()


@pytest.mark.parametrize("nx,nz", [(30, 17), (64, 33), (250, 65), (122, 41), (29, 17), (57, 33)])
@pytest.mark.parametrize("name,grid", GRIDS, ids=[g[0] for g in GRIDS])
def test_single_sweeps_fp32(nx, nz, name, grid):
    """FP32 sweeps on a stirred state rounded to FP32, against the oracle on
    the same rounded input: packed two-column kernels for even nx, the
    one-column kernels for odd nx."""
    cfg = cfg_for(nx, nz, grid, Ra=1e5, dt_fixed=1e-5)
    z = O.znodes(cfg)
    X = stirred_on(cfg, z, seed=nx * 7 + nz).astype(np.float32).astype(np.float64)
    s = solver_for(cfg, "fp32")
    for direction in (2, 0):
        Delta = 0.2 * min(cfg.aspect / nx, float(np.min(np.diff(z)))) / 4.0
        s.set_state(X)
        s.sweep(direction, Delta)
        got = s.state()
        want = O.sweep(cfg, X, direction, Delta)
        for f in (0, 3):
            assert rel_l2(got[f], want[f]) <= 2e-6, (direction, f, rel_l2(got[f], want[f]))
        scale = np.linalg.norm(want[0]) * 3.65
        for f in (1, 2):
            assert np.linalg.norm(got[f] - want[f]) / scale <= 2e-6, (direction, f)
    s.close()


@pytest.mark.parametrize("name,grid", GRIDS, ids=[g[0] for g in GRIDS])
def test_fp64_steps_match_oracle(name, grid):
    """200 FP64 steps of the 256 x 65, Ra = 1e6 configuration on a stretched
    grid from the seeded initial state: state, time and dt sequence."""
    cfg = cfg_for(256, 65, grid, Ra=1e6)
    s = solver_for(cfg, diag_every=50)
    assert np.array_equal(s.state(), O.init(cfg))
    X0 = O.init(cfg)
    assert abs(s.dt() - O.dt(cfg, X0)) <= 1e-15 * O.dt(cfg, X0)
    s.step(200)
    t_gpu, steps = s.time()
    got = s.state()
    want, t_cpu, _ = O.step(cfg, X0, 200)
    assert steps == 200 and abs(t_gpu - t_cpu) <= 1e-13 * t_cpu
    for f in range(4):
        assert rel_l2(got[f], want[f]) <= 1e-12, (f, rel_l2(got[f], want[f]))
    d_gpu = s.diagnostics()[-1]
    d_cpu = O.diag(cfg, want)
    for key in ("Nu", "Nu_conv", "Nu_K", "Nu_bot", "Nu_top", "Nu_bar", "Re", "KE", "mass", "energy"):
        assert abs(d_gpu[key] - d_cpu[key]) <= 1e-10 * max(abs(d_cpu[key]), 1e-6), key
    # trapezoid mass on the planes is conserved
    z = O.znodes(cfg)
    m0 = np.trapezoid(X0[0].mean(axis=1), z)
    assert abs(np.trapezoid(got[0].mean(axis=1), z) - m0) <= 1e-13 * m0
    s.close()


@pytest.mark.parametrize("name,grid", GRIDS, ids=[g[0] for g in GRIDS])
def test_fp32_steps(name, grid):
    cfg = cfg_for(256, 65, grid, Ra=1e6)
    s = solver_for(cfg, "fp32")
    s.step(100)
    got = s.state()
    want, _, _ = O.step(cfg, O.init(cfg), 100)
    cl = closures(cfg.gamma, cfg.eps, cfg.D, cfg.Ra, cfg.Pr)
    assert rel_l2(got[0], want[0]) <= 1e-5
    assert rel_l2(got[3], want[3]) <= 1e-5
    scale = np.linalg.norm(want[0] * math.sqrt(cfg.gamma * cl["a"]))
    for f in (1, 2):
        assert np.linalg.norm(got[f] - want[f]) / scale <= 1e-5, f
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_diagnostics_and_dt_on_same_state(precision):
    """Trapezoid weights w_k and the plate quadratic on uneven planes; dt from
    the smaller spacing next to each plane."""
    cfg = cfg_for(128, 33, dict(zstretch=2.5), Ra=1e7)
    z = O.znodes(cfg)
    X = stirred_on(cfg, z, seed=5, u_amp=0.1)
    if precision == "fp32":
        X = X.astype(np.float32).astype(np.float64)
    s = solver_for(cfg, precision)
    s.set_state(X)
    d = s.sample()
    want = O.diag(cfg, X)
    tol = 1e-12 if precision == "fp64" else 2e-6
    for key in ("Nu", "Nu_conv", "Nu_K", "Re", "KE", "mass", "energy"):
        assert abs(d[key] - want[key]) <= tol * max(abs(want[key]), 1.0), key
    # plate Nusselt numbers: the rounding of a plane mean of T (unit u: 2e-14
    # in FP64 sums of FP64 T, 2e-7 for FP32 T) enters amplified by the sum of
    # the three-plane derivative coefficients over eps (~16000 here: the
    # first spacing is 0.0025)
    u = 2e-14 if precision == "fp64" else 2e-7
    for key, (a, b, c) in (("Nu_bot", (z[0], z[1], z[2])), ("Nu_top", (z[-1], z[-2], z[-3]))):
        h1, h2 = abs(b - a), abs(c - b)
        amp = ((2 * h1 + h2) / (h1 * (h1 + h2)) + (h1 + h2) / (h1 * h2) + h1 / (h2 * (h1 + h2))) / cfg.eps
        assert abs(d[key] - want[key]) <= u * amp, (key, d[key] - want[key], u * amp)
    dt_tol = 1e-15 if precision == "fp64" else 1e-6
    assert abs(s.dt() - O.dt(cfg, X)) <= dt_tol * O.dt(cfg, X)
    s.close()


def test_uniform_grid_path_unchanged_by_explicit_uniform_planes():
    """Planes given as k/K run the stretched kernels; they agree with the
    uniform kernels to rounding of the spacings."""
    cfg_u = O.Config(nx=128, nz=33, Ra=1e6)
    cfg_s = O.Config(nx=128, nz=33, Ra=1e6, znodes=np.arange(33) / 32.0)
    out = []
    for cfg in (cfg_u, cfg_s):
        s = solver_for(cfg)
        s.step(50)
        out.append(s.state())
        s.close()
    for f in range(4):
        assert rel_l2(out[1][f], out[0][f]) <= 1e-12, f


def test_full_size_one_step_fp64_and_fp32():
    """The 4096 x 1024, Ra = 1e10 workload on the tanh grid (beta = 2) in the
    bench's launch configuration: one full step on every node against the
    oracle, and the trapezoid mass on the planes."""
    cfg = O.Config(nx=4096, nz=1024, Ra=1e10, zstretch=2.0)
    X0 = O.init(cfg)
    want, _, _ = O.step(cfg, X0, 1)
    z = O.znodes(cfg)
    m0 = np.trapezoid(X0[0].mean(axis=1), z)
    for precision, tol in (("fp64", 1e-13), ("fp32", 2e-6)):
        s = solver_for(cfg, precision)
        s.step(1)
        got = s.state()
        for f in (0, 3):
            assert rel_l2(got[f], want[f]) <= tol, (precision, f)
        scale = np.linalg.norm(want[0]) * 3.65
        for f in (1, 2):
            assert np.linalg.norm(got[f] - want[f]) / scale <= tol, (precision, f)
        mass_tol = 1e-14 if precision == "fp64" else 1e-6
        assert abs(np.trapezoid(got[0].mean(axis=1), z) - m0) <= mass_tol * m0, precision
        s.close()


# ---- 3D on stretched planes ----

def stirred_3d_on(cfg, z, seed, u_amp=0.3, t_amp=0.05):
    """3D conduction profile on the planes z with random temperature, density
    and velocity fields (velocity zero on the plates)."""
    from physics import state_from_prims
    rng = np.random.default_rng(seed)
    T_c, p_c, _ = O.profile(cfg)
    shp = (cfg.nz, cfg.ny, cfg.nx)
    Z = np.broadcast_to(np.asarray(z)[:, None, None], shp)
    T = T_c[:, None, None] * (1 + t_amp * rng.uniform(-1, 1, shp))
    u = [u_amp * rng.uniform(-1, 1, shp) for _ in range(3)]
    for f in u:
        f[0] = f[-1] = 0.0
    T[0], T[-1] = cfg.t_bot, 1.0 - cfg.eps - cfg.D
    cl = closures(cfg.gamma, cfg.eps, cfg.D, cfg.Ra, cfg.Pr)
    rho = p_c[:, None, None] / (cl["a"] * T) * (1 + 0.02 * rng.uniform(-1, 1, shp))
    return state_from_prims(cfg, rho, u[0], u[2], T, Z, uy=u[1])


def solver3_for(cfg, precision="fp64", **extra):
    import paper_2411_10372_gb300 as cm
    return cm.Solver(cfg.nx, cfg.nz, cfg.Ra, cfg.Pr, cfg.gamma, ny=cfg.ny, ndim=3, aspect=cfg.aspect,
                     precision=precision, eps=cfg.eps, D=cfg.D, cfl=cfg.cfl, dt_fixed=cfg.dt_fixed,
                     t_top=1.0 - cfg.eps - cfg.D, pert_amp=cfg.pert_amp, seed=cfg.seed, tvd_form=cfg.tvd_form,
                     zstretch=cfg.zstretch, znodes=cfg.znodes, **extra)


def check3(cfg, got, want, tol):
    for f in (0, 4):
        assert rel_l2(got[f], want[f]) <= tol, (f, rel_l2(got[f], want[f]))
    cl = closures(cfg.gamma, cfg.eps, cfg.D, cfg.Ra, cfg.Pr)
    scale = np.linalg.norm(want[0]) * math.sqrt(cfg.gamma * cl["a"])
    for f in (1, 2, 3):
        assert np.linalg.norm(got[f] - want[f]) / scale <= tol, f


SHAPES3 = [(8, 4, 9), (29, 13, 17), (36, 20, 13)]


def cfg3_for(nx, ny, nz, grid, **kw):
    if grid == "random":
        return O.Config(nx=nx, ny=ny, nz=nz, ndim=3, znodes=random_planes(nz, seed=nx + ny + nz), **kw)
    return O.Config(nx=nx, ny=ny, nz=nz, ndim=3, **grid, **kw)


@pytest.mark.parametrize("nx,ny,nz", SHAPES3)
@pytest.mark.parametrize("name,grid", GRIDS, ids=[g[0] for g in GRIDS])
def test_single_sweeps_3d(nx, ny, nz, name, grid):
    """L_z, L_y, L_x on a stirred 3D state on stretched planes: FP64 <= 1e-13,
    FP32 (same state rounded) <= 2e-6."""
    cfg = cfg3_for(nx, ny, nz, grid, Ra=1e5, dt_fixed=1e-5)
    z = O.znodes(cfg)
    X = stirred_3d_on(cfg, z, seed=nx * 100 + ny + nz)
    for precision, tol in (("fp64", 1e-13), ("fp32", 2e-6)):
        Xp = X if precision == "fp64" else X.astype(np.float32).astype(np.float64)
        s = solver3_for(cfg, precision)
        try:
            for direction in (2, 1, 0):
                Delta = 0.2 * min(cfg.aspect / nx, cfg.aspect / ny, float(np.min(np.diff(z)))) / 4.0
                s.set_state(Xp)
                s.sweep(direction, Delta)
                check3(cfg, s.state(), O.sweep(cfg, Xp, direction, Delta), tol)
        finally:
            s.close()


@pytest.mark.parametrize("name,grid", GRIDS, ids=[g[0] for g in GRIDS])
def test_steps_3d(name, grid):
    """30 full 3D steps from the seeded initial state on stretched planes:
    FP64 <= 1e-12 with time and mass; FP32 <= 1e-5."""
    cfg = cfg3_for(36, 20, 17, grid, Ra=1e6, pert_amp=0.02)
    X0 = O.init(cfg)
    want, t_cpu, _ = O.step(cfg, X0, 30)
    z = O.znodes(cfg)
    for precision, tol in (("fp64", 1e-12), ("fp32", 1e-5)):
        s = solver3_for(cfg, precision)
        try:
            s.step(30)
            t_gpu, steps = s.time()
            got = s.state()
            assert steps == 30 and abs(t_gpu - t_cpu) <= (1e-13 if precision == "fp64" else 1e-6) * t_cpu
            check3(cfg, got, want, tol)
            if precision == "fp64":
                m0 = np.trapezoid(X0[0].mean(axis=(1, 2)), z)
                assert abs(np.trapezoid(got[0].mean(axis=(1, 2)), z) - m0) <= 1e-13 * m0
                d = s.sample()
                dw = O.diag(cfg, got)
                for key in ("Nu", "Nu_bar", "Re", "KE", "mass", "energy"):
                    assert abs(d[key] - dw[key]) <= 1e-10 * max(abs(dw[key]), 1e-6), key
        finally:
            s.close()


@pytest.mark.parametrize("name,grid", GRIDS, ids=[g[0] for g in GRIDS])
def test_packed_3d_agrees_with_the_scalar_kernels_on_stretched_planes(monkeypatch, name, grid):
    """The packed FP32 3D kernels (even nx) and the one-column FP32 kernels
    (CM_3D_SCALAR) on the same stirred state on stretched planes: 6 full
    steps, the dt reductions included, agree within the FP32 bar; the packed
    kernels' plane caches hold the planes of segments of 32 rows (forced, so
    that segments start and end inside the grid)."""
    cfg = cfg3_for(122, 26, 71, grid, Ra=1e6)
    z = O.znodes(cfg)
    X = stirred_3d_on(cfg, z, seed=5, u_amp=0.1).astype(np.float32).astype(np.float64)
    out = {}
    for mode in ("packed", "scalar"):
        monkeypatch.setenv("CM_SEG_ROWS", "32")
        if mode == "scalar":
            monkeypatch.setenv("CM_3D_SCALAR", "1")
        s = solver3_for(cfg, "fp32")
        try:
            s.set_state(X)
            s.step(6)
            out[mode] = (s.state(), s.dt())
        finally:
            s.close()
    check3(cfg, out["packed"][0], out["scalar"][0], 1e-5)
    assert abs(out["packed"][1] - out["scalar"][1]) <= 1e-6 * out["scalar"][1]


def test_full_size_3d_fp32_genuinely_3d_step_on_tanh_planes():
    """The 512 x 512 x 128 FP32 box on the beta = 2 tanh grid in the
    benchmark's launch shape (segment lengths tuned at init, packed kernels
    with the blocks' plane caches) on a stirred, genuinely 3D state: one full
    step against the FP64 oracle node by node, within 1e-5 of each field's
    largest value (momenta: of rho c), the bar of the uniform full-size test."""
    import contextlib
    nx, ny, nz = 512, 512, 128
    cfg = O.Config(nx=nx, ny=ny, nz=nz, ndim=3, Ra=1e9, dt_fixed=1e-4, zstretch=2.0)
    z = O.znodes(cfg)
    X = stirred_3d_on(cfg, z, seed=321, u_amp=0.05).astype(np.float32).astype(np.float64)
    s = solver3_for(cfg, "fp32")
    try:
        s.set_state(X)
        s.step(1)
        got = s.state()
    finally:
        s.close()
    path = O.build_omp()
    with (O.library(path) if path else contextlib.nullcontext()):
        want, _, _ = O.step(cfg, X, 1)
    cl = closures(cfg.gamma, cfg.eps, cfg.D, cfg.Ra, cfg.Pr)
    rc = np.max(np.abs(want[0])) * math.sqrt(cfg.gamma * cl["a"])
    errs = []
    for f in range(5):
        scale = rc if f in (1, 2, 3) else np.max(np.abs(want[f]))
        errs.append(float(np.max(np.abs(got[f] - want[f]))) / scale)
    print("full-size 3D step on tanh planes, largest node difference per field / field scale:", errs)
    assert max(errs) <= 1e-5, errs


def test_full_size_3d_fp32_y_invariant_matches_2d_oracle():
    """The 512 x 512 x 128 FP32 box on the tanh grid (beta = 2) in the launch
    configuration the benchmark times, on y-independent data: 3 steps, y
    planes against the 2D stretched oracle (FP32 bar), every y plane equal,
    m_y exactly zero, trapezoid mass on the planes kept."""
    import paper_2411_10372_gb300 as cm
    nx, ny, nz = 512, 512, 128
    c2 = O.Config(nx=nx, nz=nz, Ra=1e7, seed=31, pert_amp=1e-2, zstretch=2.0)
    X2 = O.init(c2).astype(np.float32).astype(np.float64)
    X3 = np.zeros((5, nz, ny, nx))
    for f, g in ((0, 0), (1, 1), (3, 2), (4, 3)):
        X3[f] = X2[g][:, None, :]
    s = cm.Solver(nx, nz, 1e7, 1.0, 5.0 / 3.0, ny=ny, ndim=3, precision="fp32", pert_amp=1e-2, seed=31,
                  zstretch=2.0)
    try:
        s.set_state(X3)
        s.step(3)
        got = s.state()
    finally:
        s.close()
    want, _, _ = O.step(c2, X2, 3)
    assert np.all(got[2] == 0)
    assert np.max(np.abs(got - got[:, :, :1, :])) == 0.0
    c3 = O.Config(nx=nx, ny=1, nz=nz, ndim=3, Ra=1e7)
    w3 = np.stack([want[0], want[1], np.zeros_like(want[0]), want[2], want[3]])[:, :, None, :]
    check3(c3, got[:, :, :1, :], w3, 1e-5)
    z = O.znodes(c2)
    m0 = np.trapezoid(X3[0].mean(axis=(1, 2)), z)
    assert abs(np.trapezoid(got[0].mean(axis=(1, 2)), z) - m0) <= 1e-6 * m0


def test_checkpoint_carries_the_planes(tmp_path):
    """cm_save / cm_load: the checkpoint's parameter hash covers the plane
    heights of a stretched grid; a context on other planes (or uniform ones)
    refuses it, one on the same planes restores the state bit for bit."""
    import paper_2411_10372_gb300 as cm
    cfg = O.Config(nx=64, nz=17, Ra=1e6, zstretch=1.5)
    s = solver_for(cfg)
    s.step(3)
    X = s.state()
    path = str(tmp_path / "st.ckpt")
    cm.cm_save(path)
    s.close()
    for other in (O.Config(nx=64, nz=17, Ra=1e6), O.Config(nx=64, nz=17, Ra=1e6, zstretch=1.6)):
        s = solver_for(other)
        with pytest.raises(cm.CMError) as e:
            cm.cm_load(path)
        assert e.value.code == cm.CM_EBADCKPT
        s.close()
    s = solver_for(cfg)
    cm.cm_load(path)
    assert np.array_equal(s.state(), X)
    s.close()
