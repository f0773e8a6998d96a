"""The library's adjoint (cm_adj_forward / cm_adj_backward, FP64 2D) against
torch.autograd on oracle/torch_ref.py, whose states and gradients are pinned
to the C oracle (tests/test_torch_ref_pins.py).

Bars: J equal within 1e-12 (the GPU forward is the oracle's arithmetic); the
gradients dJ/dX^0 (relative L2 per field), dJ/dT0 and dJ/dRa within 1e-9
(reverse mode in a different association order; the flow's sensitivity
magnifies rounding by a few orders over the run).  Gradients do not depend
on the checkpoint interval (bit for bit: the recomputed segments are
bit-identical; also when every sweep input is kept instead).  At the full
1024 x 256 size a directional derivative
matches central finite differences of the GPU forward.  The same holds on
stretched z-grids (the tanh grid and given planes), where the reverse stages
use the conservative form's per-plane spans and weights.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from oracle.torch_ref import Model, isobaric_state

pytestmark = pytest.mark.gpu


def _stretched(cfg):
    return cfg.zstretch != 0.0 or cfg.znodes is not None


def _model(cfg, frozen=False):
    return Model(cfg.nx, cfg.nz, Pr=cfg.Pr, gamma=cfg.gamma, eps=cfg.eps, D=cfg.D, aspect=cfg.aspect,
                 gravity=cfg.gravity, t_bot=cfg.t_bot, t_top=cfg.t_top, stokes=cfg.stokes, tvd_form=cfg.tvd_form,
                 znodes=O.znodes(cfg) if _stretched(cfg) else None, frozen_phi=frozen)


def _given_planes(nz):
    s = np.linspace(0.0, 1.0, nz)
    z = s - 0.6 * np.sin(2 * np.pi * s) / (2 * np.pi)
    z[0], z[-1] = 0.0, 1.0
    return z


def _solver(cfg, limiter=0):
    import paper_2411_10372_gb300 as cm
    t_top = (1.0 - cfg.eps - cfg.D) if cfg.t_top is None else cfg.t_top
    return cm.Solver(cfg.nx, cfg.nz, cfg.Ra, cfg.Pr, cfg.gamma, aspect=cfg.aspect, precision="fp64", eps=cfg.eps,
                     D=cfg.D, cfl=cfg.cfl, dt_fixed=cfg.dt_fixed, gravity=cfg.gravity, t_bot=cfg.t_bot,
                     t_top=t_top, pert_amp=cfg.pert_amp, stokes=cfg.stokes, seed=cfg.seed, tvd_form=cfg.tvd_form,
                     zstretch=cfg.zstretch, znodes=cfg.znodes, adj_limiter=limiter)


def _gpu_gradients(cfg, nsteps, K, win, X0=None, limiter=0):
    import paper_2411_10372_gb300 as cm
    s = _solver(cfg, limiter)
    try:
        if X0 is not None:
            s.set_state(X0)
        J = cm.cm_adj_forward(nsteps, K, win)
        gX = np.empty((4, cfg.nz, cfg.nx))
        gT = np.empty((cfg.nz, cfg.nx))
        gRa = cm.cm_adj_backward(gX, gT)
    finally:
        s.close()
    return J, gX, gT, gRa


def _torch_gradients(cfg, X0, nsteps, win, frozen=False):
    """J and its gradients by autograd, with the oracle's CFL dts (which the
    FP64 GPU forward reproduces bit for bit)."""
    X, dts = X0, []
    for _ in range(nsteps):
        X, _, d = O.step(cfg, X, 1)
        dts.append(float(d[0]))
    m = _model(cfg, frozen)
    rho = X0[0]
    ux, uz = X0[1] / rho, X0[2] / rho
    z = m.z.numpy()
    T0 = m.b * (X0[3] / rho - 0.5 * (ux * ux + uz * uz) - m.g * z)
    P0 = m.a * rho * T0
    X0t = torch.tensor(X0, requires_grad=True)
    Ra = torch.tensor(cfg.Ra, dtype=torch.float64, requires_grad=True)
    J = m.objective(X0t, Ra, dts, win)
    gX, gRa = torch.autograd.grad(J, [X0t, Ra])
    T0t = torch.tensor(T0, requires_grad=True)
    Xi = isobaric_state(m, T0t, torch.from_numpy(P0), torch.from_numpy(ux), torch.from_numpy(uz))
    gT, = torch.autograd.grad(m.objective(Xi, cfg.Ra, dts, win), [T0t])
    gT = gT.numpy().copy()
    gT[0] = gT[-1] = 0.0
    return float(J.detach()), gX.numpy(), gT, float(gRa)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("tvd,zgrid", [(O.TVD_SPLIT, "uniform"), (O.TVD_SUM, "uniform"), (O.TVD_OFF, "uniform"),
                                       (O.TVD_SPLIT, "tanh"), (O.TVD_SUM, "given"), (O.TVD_OFF, "tanh")])
def test_adjoint_matches_autograd(tvd, zgrid):
    kw = {"uniform": {}, "tanh": {"zstretch": 1.5}, "given": {"znodes": _given_planes(9)}}[zgrid]
    cfg = O.Config(nx=32, nz=9, Ra=3e5, seed=21, pert_amp=3e-2, tvd_form=tvd, **kw)
    nsteps, K, win = 30, 7, 21
    X0 = O.init(cfg)
    J, gX, gT, gRa = _gpu_gradients(cfg, nsteps, K, win)
    Jt, gXt, gTt, gRat = _torch_gradients(cfg, X0, nsteps, win)
    assert abs(J - Jt) <= 1e-12 * abs(Jt)
    for f in range(4):
        assert _rel(gX[f], gXt[f]) <= 1e-9, (f, _rel(gX[f], gXt[f]))
    assert _rel(gT, gTt) <= 1e-9
    assert np.all(gT[0] == 0) and np.all(gT[-1] == 0)
    assert abs(gRa - gRat) <= 1e-9 * abs(gRat)


@pytest.mark.parametrize("beta", [0.0, 1.5])
def test_adjoint_on_a_stirred_state(beta):
    """Every branch of the scheme active: random velocities, odd sizes, x-sweep
    TVD at both signs of the ratios; uniform and tanh z-grids."""
    from test_gpu_parity import stirred_state
    cfg = O.Config(nx=29, nz=11, Ra=1e5, seed=4, zstretch=beta)
    X0 = stirred_state(cfg, seed=8, u_amp=0.2, t_amp=0.03)
    nsteps, K, win = 12, 5, 1
    J, gX, gT, gRa = _gpu_gradients(cfg, nsteps, K, win, X0)
    Jt, gXt, gTt, gRat = _torch_gradients(cfg, X0, nsteps, win)
    assert abs(J - Jt) <= 1e-12 * abs(Jt)
    for f in range(4):
        assert _rel(gX[f], gXt[f]) <= 1e-9, (f, _rel(gX[f], gXt[f]))
    assert abs(gRa - gRat) <= 1e-9 * abs(gRat)


@pytest.mark.parametrize("beta", [0.0, 1.5])
def test_gradients_do_not_depend_on_checkpoint_interval(beta):
    cfg = O.Config(nx=40, nz=13, Ra=1e6, seed=2, pert_amp=2e-2, zstretch=beta)
    ref = None
    for K in (1, 6, 25, 0):  # 0: every sweep input kept, nothing recomputed
        J, gX, gT, gRa = _gpu_gradients(cfg, 25, K, 11)
        if ref is None:
            ref = (J, gX, gT, gRa)
        else:
            assert J == ref[0] and gRa == ref[3]
            assert np.array_equal(gX, ref[1]) and np.array_equal(gT, ref[2])


def test_backward_can_repeat_and_rejects_misuse():
    import paper_2411_10372_gb300 as cm
    cfg = O.Config(nx=32, nz=9, Ra=1e5)
    s = _solver(cfg)
    try:
        with pytest.raises(cm.CMError):
            cm.cm_adj_backward(None, None)
        with pytest.raises(cm.CMError):
            cm.cm_adj_forward(10, 3, 11)
        with pytest.raises(cm.CMError):
            cm.cm_adj_forward(10, -1, 5)
        cm.cm_adj_forward(10, 3, 5)
        g1, g2 = cm.cm_adj_backward(None, None), cm.cm_adj_backward(None, None)
        assert g1 == g2 and g1 != 0.0
    finally:
        s.close()
    s = cm.Solver(32, 9, 1e5, precision="fp32")
    try:
        with pytest.raises(cm.CMError) as e:
            cm.cm_adj_forward(4, 2, 1)
        assert e.value.code == cm.CM_EINVAL
    finally:
        s.close()


def test_autograd_function_wraps_the_library():
    import paper_2411_10372_gb300 as cm
    from paper_2411_10372_gb300.adjoint import NuObjective
    cfg = O.Config(nx=32, nz=9, Ra=3e5, seed=21, pert_amp=3e-2)
    X0 = O.init(cfg)
    J, gX, gT, gRa = _gpu_gradients(cfg, 20, 6, 11)
    X0t = torch.tensor(X0, requires_grad=True)
    Ra = torch.tensor(cfg.Ra, dtype=torch.float64, requires_grad=True)
    Jf = NuObjective.apply(X0t, Ra, dict(nx=32, nz=9, Pr=1.0, gamma=5.0 / 3.0), 20, 6, 11)
    Jf.backward()
    assert float(Jf.detach()) == J
    assert np.array_equal(X0t.grad.numpy(), gX)
    assert float(Ra.grad) == gRa
    del cm


@pytest.mark.parametrize("tvd,tol", [(O.TVD_OFF, 1e-8), (O.TVD_SPLIT, 1e-4)])
def test_full_size_directional_derivative(tvd, tol):
    """1024 x 256, Ra = 1e8, FP64 (the adjoint workload's grid): 40 steps at a
    fixed dt, window 21..40; the adjoint's <dJ/dT0, v> against central
    differences of J from two more GPU forward runs.  Without the TVD term J
    is smooth and the difference agrees to 1e-8; with it, a difference of
    step 1e-5 crosses corners of the limiter (phi at 2r = 0 and 1, C at
    Co = 1/2) at some of the 2.6e5 nodes, which costs ~1e-5 (measured:
    1e-5 to 1e-7, not monotone in the step), hence 1e-4."""
    import paper_2411_10372_gb300 as cm
    base = O.Config(nx=1024, nz=256, Ra=1e8, seed=12345, tvd_form=tvd)
    X0 = O.init(base)
    dt = 0.8 * O.dt(base, X0)
    cfg = O.Config(nx=1024, nz=256, Ra=1e8, seed=12345, dt_fixed=dt, tvd_form=tvd)
    nsteps, K, win = 40, 10, 21
    J, gX, gT, gRa = _gpu_gradients(cfg, nsteps, K, win, X0)
    rng = np.random.default_rng(99)
    v = np.zeros((cfg.nz, cfg.nx))
    v[1:-1] = rng.uniform(-1, 1, (cfg.nz - 2, cfg.nx))
    m = _model(cfg)
    rho = X0[0]
    T0 = m.b * (X0[3] / rho - m.g * m.z.numpy())
    P0 = m.a * rho * T0
    h = 1e-5
    Js = []
    for sgn in (1.0, -1.0):
        Xs = isobaric_state(m, torch.from_numpy(T0 + sgn * h * v), torch.from_numpy(P0)).numpy()
        s = _solver(cfg)
        try:
            s.set_state(Xs)
            Js.append(cm.cm_adj_forward(nsteps, K, win))
        finally:
            s.close()
    fd = (Js[0] - Js[1]) / (2 * h)
    ad = float(np.sum(gT * v))
    assert math.isfinite(ad) and abs(ad) > 1.0
    assert abs(fd - ad) <= tol * abs(ad), (fd, ad)


@pytest.mark.parametrize("tvd,zgrid", [(O.TVD_SPLIT, "uniform"), (O.TVD_SUM, "uniform"), (O.TVD_SPLIT, "tanh")])
def test_frozen_limiter_reading_matches_autograd(tvd, zgrid):
    """CM_ADJ_PHI_FROZEN: no derivative through the limiter's ratios r; the
    same reading in the PyTorch restatement (the ratios detached)."""
    import paper_2411_10372_gb300 as cm
    kw = {"uniform": {}, "tanh": {"zstretch": 1.5}}[zgrid]
    cfg = O.Config(nx=32, nz=9, Ra=3e5, seed=21, pert_amp=3e-2, tvd_form=tvd, **kw)
    nsteps, K, win = 30, 7, 21
    X0 = O.init(cfg)
    J, gX, gT, gRa = _gpu_gradients(cfg, nsteps, K, win, limiter=cm.CM_ADJ_PHI_FROZEN)
    Jt, gXt, gTt, gRat = _torch_gradients(cfg, X0, nsteps, win, frozen=True)
    assert abs(J - Jt) <= 1e-12 * abs(Jt)
    for f in range(4):
        assert _rel(gX[f], gXt[f]) <= 1e-9, (f, _rel(gX[f], gXt[f]))
    assert _rel(gT, gTt) <= 1e-9
    assert abs(gRa - gRat) <= 1e-9 * abs(gRat)
    Je, gXe, _, _ = _gpu_gradients(cfg, nsteps, K, win)
    assert Je == J and not np.array_equal(gXe, gX)  # the two readings differ in the reverse pass only


def test_replayed_dts():
    """cm_adj_get_dts returns the CFL dts of a run; cm_adj_set_dts makes the
    next forward of that many steps take them: the same start state then gives
    the same J bit for bit, and another start state runs on those dts."""
    import paper_2411_10372_gb300 as cm
    cfg = O.Config(nx=64, nz=17, Ra=1e6, seed=5, pert_amp=1e-2)
    s = _solver(cfg)
    try:
        X0 = s.state()
        J = cm.cm_adj_forward(20, 5, 11)
        dts = cm.cm_adj_get_dts(20)
        assert np.all(dts > 0)  # constant here: the bottom plate (u = 0, T = 1) sets the CFL bound
        with pytest.raises(cm.CMError):
            cm.cm_adj_get_dts(19)
        with pytest.raises(cm.CMError):
            cm.cm_adj_set_dts([1e-3, -1.0])
        s.set_state(X0)
        cm.cm_adj_set_dts(dts * 0.5)
        Jh = cm.cm_adj_forward(20, 5, 11)
        assert np.array_equal(cm.cm_adj_get_dts(20), dts * 0.5) and Jh != J
        s.set_state(X0)
        cm.cm_adj_set_dts(dts)
        assert cm.cm_adj_forward(20, 5, 11) == J
        cm.cm_adj_set_dts(None)
        s.set_state(X0)
        assert cm.cm_adj_forward(20, 20, 11) == J  # the CFL rule again
    finally:
        s.close()


def _config5_start():
    """The adjoint workload: 1024 x 256, Ra = 1e8, FP64, seed 99, two steps in
    (as the bench takes it), and a direction v in the interior temperature."""
    import paper_2411_10372_gb300 as cm
    cfg = O.Config(nx=1024, nz=256, Ra=1e8, seed=99)
    s = _solver(cfg)
    try:
        s.step(2)
        X0 = s.state()
    finally:
        s.close()
    m = _model(cfg)
    rho = X0[0]
    ux, uz = X0[1] / rho, X0[2] / rho
    T0 = m.b * (X0[3] / rho - 0.5 * (ux * ux + uz * uz) - m.g * m.z.numpy())
    P0 = m.a * rho * T0
    v = np.zeros((cfg.nz, cfg.nx))
    v[1:-1] = np.random.default_rng(99).uniform(-1, 1, (cfg.nz - 2, cfg.nx))

    def perturbed(h):
        return isobaric_state(m, torch.from_numpy(T0 + h * v), torch.from_numpy(P0), torch.from_numpy(ux),
                              torch.from_numpy(uz)).numpy()
    return cfg, X0, v, perturbed, cm


def _replayed_J(cfg, X, dts, win, Ra=None):
    import paper_2411_10372_gb300 as cm
    c = O.Config(nx=cfg.nx, nz=cfg.nz, Ra=cfg.Ra if Ra is None else Ra, seed=cfg.seed)
    s = _solver(c)
    try:
        s.set_state(X)
        cm.cm_adj_set_dts(dts)
        return cm.cm_adj_forward(len(dts), len(dts), win)
    finally:
        s.close()


def _adjoint(cfg, X0, nsteps, K, win, limiter):
    import paper_2411_10372_gb300 as cm
    s = _solver(cfg, limiter)
    try:
        s.set_state(X0)
        J = cm.cm_adj_forward(nsteps, K, win)
        dts = cm.cm_adj_get_dts(nsteps)
        gT = np.empty((cfg.nz, cfg.nx))
        gRa = cm.cm_adj_backward(None, gT)
    finally:
        s.close()
    return J, dts, gT, gRa


def test_config5_gradient_frozen_limiter_against_central_differences():
    """The adjoint workload in full: 2000 steps on the CFL dts, checkpoints
    every 100, J = mean Nu_bar over steps 1501..2000.  With the frozen-limiter
    reading, <dJ/dT0, v> matches central differences of J (the runs replay the
    same dts) at steps 1e-4 and 1e-5 (measured: 3e-4 and 2.4e-3; the finite
    differences themselves spread by 3e-3 over steps 1e-3..1e-6, because the
    limiter's corners make J rough at small scales)."""
    cfg, X0, v, perturbed, cm = _config5_start()
    J, dts, gT, gRa = _adjoint(cfg, X0, 2000, 100, 1501, cm.CM_ADJ_PHI_FROZEN)
    ad = float(np.sum(gT * v))
    assert math.isfinite(gRa) and abs(ad) > 0.1
    for h in (1e-4, 1e-5):
        fd = (_replayed_J(cfg, perturbed(h), dts, 1501) - _replayed_J(cfg, perturbed(-h), dts, 1501)) / (2 * h)
        assert abs(fd - ad) <= 5e-3 * abs(ad), (h, fd, ad)


def test_exact_limiter_reading_to_200_steps_and_its_growth_beyond():
    """The exact derivative (phi' = 2 on 0 < 2r < 1) is the derivative of the
    discrete map: over 200 steps it matches central differences within 1e-4
    (measured 7e-6).  The vector limiter's ratio is not Lipschitz (the ratio
    of two dot products where dX_+ -> 0), and by 500 steps its tangent map
    has grown by orders of magnitude beyond the bounded frozen-limiter
    gradient, while J's finite differences stay near the latter."""
    cfg, X0, v, perturbed, cm = _config5_start()
    J, dts, gT, _ = _adjoint(cfg, X0, 200, 50, 151, cm.CM_ADJ_PHI_EXACT)
    ad = float(np.sum(gT * v))
    h = 1e-5
    fd = (_replayed_J(cfg, perturbed(h), dts, 151) - _replayed_J(cfg, perturbed(-h), dts, 151)) / (2 * h)
    assert abs(fd - ad) <= 1e-4 * abs(ad), (fd, ad)
    _, _, gTe, _ = _adjoint(cfg, X0, 500, 100, 376, cm.CM_ADJ_PHI_EXACT)
    _, _, gTf, _ = _adjoint(cfg, X0, 500, 100, 376, cm.CM_ADJ_PHI_FROZEN)
    assert np.linalg.norm(gTe) > 100 * np.linalg.norm(gTf)


def test_dJ_dRa_frozen_limiter_against_central_differences():
    """dJ/dRa through mu and K at 500 steps (window 376..500) against central
    differences in Ra at relative steps 1e-2 and 1e-3 on the replayed dts
    (measured 1.4e-3 and 2.2e-3)."""
    cfg, X0, v, perturbed, cm = _config5_start()
    J, dts, gT, gRa = _adjoint(cfg, X0, 500, 100, 376, cm.CM_ADJ_PHI_FROZEN)
    for h in (1e-2, 1e-3):
        fd = (_replayed_J(cfg, X0, dts, 376, cfg.Ra * (1 + h)) - _replayed_J(cfg, X0, dts, 376, cfg.Ra * (1 - h))) / (
            2 * h * cfg.Ra)
        assert abs(fd - gRa) <= 1e-2 * abs(gRa), (h, fd, gRa)


def test_temperature_objective_through_autograd():
    """NuObjectiveT: J as a function of the initial temperature field (the
    initial condition of cm_init built by cm_set_temperature).  Its autograd
    gradient is the library's dJ/dT0 bit for bit, equal for CPU and CUDA
    tensors, zero on the plates, and matches central differences of J
    (TVD term off: J smooth)."""
    import paper_2411_10372_gb300 as cm
    from paper_2411_10372_gb300.adjoint import NuObjectiveT
    nx, nz, nsteps, K, win = 48, 13, 16, 5, 9
    grid = dict(nx=nx, nz=nz, tvd_form=O.TVD_OFF, dt_fixed=2e-3)
    rng = np.random.default_rng(3)
    z = np.linspace(0.0, 1.0, nz)[:, None]
    T0 = (1.0 - 0.6 * z) + 1e-2 * rng.uniform(-1, 1, (nz, nx))
    s = cm.Solver(nx, nz, 1e6, precision="fp64", tvd_form=O.TVD_OFF, dt_fixed=2e-3)
    try:
        cm.cm_set_temperature(T0)
        X = s.state()
        J = cm.cm_adj_forward(nsteps, K, win)
        gT = np.empty((nz, nx))
        cm.cm_adj_backward(None, gT)
    finally:
        s.close()
    assert np.all(X[1:3] == 0.0) and np.all(gT[0] == 0) and np.all(gT[-1] == 0)
    grads = []
    for device in ("cpu", "cuda"):
        t = torch.tensor(T0, device=device, requires_grad=True)
        Jt = NuObjectiveT.apply(t, torch.tensor(1e6, dtype=torch.float64), grid, nsteps, K, win)
        Jt.backward()
        assert float(Jt.detach()) == J
        grads.append(t.grad.cpu().numpy())
    assert np.array_equal(grads[0], gT) and np.array_equal(grads[1], gT)
    v = np.zeros((nz, nx))
    v[1:-1] = rng.uniform(-1, 1, (nz - 2, nx))
    h = 1e-6
    Jp = float(NuObjectiveT.apply(torch.tensor(T0 + h * v), torch.tensor(1e6, dtype=torch.float64), grid, nsteps, K,
                                  win))
    cm.cm_finalize()
    Jm = float(NuObjectiveT.apply(torch.tensor(T0 - h * v), torch.tensor(1e6, dtype=torch.float64), grid, nsteps, K,
                                  win))
    cm.cm_finalize()
    fd = (Jp - Jm) / (2 * h)
    ad = float(np.sum(gT * v))
    assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)
