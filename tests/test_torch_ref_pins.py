"""Pins of oracle/torch_ref.py, the PyTorch restatement of the 2D step whose
autograd gradient is the reference for the library's adjoint.

(1) Its states equal the C oracle's, step by step, from the same input with
the same dt (the C oracle is itself pinned by tests/test_oracle_pins.py), on
uniform and on stretched z-grids.
(2) Its Nu_bar equals the C oracle's diagnostics.
(3) Its autograd gradient of J (a time average of Nu_bar over a window of
steps, dt frozen) matches central finite differences of J computed with the
C oracle alone, along random directions of the initial temperature and of Ra.
That last check is the definition of the derivative; it does not use autograd.
"""
import numpy as np
import pytest
import torch

import oracle as O
from oracle.torch_ref import Model, TVD_OFF, TVD_SPLIT, TVD_SUM, isobaric_state


def _model(cfg):
    stretched = cfg.zstretch != 0.0 or cfg.znodes is not None
    return Model(cfg.nx, cfg.nz, Pr=cfg.Pr, gamma=cfg.gamma, eps=cfg.eps, D=cfg.D, aspect=cfg.aspect,
                 gravity=cfg.gravity, t_bot=cfg.t_bot, t_top=cfg.t_top, stokes=cfg.stokes, tvd_form=cfg.tvd_form,
                 znodes=O.znodes(cfg) if stretched else None)


def _given_planes(nz):
    s = np.linspace(0.0, 1.0, nz)
    z = s - 0.6 * np.sin(2 * np.pi * s) / (2 * np.pi)
    z[0], z[-1] = 0.0, 1.0
    return z


@pytest.mark.parametrize("tvd,zgrid", [(TVD_SPLIT, "uniform"), (TVD_SUM, "uniform"), (TVD_OFF, "uniform"),
                                       (TVD_SPLIT, "tanh"), (TVD_SUM, "tanh"), (TVD_SPLIT, "given")])
def test_states_match_c_oracle(tvd, zgrid):
    """On uniform planes, on the tanh grid (beta = 1.5) and on given planes."""
    kw = {"uniform": {}, "tanh": {"zstretch": 1.5}, "given": {"znodes": _given_planes(9)}}[zgrid]
    cfg = O.Config(nx=24, nz=9, Ra=1e5, seed=3, pert_amp=2e-2, tvd_form=tvd, **kw)
    m = _model(cfg)
    X = O.init(cfg)
    Xt = torch.from_numpy(X.copy())
    mu, kth = m.coefs(cfg.Ra)
    for _ in range(12):
        X, _, dts = O.step(cfg, X, 1)
        Xt = m.step(Xt, float(dts[0]), mu, kth)
        for f in range(4):
            scale = max(np.max(np.abs(X[f])), np.max(np.abs(X[0])))
            assert np.max(np.abs(Xt[f].numpy() - X[f])) <= 1e-13 * scale, f


@pytest.mark.parametrize("beta", [0.0, 1.5])
def test_nu_bar_matches_c_oracle(beta):
    cfg = O.Config(nx=32, nz=11, Ra=1e6, seed=5, pert_amp=5e-2, zstretch=beta)
    X, _, _ = O.step(cfg, O.init(cfg), 30)
    m = _model(cfg)
    got = float(m.nu_bar(torch.from_numpy(X)))
    want = O.diag(cfg, X)["Nu_bar"]
    assert abs(got - want) <= 1e-12 * max(1.0, abs(want))


def _J_oracle(cfg, X0, nsteps, win):
    """J from the C oracle only: fixed dt, mean of Nu_bar over steps win..nsteps."""
    X, acc = X0, 0.0
    for n in range(1, nsteps + 1):
        X, _, _ = O.step(cfg, X, 1)
        if n >= win:
            acc += O.diag(cfg, X)["Nu_bar"]
    return acc / (nsteps - win + 1)


@pytest.mark.parametrize("tvd,beta", [(TVD_SPLIT, 0.0), (TVD_SUM, 0.0), (TVD_SPLIT, 1.5)])
def test_autograd_gradient_matches_finite_differences_of_c_oracle(tvd, beta):
    nsteps, win = 16, 9
    base = O.Config(nx=20, nz=9, Ra=2e5, seed=9, pert_amp=3e-2, tvd_form=tvd, zstretch=beta)
    X0 = O.init(base)
    dt = 0.8 * O.dt(base, X0)
    cfg = O.Config(nx=20, nz=9, Ra=2e5, seed=9, pert_amp=3e-2, tvd_form=tvd, dt_fixed=dt, zstretch=beta)
    m = _model(cfg)
    rng = np.random.default_rng(17)
    # X0 as an isobaric function of the temperature field T0 (plates fixed)
    rho = X0[0]
    T0 = m.b * (X0[3] / rho - m.g * m.z.numpy())
    P0 = m.a * rho * T0
    T0t = torch.tensor(T0, requires_grad=True)
    Ra = torch.tensor(cfg.Ra, dtype=torch.float64, requires_grad=True)
    X0t = isobaric_state(m, T0t, torch.from_numpy(P0))
    J = m.objective(X0t, Ra, [dt] * nsteps, win)
    J.backward()
    gT, gRa = T0t.grad.numpy(), float(Ra.grad)
    # directional derivative along a random interior temperature perturbation
    v = np.zeros_like(T0)
    v[1:-1] = rng.uniform(-1, 1, (cfg.nz - 2, cfg.nx))
    h = 1e-6
    Xp = isobaric_state(m, torch.from_numpy(T0 + h * v), torch.from_numpy(P0)).numpy()
    Xm = isobaric_state(m, torch.from_numpy(T0 - h * v), torch.from_numpy(P0)).numpy()
    fd = (_J_oracle(cfg, Xp, nsteps, win) - _J_oracle(cfg, Xm, nsteps, win)) / (2 * h)
    ad = float(np.sum(gT * v))
    assert abs(ad) > 1e-6
    assert abs(fd - ad) <= 1e-5 * abs(ad), (fd, ad)
    # Ra through mu and K
    hr = 1e-6 * cfg.Ra
    cp = O.Config(nx=20, nz=9, Ra=cfg.Ra + hr, seed=9, pert_amp=3e-2, tvd_form=tvd, dt_fixed=dt, zstretch=beta)
    cm_ = O.Config(nx=20, nz=9, Ra=cfg.Ra - hr, seed=9, pert_amp=3e-2, tvd_form=tvd, dt_fixed=dt, zstretch=beta)
    fdr = (_J_oracle(cp, X0, nsteps, win) - _J_oracle(cm_, X0, nsteps, win)) / (2 * hr)
    assert abs(gRa) > 0
    assert abs(fdr - gRa) <= 1e-4 * abs(gRa), (fdr, gRa)
