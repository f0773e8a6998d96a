"""Mutation test of the pins of oracle/torch_ref.py (the PyTorch restatement
whose autograd gradient is the reference for the library's adjoint).

Each case plants one plausible mistake in a copy of torch_ref.py, mostly in
its stretched-grid form (cell widths, spans, TVD weights, plate rules, the
three-plane plate derivative), and checks that at least one comparison with
the C oracle fails on it: states step by step on the tanh grid and on given
planes, Nu_bar, or the autograd gradient against central differences of the
C oracle's J.  The mistakes are planted in the restatement, on the CPU.
"""
import os
import types

import numpy as np
import pytest
import torch

import oracle as O

SRC = os.path.join(os.path.dirname(O.__file__), "torch_ref.py")

# (name, text in torch_ref.py, replacement)
MUTANTS = [
    ("tvd_weights_swapped", "Yi = Y1 + (self.rp * Dall[:, 1:K] - self.rm * Dall[:, 0:K - 1])",
     "Yi = Y1 + (self.rm * Dall[:, 1:K] - self.rp * Dall[:, 0:K - 1])"),
    ("tvd_weights_dropped", "Yi = Y1 + (self.rp * Dall[:, 1:K] - self.rm * Dall[:, 0:K - 1])",
     "Yi = Y1 + (Dall[:, 1:K] - Dall[:, 0:K - 1])"),
    ("rm_from_the_upper_spacing", "self.rm = (hp[0:K - 1] / w[1:K])[:, None]",
     "self.rm = (hp[1:K] / w[1:K])[:, None]"),
    ("flux_factor_over_spacing", "lam = Delta / self.w[1:K] if st else Delta / hz",
     "lam = Delta / self.hp[1:K] if st else Delta / hz"),
    ("bottom_plate_full_cell", "lam_b = Delta / self.w[0, 0] if st else 2.0 * (Delta / hz)",
     "lam_b = Delta / (2.0 * self.w[0, 0]) if st else 2.0 * (Delta / hz)"),
    ("top_plate_uses_bottom_width", "lam_t = Delta / self.w[K, 0] if st else 2.0 * (Delta / hz)",
     "lam_t = Delta / self.w[1, 0] if st else 2.0 * (Delta / hz)"),
    ("one_sided_derivative_over_width", "return (f[1:] - f[:-1]) / (self.hp if st else hz)",
     "return (f[1:] - f[:-1]) / (self.w[1:] if st else hz)"),
    ("courant_of_the_lower_interface", "Delta, self.hp[1:K - 1] if st else hz)",
     "Delta, self.hp[0:K - 2] if st else hz)"),
    ("central_span_uniform", "return (f[2:] - f[:-2]) / (self.sc if self.stretched else 2.0 * hz)",
     "return (f[2:] - f[:-2]) / (2.0 * hz)"),
    ("cell_width_full_on_plates", "w = torch.cat([hp[:1] / 2.0, (hp[:-1] + hp[1:]) / 2.0, hp[-1:] / 2.0])",
     "w = torch.cat([hp[:1], (hp[:-1] + hp[1:]) / 2.0, hp[-1:]])"),
    ("plate_quadratic_middle_coefficient", "+ (h1 + h2) / (h1 * h2) * v[1]", "+ (h1 + h2) / (h1 * h1) * v[1]"),
    ("top_nusselt_sign", "nt = (1.0 / self.eps) * d3(g, z[K] - z[K - 1], z[K - 1] - z[K - 2])",
     "nt = -(1.0 / self.eps) * d3(g, z[K] - z[K - 1], z[K - 1] - z[K - 2])"),
    ("stretched_tsa_uses_index", "f = [T[q].sum() / self.nx - (1.0 - self.D * z[q]) for q in range(3)]",
     "f = [T[q].sum() / self.nx - (1.0 - self.D * (q / K)) for q in range(3)]"),
    ("planes_ignored_in_potential", "            self.z = z[:, None]\n", "\n"),
    ("stokes_sign", "ta = mu * ((daa + daa) + self.stokes * div)", "ta = mu * ((daa + daa) - self.stokes * div)"),
    ("gravity_source_sign", "S = torch.stack([S[0], S[1], -self.g * X[0, 1:K], S[3]])",
     "S = torch.stack([S[0], S[1], self.g * X[0, 1:K], S[3]])"),
]


def _load(src):
    mod = types.ModuleType("torch_ref_mutant")
    exec(compile(src, "torch_ref_mutant.py", "exec"), mod.__dict__)
    return mod


def _given_planes(nz):
    s = np.linspace(0.0, 1.0, nz)
    z = s - 0.6 * np.sin(2 * np.pi * s) / (2 * np.pi)
    z[0], z[-1] = 0.0, 1.0
    return z


def _model(M, cfg):
    return M.Model(cfg.nx, cfg.nz, Pr=cfg.Pr, gamma=cfg.gamma, eps=cfg.eps, D=cfg.D, aspect=cfg.aspect,
                   gravity=cfg.gravity, t_bot=cfg.t_bot, t_top=cfg.t_top, stokes=cfg.stokes, tvd_form=cfg.tvd_form,
                   znodes=O.znodes(cfg))


def _states_agree(M, cfg, nsteps=12):
    m = _model(M, cfg)
    X = O.init(cfg)
    Xt = torch.from_numpy(X.copy())
    mu, kth = m.coefs(cfg.Ra)
    for _ in range(nsteps):
        X, _, dts = O.step(cfg, X, 1)
        Xt = m.step(Xt, float(dts[0]), mu, kth)
        for f in range(4):
            scale = max(np.max(np.abs(X[f])), np.max(np.abs(X[0])))
            if not np.max(np.abs(Xt[f].numpy() - X[f])) <= 1e-13 * scale:
                return False
    return True


def _nu_agrees(M, cfg):
    X, _, _ = O.step(cfg, O.init(cfg), 30)
    got = float(_model(M, cfg).nu_bar(torch.from_numpy(X)))
    want = O.diag(cfg, X)["Nu_bar"]
    return abs(got - want) <= 1e-12 * max(1.0, abs(want))


def _gradient_agrees(M, beta):
    """Autograd of J along a random interior temperature direction against
    central differences of the C oracle's J (fixed dt)."""
    nsteps, win = 10, 6
    base = O.Config(nx=16, nz=9, Ra=2e5, seed=9, pert_amp=3e-2, zstretch=beta)
    X0 = O.init(base)
    dt = 0.8 * O.dt(base, X0)
    cfg = O.Config(nx=16, nz=9, Ra=2e5, seed=9, pert_amp=3e-2, dt_fixed=dt, zstretch=beta)
    m = _model(M, cfg)
    rho = X0[0]
    T0 = m.b * (X0[3] / rho - m.g * m.z.numpy())
    P0 = m.a * rho * T0
    T0t = torch.tensor(T0, requires_grad=True)
    J = m.objective(M.isobaric_state(m, T0t, torch.from_numpy(P0)), cfg.Ra, [dt] * nsteps, win)
    J.backward()
    v = np.zeros_like(T0)
    v[1:-1] = np.random.default_rng(17).uniform(-1, 1, (cfg.nz - 2, cfg.nx))

    def J_oracle(T):
        # the oracle's own isobaric state: rho = p / (a T), zero velocity
        X = O.init(cfg)
        cl_a = m.a
        z = O.znodes(cfg)[:, None]
        r = P0 / (cl_a * T)
        X[0], X[1], X[2] = r, 0.0, 0.0
        X[3] = r * (T / m.b + m.g * z)
        acc = 0.0
        for n in range(1, nsteps + 1):
            X, _, _ = O.step(cfg, X, 1)
            if n >= win:
                acc += O.diag(cfg, X)["Nu_bar"]
        return acc / (nsteps - win + 1)
    h = 1e-6
    fd = (J_oracle(T0 + h * v) - J_oracle(T0 - h * v)) / (2 * h)
    ad = float(np.sum(T0t.grad.numpy() * v))
    return abs(fd - ad) <= 1e-5 * max(abs(ad), 1e-12)


def _all_pins_pass(M):
    for zgrid in ("tanh", "given"):
        kw = {"tanh": {"zstretch": 1.5}, "given": {"znodes": _given_planes(9)}}[zgrid]
        if not _states_agree(M, O.Config(nx=24, nz=9, Ra=1e5, seed=3, pert_amp=2e-2, **kw)):
            return False
    if not _nu_agrees(M, O.Config(nx=32, nz=11, Ra=1e6, seed=5, pert_amp=5e-2, zstretch=1.5)):
        return False
    return _gradient_agrees(M, 1.5)


def test_pins_pass_on_unmutated_copy():
    M = _load(open(SRC).read())
    assert _all_pins_pass(M)


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site of {name} not found exactly once"
    M = _load(src.replace(old, new))
    try:
        caught = not _all_pins_pass(M)
    except Exception:  # a mutant that no longer runs is caught as well
        caught = True
    assert caught, name
