"""Batched ensemble (many uneven 2D boxes, FP32, one launch per sweep for all
boxes, graph-replayed steps): every box must agree with its own single-box
run, and a box must match the FP64 oracle within the FP32 bar of
tests/test_gpu_parity.py.  Batch and solo runs may split rows into segments
differently (the autotuner).  The default FP32 sweeps are reproducible bit
for bit only for a fixed split (at the FP32 noise level otherwise), which this
unstable flow amplifies to ~2e-6 over 63 steps, so 1e-5 is their bar, far
below what a wrong work item, dt slot or graph replay would produce; with
cm_params.layout_exact = 1 every box equals its solo run bit for bit."""
import ctypes
import math

import numpy as np
import pytest

import oracle as O
from physics import closures

pytestmark = pytest.mark.gpu

SIZES = [(68, 17), (132, 33), (160, 40), (256, 64), (520, 130)]
RAS = [1e5, 3e6, 1e7, 1e6, 1e8]


def _grids(cm):
    return [cm.cm_grid(2, nx, 1, nz, 4.0) for nx, nz in SIZES]


def _params(cm, seed=777):
    p = cm.cm_default_params()
    p.precision = cm.CM_FP32
    p.seed = seed
    return p


def test_batch_boxes_equal_their_solo_runs():
    import paper_2411_10372_gb300 as cm
    nsteps = 63  # one 50-step graph replay plus direct launches, odd count
    cm.cm_batch_init(_grids(cm), RAS, 1.0, 5.0 / 3.0, _params(cm))
    seg_z, seg_x = cm.cm_batch_tuning()
    assert all(s in (6, 8, 10, 12, 14, 16, 20, 24, 29, 32, 40, 48, 64, 96, 128) for s in seg_z + seg_x)
    cm.cm_batch_step(nsteps)
    diags = cm.cm_batch_diagnostics()
    batch_states = []
    for b, (nx, nz) in enumerate(SIZES):
        out = np.empty((4, nz, nx))
        batch_states.append(cm.cm_batch_get_state(b, out))
    cm.cm_batch_finalize()
    for b, (nx, nz) in enumerate(SIZES):
        s = cm.Solver(nx, nz, RAS[b], 1.0, 5.0 / 3.0, precision="fp32", seed=777 + b)
        s.step(nsteps)
        solo = s.state()
        d = s.sample()
        s.close()
        for f in range(4):
            err = np.linalg.norm(batch_states[b][f] - solo[f]) / np.linalg.norm(solo[f] if f in (0, 3) else solo[0])
            assert err <= 1e-5, (b, f, err)
        assert diags[b]["step"] == nsteps and d["step"] == nsteps
        for k in ("t", "dt", "mass"):
            assert abs(diags[b][k] - d[k]) <= 1e-5 * abs(d[k]), (b, k)


@pytest.mark.parametrize("split", [0, 1])
def test_layout_exact_batch_boxes_equal_their_solo_runs_bit_for_bit(split):
    """With cm_params.layout_exact = 1 the FP32 sweeps round alike whatever
    the segment split, so every box of the batch (its own segment lengths
    from the batch tuner, its own kernels) equals its single-box run bit for
    bit, time and dt included; in either order of the half steps
    (cm_params.split)."""
    import paper_2411_10372_gb300 as cm
    nsteps = 63
    p = _params(cm)
    p.layout_exact = 1
    p.split = split
    cm.cm_batch_init(_grids(cm), RAS, 1.0, 5.0 / 3.0, p)
    cm.cm_batch_step(nsteps)
    diags = cm.cm_batch_diagnostics()
    batch_states = [cm.cm_batch_get_state(b, np.empty((4, nz, nx))) for b, (nx, nz) in enumerate(SIZES)]
    cm.cm_batch_finalize()
    for b, (nx, nz) in enumerate(SIZES):
        s = cm.Solver(nx, nz, RAS[b], 1.0, 5.0 / 3.0, precision="fp32", seed=777 + b, layout_exact=1, split=split)
        s.step(nsteps)
        solo = s.state()
        d = s.sample()
        s.close()
        assert np.array_equal(batch_states[b], solo), (b, float(np.max(np.abs(batch_states[b] - solo))))
        assert diags[b]["t"] == d["t"] and diags[b]["dt"] == d["dt"]


@pytest.mark.parametrize("split", [0, 1])
def test_batch_box_matches_oracle(split):
    import paper_2411_10372_gb300 as cm
    nsteps = 40
    p = _params(cm, seed=5)
    p.split = split
    cm.cm_batch_init(_grids(cm), RAS, 1.0, 5.0 / 3.0, p)
    cm.cm_batch_step(nsteps)
    b = 3
    nx, nz = SIZES[b]
    got = cm.cm_batch_get_state(b, np.empty((4, nz, nx)))
    masses = [d["mass"] for d in cm.cm_batch_diagnostics()]
    cm.cm_batch_finalize()
    cfg = O.Config(nx=nx, nz=nz, Ra=RAS[b], seed=5 + b, split=split)
    want, _, _ = O.step(cfg, O.init(cfg), nsteps)
    rel = lambda a, w: float(np.linalg.norm(a - w) / np.linalg.norm(w))
    assert rel(got[0], want[0]) <= 1e-5 and rel(got[3], want[3]) <= 1e-5
    cl = closures(cfg.gamma, cfg.eps, cfg.D, cfg.Ra, cfg.Pr)
    scale = np.linalg.norm(want[0]) * math.sqrt(cfg.gamma * cl["a"])
    for f in (1, 2):
        assert np.linalg.norm(got[f] - want[f]) / scale <= 1e-5
    assert abs(masses[b] - O.diag(cfg, want)["mass"]) <= 1e-6


def test_batch_rejects_bad_boxes():
    import paper_2411_10372_gb300 as cm
    with pytest.raises(cm.CMError) as e:
        cm.cm_batch_init([cm.cm_grid(2, 65, 1, 17, 4.0)], [1e6], 1.0, 5.0 / 3.0, _params(cm))
    assert e.value.code == cm.CM_EINVAL
    p = _params(cm)
    p.precision = cm.CM_FP64
    with pytest.raises(cm.CMError):
        cm.cm_batch_init([cm.cm_grid(2, 64, 1, 17, 4.0)], [1e6], 1.0, 5.0 / 3.0, p)


def test_stretched_batch_boxes_equal_their_solo_runs():
    """Boxes on tanh z-grids (beta 1 and 2), one on given planes and one
    uniform box share a batch: the plane-table sweeps step every box, and each
    box equals its solo run on the same planes (the uniform box: znodes =
    k/K).  The plate Nusselt numbers and the mass use the stretched-grid
    weights, which differ from the uniform ones by far more than the bars
    (eps = 0.1 is the default of _params)."""
    import paper_2411_10372_gb300 as cm
    sizes = [(68, 17), (132, 33), (160, 40), (256, 64)]
    ras = [1e5, 3e6, 1e7, 1e6]
    s0 = np.linspace(0.0, 1.0, sizes[2][1])
    given = s0 - 0.6 * np.sin(2 * np.pi * s0) / (2 * np.pi)  # plates refined, strictly increasing
    given[0], given[-1] = 0.0, 1.0
    uniform = np.arange(sizes[3][1]) / (sizes[3][1] - 1)
    solo_kw = [dict(zstretch=1.0), dict(zstretch=2.0), dict(znodes=given), dict(znodes=uniform)]
    given_ptr = given.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    grids = [cm.cm_grid(2, sizes[0][0], 1, sizes[0][1], 4.0, 1.0), cm.cm_grid(2, sizes[1][0], 1, sizes[1][1], 4.0, 2.0),
             cm.cm_grid(2, sizes[2][0], 1, sizes[2][1], 4.0, 0.0, given_ptr), cm.cm_grid(2, sizes[3][0], 1, sizes[3][1], 4.0)]
    nsteps = 63
    cm.cm_batch_init(grids, ras, 1.0, 5.0 / 3.0, _params(cm, seed=91))
    cm.cm_batch_step(nsteps)
    diags = cm.cm_batch_diagnostics()
    states = [cm.cm_batch_get_state(b, np.empty((4, nz, nx))) for b, (nx, nz) in enumerate(sizes)]
    cm.cm_batch_finalize()
    for b, (nx, nz) in enumerate(sizes):
        s = cm.Solver(nx, nz, ras[b], 1.0, 5.0 / 3.0, precision="fp32", seed=91 + b, **solo_kw[b])
        s.step(nsteps)
        solo = s.state()
        d = s.sample()
        z = s.z
        s.close()
        for f in range(4):
            err = np.linalg.norm(states[b][f] - solo[f]) / np.linalg.norm(solo[f] if f in (0, 3) else solo[0])
            assert err <= 1e-5, (b, f, err)
        assert diags[b]["status"] == 0 and diags[b]["step"] == nsteps
        for k in ("t", "dt", "mass"):
            assert abs(diags[b][k] - d[k]) <= 1e-5 * abs(d[k]), (b, k)
        # plate Nu: a difference of the plane means of T (1e-6 allowed, the
        # FP32 split noise) enters amplified by the three-plane derivative
        # coefficients over eps; uniform-grid weights on these planes would be
        # off by O(1)
        for k, (a, m, c) in (("Nu_bot", z[:3]), ("Nu_top", z[::-1][:3])):
            h1, h2 = abs(m - a), abs(c - m)
            amp = ((2 * h1 + h2) / (h1 * (h1 + h2)) + (h1 + h2) / (h1 * h2) + h1 / (h2 * (h1 + h2))) / 0.1
            assert abs(diags[b][k] - d[k]) <= 1e-6 * amp, (b, k, diags[b][k], d[k], 1e-6 * amp)


def test_batch_rejects_a_box_beyond_the_explicit_diffusion_bound():
    """cm_init's bound on the explicit diffusion number holds per box: on
    the tanh grid of beta = 2 the 1016 x 254 box at Ra = 1.5e5 has a first
    spacing of 5.8e-4 and a diffusion number of 1.36 at its first dt."""
    import paper_2411_10372_gb300 as cm
    grids = [cm.cm_grid(2, 128, 1, 32, 4.0, 2.0), cm.cm_grid(2, 1016, 1, 254, 4.0, 2.0)]
    with pytest.raises(cm.CMError) as e:
        cm.cm_batch_init(grids, [1e7, 1.48e5], 1.0, 5.0 / 3.0, _params(cm))
    assert e.value.code == cm.CM_EUNSTABLE and "box 1" in str(e.value), str(e.value)
    with pytest.raises(cm.CMError) as e:
        cm.Solver(1016, 254, 1.48e5, 1.0, 5.0 / 3.0, precision="fp32", zstretch=2.0)
    assert e.value.code == cm.CM_EUNSTABLE
    cm.cm_batch_init([cm.cm_grid(2, 1016, 1, 254, 4.0, 1.0)], [1.48e5], 1.0, 5.0 / 3.0, _params(cm))
    cm.cm_batch_finalize()


@pytest.mark.parametrize("beta", [0.0, 1.5])
def test_large_batch_stages_coefficients_in_shared_memory(beta):
    """More boxes than the constant-memory table holds (300 > 256): the
    kernels that stage each box's coefficients in shared memory run, and a
    box of an uneven mix (different Ra, hence different mu and K) still
    equals its solo run."""
    import paper_2411_10372_gb300 as cm
    n = 300
    sizes = [(16 + 2 * (b % 5), 6 + b % 4) for b in range(n)]
    ras = [1e5 * (1 + b % 7) for b in range(n)]
    grids = [cm.cm_grid(2, nx, 1, nz, 4.0, beta) for nx, nz in sizes]
    cm.cm_batch_init(grids, ras, 1.0, 5.0 / 3.0, _params(cm, seed=31))
    nsteps = 7
    cm.cm_batch_step(nsteps)
    diags = cm.cm_batch_diagnostics()
    picks = (0, 137, 299)
    states = {b: cm.cm_batch_get_state(b, np.empty((4, sizes[b][1], sizes[b][0]))) for b in picks}
    cm.cm_batch_finalize()
    assert all(d["status"] == 0 and d["step"] == nsteps for d in diags)
    for b in picks:
        nx, nz = sizes[b]
        s = cm.Solver(nx, nz, ras[b], 1.0, 5.0 / 3.0, precision="fp32", seed=31 + b, zstretch=beta)
        s.step(nsteps)
        solo = s.state()
        s.close()
        for f in range(4):
            err = np.linalg.norm(states[b][f] - solo[f]) / np.linalg.norm(solo[f] if f in (0, 3) else solo[0])
            assert err <= 1e-5, (b, f, err)
