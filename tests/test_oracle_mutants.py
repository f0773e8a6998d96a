"""Mutation test of the oracle's pins.

Each case plants one plausible mistake (a dropped term, a wrong sign, index or
factor, a transposed operand) in a copy of oracle/cm_oracle.c, builds it, and
checks that at least one pin of tests/test_oracle_pins.py fails on it.  The
mistakes are planted in the oracle, on the CPU; the CUDA path is not involved.
"""
import os
import subprocess
import tempfile

import pytest

import oracle as O
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(O.__file__), "cm_oracle.c")

# (name, text in cm_oracle.c, replacement)
MUTANTS = [
    ("stokes_sign", "(i == al ? p->stokes * div : 0.0)", "(i == al ? -p->stokes * div : 0.0)"),
    ("no_pressure_in_flux", "(i == al ? pr : 0.0)", "0.0"),
    ("pressure_in_z_row_only", "(i == al ? pr : 0.0)", "(i == 2 ? pr : 0.0)"),
    ("gravity_sign", "double S = (c == 3) ? -p->g * X[n] : 0.0;", "double S = (c == 3) ? p->g * X[n] : 0.0;"),
    ("no_viscous_work", "p->kth * dT[al] - work", "p->kth * dT[al]"),
    ("heat_flux_sign", "- p->kth * dT[al]", "+ p->kth * dT[al]"),
    ("tau_transposed", "du[i][al] + du[al][i]", "du[i][al] + du[i][al]"),
    ("corrector_uses_Fn_literal",
     "X[c * N + n] - lam * (w->FP[c * N + np] - w->FP[c * N + n]) + Delta * S;",
     "X[c * N + n] - lam * (w->F[c * N + np] - w->FP[c * N + n]) + Delta * S;"),
    ("no_average", "Y[c * N + n] = (w->XP[c * N + n] + w->XC[c * N + n]) / 2.0;\n                }\n            }\n    /* TVD flux D at",
     "Y[c * N + n] = w->XC[c * N + n];\n                }\n            }\n    /* TVD flux D at"),
    ("wall_half_cell_factor", "X[nK] + (Delta / p->w[K]) * w->F[nK1]", "X[nK] + (Delta / (2.0 * p->w[K])) * w->F[nK1]"),
    ("plate_temperatures_swapped", "double Tw = top ? p->t_top : p->t_bot;", "double Tw = top ? p->t_bot : p->t_top;"),
    ("tvd_sum_form", "(p->tvd_form == 0) ? Gfun(rp, C) + Gfun(rm, C) : Gfun(rp + rm, C)",
     "(p->tvd_form == 1) ? Gfun(rp, C) + Gfun(rm, C) : Gfun(rp + rm, C)"),
    ("tvd_sign", "Y[c * N + n] + (w->D[c * N + n] - w->D[c * N + nm]);\n            }\n}",
     "Y[c * N + n] - (w->D[c * N + n] - w->D[c * N + nm]);\n            }\n}"),
    ("tvd_rminus_index", "dp[c] = X[c * N + n2] - X[c * N + n1];", "dp[c] = X[c * N + n0] - X[c * N + nm];"),
    ("courant_full_dt", "double Co = Delta * fmax(A[n0], A[n1]) / h;",
     "double Co = 2.0 * Delta * fmax(A[n0], A[n1]) / h;"),
    ("split_order_x_first", "printed2[4] = {2, 0, 2, 0}", "printed2[4] = {0, 2, 0, 2}"),
    ("split_palindrome_is_printed_order", "palindrome2[4] = {0, 2, 2, 0}", "palindrome2[4] = {2, 0, 2, 0}"),
    ("split_3d_order_y_last", "printed3[6] = {2, 1, 0, 2, 1, 0}", "printed3[6] = {2, 0, 1, 2, 0, 1}"),
    ("limiter_phi_no_factor2", "fmin(2.0 * r, 1.0)", "fmin(r, 1.0)"),
    ("courant_coefficient_unclamped", "return Co <= 0.5 ? Co * (1.0 - Co) : 0.25;", "return Co * (1.0 - Co);"),
    ("nu_conv_coefficient", "out[1] = sRP / p.eps * (s_conv / vol);", "out[1] = sRP * (s_conv / vol);"),
    ("nu_k_coefficient", "out[2] = p.D * sRP / 2.0 * (s_k / vol);", "out[2] = p.D * sRP * (s_k / vol);"),
    ("tsa_sign", "double Tsa = T - (1.0 - p.D * z);", "double Tsa = T - (1.0 + p.D * z);"),
    ("plate_nu_first_order", "(-3.0 * f[0] + 4.0 * f[1] - f[2]) / (2.0 * dz)", "(f[1] - f[0]) / dz"),
    ("re_missing_sqrt", "sqrt(p.Ra / p.Pr) * sqrt(s_u2 / vol)", "sqrt(p.Ra / p.Pr) * (s_u2 / vol)"),
    ("sound_speed_missing_gamma", "double c = sqrt(p->gam * p->a * w->T[n]);", "double c = sqrt(p->a * w->T[n]);"),
    ("perturb_plates", "if (k > 0 && k < p.nz - 1) T = Tc[k]", "T = Tc[k]"),
    ("potential_missing_in_T", "- p->g * zk(p, k));", ");"),
    ("div_missing_dy", "double div = du[0][0] + du[1][1] + du[2][2];", "double div = du[0][0] + du[2][2];"),
    ("y_tvd_rminus_row", "int j1 = (al == 1) ? (j + 1) % p->ny : j;", "int j1 = j;"),
    # stretched z-grid
    ("tanh_missing_normalisation", "return 0.5 * (1.0 + tanh(beta * s) / tanh(beta));",
     "return 0.5 * (1.0 + tanh(beta * s));"),
    ("stretched_inner_derivative_uses_width", "span = (d == 2) ? (fwd ? p->hp[k] : p->hp[k - 1]) : p->h[d];",
     "span = (d == 2) ? p->w[k] : p->h[d];"),
    ("stretched_backward_derivative_index", "span = (d == 2) ? (fwd ? p->hp[k] : p->hp[k - 1]) : p->h[d];",
     "span = (d == 2) ? (fwd ? p->hp[k] : p->hp[k]) : p->h[d];"),
    ("stretched_cross_span", "span = (d == 2) ? p->hp[k - 1] + p->hp[k] : 2.0 * p->h[d];",
     "span = (d == 2) ? 2.0 * p->hp[k] : 2.0 * p->h[d];"),
    ("stretched_predictor_over_spacing",
     "double lam = Delta / p->w[k];\n                size_t n = idx(p, i, j, k), nm",
     "double lam = Delta / p->hp[k];\n                size_t n = idx(p, i, j, k), nm"),
    ("stretched_corrector_over_spacing",
     "double lam = Delta / p->w[k];\n                size_t n = idx(p, i, j, k), np",
     "double lam = Delta / p->hp[k - 1];\n                size_t n = idx(p, i, j, k), np"),
    ("stretched_plate_half_cell", "(Delta / p->w[0]) * w->FP[n1]", "(Delta / p->hp[0]) * w->FP[n1]"),
    ("stretched_tvd_weights_swapped", "double rp = p->hp[k] / p->w[k], rm = p->hp[k - 1] / p->w[k];",
     "double rp = p->hp[k - 1] / p->w[k], rm = p->hp[k] / p->w[k];"),
    ("stretched_tvd_unweighted", "(rp * w->D[c * N + n] - rm * w->D[c * N + nm])",
     "(w->D[c * N + n] - w->D[c * N + nm])"),
    ("stretched_width_one_sided", "p->w[k] = (p->hp[k - 1] + p->hp[k]) / 2.0;", "p->w[k] = p->hp[k];"),
    ("stretched_courant_over_cell_width", "tvd_flux(p, X, w->A, Delta, p->hp[k], idx(p, i, j, k - 1)",
     "tvd_flux(p, X, w->A, Delta, p->w[k], idx(p, i, j, k - 1)"),
    ("stretched_courant_over_spacing_below", "tvd_flux(p, X, w->A, Delta, p->hp[k], idx(p, i, j, k - 1)",
     "tvd_flux(p, X, w->A, Delta, p->hp[k - 1], idx(p, i, j, k - 1)"),
    ("stretched_cfl_largest_spacing", "return fmin(p->hp[k - 1], p->hp[k]);", "return fmax(p->hp[k - 1], p->hp[k]);"),
    ("stretched_diag_uniform_weights", "double wgt = p.stretched ? p.w[k] : ((k == 0 || k == p.nz - 1) ? 0.5 : 1.0);",
     "double wgt = (k == 0 || k == p.nz - 1) ? 0.5 : 1.0;"),
    ("stretched_plate_nu_coefficient", "-(2.0 * h1 + h2) / (h1 * (h1 + h2)) * f[0]", "-(2.0 * h1 + h2) / (h1 * (h1 + h1)) * f[0]"),
    ("stretched_plate_nu_top_spacing", "h2 = p.z[K - 1] - p.z[K - 2];", "h2 = p.z[K] - p.z[K - 1];"),
    # extended diagnostics
    ("ext_dz3_weights_swapped", "return (hm * hm * fp - hp * hp * fm + (hp * hp - hm * hm) * f0)",
     "return (hp * hp * fp - hm * hm * fm + (hm * hm - hp * hp) * f0)"),
    ("ext_dzz3_missing_factor", "return 2.0 * ((fp - f0) / hp - (f0 - fm) / hm) / (hm + hp);",
     "return ((fp - f0) / hp - (f0 - fm) / hm) / (hm + hp);"),
    ("ext_fn_missing_x_advection", "s[0] += rho * ((ux * dxuz + uy * dyuz) + uz * dzuz);",
     "s[0] += rho * (uy * dyuz + uz * dzuz);"),
    ("ext_fn_missing_y_advection", "s[0] += rho * ((ux * dxuz + uy * dyuz) + uz * dzuz);",
     "s[0] += rho * (ux * dxuz + uz * dzuz);"),
    ("ext_fp_sign", "s[1] += -dz3(&p, k, Pr[zm], Pr[n], Pr[zp]);", "s[1] += dz3(&p, k, Pr[zm], Pr[n], Pr[zp]);"),
    ("ext_fv_stokes_factor", "(2.0 + p.stokes) * dzz", "(1.0 + p.stokes) * dzz"),
    ("ext_correlation_no_sqrt", "out[0] = (s_conv / vol) / sqrt(out[1] * out[2]);",
     "out[0] = (s_conv / vol) / (out[1] * out[2]);"),
    ("ext_bl_bulk_band", "if (p.z[k] >= 0.25 && p.z[k] <= 0.75) {", "if (p.z[k] >= 0.0 && p.z[k] <= 0.75) {"),
    ("ext_bl_top_sign", "out[4] = (sb[0] - tb) / dtp;", "out[4] = (tb - sb[0]) / dtp;"),
    ("ext_bl_bottom_plane", "out[3] = (tb - sa[0]) / db;", "out[3] = (tb - sa[1]) / db;"),
    ("ext_r_missing_half", "double r = p.b * u2 / (2.0 * T[n]);", "double r = p.b * u2 / T[n];"),
    ("ext_rhoA_exponent", "pow(1.0 - p.D * z, 1.0 / (p.gam - 1.0))", "pow(1.0 - p.D * z, p.gam / (p.gam - 1.0))"),
    ("ext_rms_without_root", "out[(size_t)k * 9 + 8] = sqrt(usum / cells);", "out[(size_t)k * 9 + 8] = usum / cells;"),
    ("ext_slope_bl_tolerance_unscaled", "double target = tol * p->D,", "double target = tol,"),
    ("ext_slope_bl_no_interpolation", "return dprev + (sprev - target) / (sprev - s) * (d - dprev);", "return d;"),
    ("ext_slope_bl_of_T_not_Tsa", "sal[k] = TA[k] - (1.0 - p.D * p.z[k]);", "sal[k] = TA[k];"),
    ("ext_slope_central_weights", "+ (h2 - h1) / (h1 * h2) * sa[k] +", "+ (h1 - h2) / (h1 * h2) * sa[k] +"),
]


def _pin_calls():
    calls = []
    for name in dir(pins):
        fn = getattr(pins, name)
        if not name.startswith("test_") or not callable(fn):
            continue
        marks = [m.name for m in getattr(fn, "pytestmark", [])]
        if "slow" in marks:
            continue
        if name == "test_tvd_reading_davis_split_form_is_tvd":
            calls += [(f"{name}[{c}]", (lambda c=c, fn=fn: fn(c))) for c in (0.1, 0.2, 0.25, 0.4)]
        elif name == "test_xy_exchange_symmetry_3d":
            calls += [(f"{name}[{d}]", (lambda d=d, m=m, fn=fn: fn(d, m))) for d, m in ((1, 0), (0, 1), (2, 2))]
        elif name == "test_stretched_z_contact_tvd_flux_by_hand":
            calls += [(f"{name}[{b}]", (lambda b=b, fn=fn: fn(b))) for b in (1.5, 2.5)]
        elif name == "test_single_sweep_on_contact_step_by_hand":
            calls += [(f"{name}[{d}]", (lambda d=d, fn=fn: fn(d))) for d in (0.006, 0.012)]
        elif name == "test_sound_damping_pins_stokes_reading":
            calls += [(f"{name}[-]", lambda fn=fn: fn(-2.0 / 3.0, True)),
                      (f"{name}[+]", lambda fn=fn: fn(2.0 / 3.0, False))]
        else:
            calls.append((name, fn))
    return calls


def test_pins_pass_on_unmutated_oracle_copy(tmp_path):
    lib = _build(tmp_path, open(SRC).read(), "clean")
    with O.library(lib):
        failed = [n for n, fn in _pin_calls() if not _passes(fn)]
    assert failed == []


def _build(tmp, src, tag):
    c = os.path.join(tmp, f"m_{tag}.c")
    so = os.path.join(tmp, f"m_{tag}.so")
    with open(c, "w") as f:
        f.write(src)
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", so, c, "-lm"],
                   check=True)
    return so


def _passes(fn):
    try:
        fn()
        return True
    except (AssertionError, FloatingPointError, ValueError, OverflowError, ZeroDivisionError):
        return False


# a mutated oracle may produce empty or non-finite fields (a mean of nothing,
# an overflow): numpy's warnings about them are expected here
@pytest.mark.filterwarnings("ignore::RuntimeWarning")
@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    lib = _build(tmp_path, src.replace(old, new), name)
    import numpy as np
    with O.library(lib), np.errstate(all="ignore"):
        caught = [n for n, fn in _pin_calls() if not _passes(fn)]
    print(name, "caught by", caught)
    assert caught, f"no pin fails on mutant {name}"
