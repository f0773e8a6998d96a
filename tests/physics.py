"""Closed forms and textbook routines the oracle is pinned against.

Everything here is written from the mathematics (nondimensional closures of
Sec. 2 of arXiv 2411.10372, linear acoustics, the exact Riemann solver for an
ideal gas) and never from the oracle's code.
"""
from __future__ import annotations

import math

import numpy as np


def closures(gamma, eps, D, Ra, Pr):
    """p = a rho T, e = T/b, mu, K, c_p of the nondimensional equations."""
    a = (gamma - 1.0) / (gamma * eps * D)
    b = gamma * eps * D
    mu = math.sqrt(Pr / Ra)
    K = 1.0 / (eps * D * math.sqrt(Ra * Pr))
    cv = 1.0 / b
    cp = cv + a           # R = a for p = rho R T
    return dict(a=a, b=b, mu=mu, K=K, cv=cv, cp=cp)


def state_from_prims(cfg, rho, ux, uz, T, z=None, uy=None):
    """Conserved 2D/3D state from primitive fields (gravity potential g z)."""
    c = closures(cfg.gamma, cfg.eps, cfg.D, cfg.Ra, cfg.Pr)
    g = cfg.gravity / cfg.eps
    if z is None:
        z = np.zeros_like(rho)
    if uy is None:
        uy = np.zeros_like(rho)
    E = rho * (0.5 * (ux * ux + uy * uy + uz * uz) + T / c["b"] + g * z)
    if cfg.ndim == 3:
        return np.stack([rho, rho * ux, rho * uy, rho * uz, E]).astype(np.float64)
    return np.stack([rho, rho * ux, rho * uz, E]).astype(np.float64)


def prims_from_state(cfg, X, z=None):
    c = closures(cfg.gamma, cfg.eps, cfg.D, cfg.Ra, cfg.Pr)
    g = cfg.gravity / cfg.eps
    rho = X[0]
    if cfg.ndim == 3:
        ux, uy, uz, E = X[1] / rho, X[2] / rho, X[3] / rho, X[4]
    else:
        ux, uz, E = X[1] / rho, X[2] / rho, X[3]
        uy = np.zeros_like(rho)
    if z is None:
        z = np.zeros_like(rho)
    T = c["b"] * (E / rho - 0.5 * (ux * ux + uy * uy + uz * uz) - g * z)
    return rho, ux, uy, uz, T, c["a"] * rho * T


def mode(f, axis=-1, k=1):
    """Complex Fourier coefficient of wavenumber index k along a periodic axis."""
    n = f.shape[axis]
    return np.fft.fft(f, axis=axis).take(k, axis=axis) / n * 2.0


def sine_mode(f, z, m=1):
    """Projection of f(z) (nodes on both plates) on sin(m pi z), trapezoid rule."""
    w = np.ones_like(z)
    w[0] = w[-1] = 0.5
    s = np.sin(m * np.pi * z)
    return float(np.sum(w * f * s) / np.sum(w * s * s))


def total_variation(u):
    return float(np.sum(np.abs(np.roll(u, -1) - u)))


# ---- exact Riemann solver for the ideal-gas Euler equations (Toro, ch. 4) ----
def _f_side(p, rhoK, pK, cK, gamma):
    if p > pK:  # shock
        A = 2.0 / ((gamma + 1.0) * rhoK)
        B = (gamma - 1.0) / (gamma + 1.0) * pK
        f = (p - pK) * math.sqrt(A / (p + B))
        df = math.sqrt(A / (B + p)) * (1.0 - 0.5 * (p - pK) / (B + p))
    else:       # rarefaction
        pr = p / pK
        f = 2.0 * cK / (gamma - 1.0) * (pr ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)
        df = 1.0 / (rhoK * cK) * pr ** (-(gamma + 1.0) / (2.0 * gamma))
    return f, df


def riemann_exact(rl, ul, pl, rr, ur, pr, gamma, xi):
    """Density, velocity, pressure at similarity coordinates xi = x/t."""
    cl = math.sqrt(gamma * pl / rl)
    cr = math.sqrt(gamma * pr / rr)
    p = 0.5 * (pl + pr)
    for _ in range(100):
        fl, dfl = _f_side(p, rl, pl, cl, gamma)
        fr, dfr = _f_side(p, rr, pr, cr, gamma)
        pn = p - (fl + fr + ur - ul) / (dfl + dfr)
        pn = max(pn, 1e-12)
        if abs(pn - p) < 1e-14 * p:
            p = pn
            break
        p = pn
    fl, _ = _f_side(p, rl, pl, cl, gamma)
    fr, _ = _f_side(p, rr, pr, cr, gamma)
    us = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    g1 = (gamma - 1.0) / (gamma + 1.0)
    out = np.zeros((3, len(xi)))
    for n, s in enumerate(xi):
        if s <= us:  # left of contact
            if p > pl:
                sl = ul - cl * math.sqrt((gamma + 1) / (2 * gamma) * p / pl + (gamma - 1) / (2 * gamma))
                if s <= sl:
                    out[:, n] = (rl, ul, pl)
                else:
                    out[:, n] = (rl * (p / pl + g1) / (g1 * p / pl + 1), us, p)
            else:
                shl = ul - cl
                cls = cl * (p / pl) ** ((gamma - 1) / (2 * gamma))
                stl = us - cls
                if s <= shl:
                    out[:, n] = (rl, ul, pl)
                elif s >= stl:
                    out[:, n] = (rl * (p / pl) ** (1 / gamma), us, p)
                else:
                    c = 2 / (gamma + 1) * (cl + (gamma - 1) / 2 * (ul - s))
                    u = 2 / (gamma + 1) * (cl + (gamma - 1) / 2 * ul + s)
                    r = rl * (c / cl) ** (2 / (gamma - 1))
                    out[:, n] = (r, u, pl * (c / cl) ** (2 * gamma / (gamma - 1)))
        else:
            if p > pr:
                sr = ur + cr * math.sqrt((gamma + 1) / (2 * gamma) * p / pr + (gamma - 1) / (2 * gamma))
                if s >= sr:
                    out[:, n] = (rr, ur, pr)
                else:
                    out[:, n] = (rr * (p / pr + g1) / (g1 * p / pr + 1), us, p)
            else:
                shr = ur + cr
                crs = cr * (p / pr) ** ((gamma - 1) / (2 * gamma))
                str_ = us + crs
                if s >= shr:
                    out[:, n] = (rr, ur, pr)
                elif s <= str_:
                    out[:, n] = (rr * (p / pr) ** (1 / gamma), us, p)
                else:
                    c = 2 / (gamma + 1) * (cr - (gamma - 1) / 2 * (ur - s))
                    u = 2 / (gamma + 1) * (-cr + (gamma - 1) / 2 * ur + s)
                    r = rr * (c / cr) ** (2 / (gamma - 1))
                    out[:, n] = (r, u, pr * (c / cr) ** (2 * gamma / (gamma - 1)))
    return out
