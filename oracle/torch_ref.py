"""Plain PyTorch (CPU, float64) restatement of the 2D step of Sec. 3.1, for the
reverse-mode checks: torch.autograd differentiates it.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): imported by tests/ and
nothing else.  It shares no code with the CUDA path and is pinned to the C
oracle (tests/test_torch_ref_pins.py): same states step by step, same Nu_bar.

The step is written from the paper like oracle/cm_oracle.c (Sec. 2 closures;
Sec. 3.1 predictor with forward differences along the sweep, corrector with
backward ones, central differences across, average, TVD term in the Davis
form; Eq. time_step splitting L_x L_z L_x L_z at dt/2), on whole arrays.  Each
step's dt is an input (the adjoint treats dt as a constant).  Non-smooth
points are written with torch.where so that autograd takes the same one-sided
derivatives as the library: phi'(r) = 2 only on 0 < 2r < 1, d|u|/du = 0 at 0,
the Co(1 - Co) branch at Co = 1/2, and the first argument on a tie of
max(A_k, A_k+1).  With frozen_phi the ratios r enter as constants (phi' = 0),
the library's second reading of the limiter's derivative.

On a stretched z-grid (znodes: the nz plane heights, Sec. 3) the z sweep is
written in conservative form as in the C oracle: the flux differences of
plane k over its cell width w_k (half cells on the plates), one-sided
derivatives over the spacing they span, TVD fluxes weighted by spacing over
width with the Courant number over the interface spacing; the x sweep's
central z-differences over the distance of the two planes they use; the plate
Nusselt numbers from the derivative of the quadratic through three planes.
"""
from __future__ import annotations

import torch

TVD_SPLIT, TVD_SUM, TVD_OFF = 0, 1, 2


class Model:
    """The 2D box of aspect ratio `aspect` with nx periodic columns and nz
    planes including both plates (plate temperatures t_bot and t_top)."""

    def __init__(self, nx, nz, Pr=1.0, gamma=5.0 / 3.0, eps=0.1, D=0.5, aspect=4.0, gravity=1.0, t_bot=1.0,
                 t_top=None, stokes=-2.0 / 3.0, tvd_form=TVD_SPLIT, znodes=None, frozen_phi=False):
        self.nx, self.nz, self.K = nx, nz, nz - 1
        self.Pr, self.gamma, self.eps, self.D = Pr, gamma, eps, D
        self.a = (gamma - 1.0) / (gamma * eps * D)
        self.b = gamma * eps * D
        self.g = gravity / eps
        self.cs2 = gamma * self.a
        self.hx = aspect / nx
        self.hz = 1.0 / (nz - 1)
        self.stokes = stokes
        self.tvd_form = tvd_form
        # frozen_phi: autograd takes no derivative through the limiter's ratios
        # (the reverse-mode reading phi' = 0); the step's values are unchanged
        self.frozen_phi = frozen_phi
        t_top = (1.0 - eps - D) if t_top is None else t_top
        self.e_bot = t_bot / self.b + self.g * 0.0
        self.e_top = t_top / self.b + self.g * 1.0
        self.z = (torch.arange(nz, dtype=torch.float64) / (nz - 1))[:, None]
        self.stretched = znodes is not None
        if self.stretched:
            z = torch.as_tensor(znodes, dtype=torch.float64).reshape(nz)
            K = nz - 1
            hp = z[1:] - z[:-1]                              # spacing of interval k (planes k, k+1)
            w = torch.cat([hp[:1] / 2.0, (hp[:-1] + hp[1:]) / 2.0, hp[-1:] / 2.0])  # cell widths
            self.z = z[:, None]
            self.hp = hp[:, None]
            self.w = w[:, None]
            self.sc = (hp[:-1] + hp[1:])[:, None]            # central span of planes 1..K-1
            self.rp = (hp[1:K] / w[1:K])[:, None]            # TVD weights of planes 1..K-1
            self.rm = (hp[0:K - 1] / w[1:K])[:, None]

    # mu = sqrt(Pr/Ra), K = 1/(eps D sqrt(Ra Pr)) (Sec. 2)
    def coefs(self, Ra):
        Ra = torch.as_tensor(Ra, dtype=torch.float64)
        return torch.sqrt(self.Pr / Ra), 1.0 / (self.eps * self.D * torch.sqrt(Ra * self.Pr))

    def prims(self, X, z):
        r = X[0]
        ux = X[1] / r
        uz = X[2] / r
        T = self.b * (X[3] / r - 0.5 * (ux * ux + uz * uz) - self.g * z)
        return ux, uz, T, self.a * r * T

    def _flux(self, q, ua, uc, p, daa, dac, daT, dca, dcc, along_z, mu, kth):
        """F_al in 2D by components along (a) and across (c) the sweep:
        [m_a ; m_a u_a - tau_a + p ; m_c u_a - tau_c ; u_a (E + p) - K dT/da - u.tau_a],
        tau_a = mu (2 d_a u_a + s div u), tau_c = mu (d_a u_c + d_c u_a)."""
        fa, fc = (2, 1) if along_z else (1, 2)
        div = daa + dcc
        ta = mu * ((daa + daa) + self.stokes * div)
        tc = mu * (dac + dca)
        tx, tz = (tc, ta) if along_z else (ta, tc)
        ux, uz = (uc, ua) if along_z else (ua, uc)
        F = [None] * 4
        F[0] = q[fa]
        F[fa] = (q[fa] * ua - ta) + p
        F[fc] = q[fc] * ua - tc
        F[3] = (ua * (q[3] + p) - kth * daT) - (ux * tx + uz * tz)
        return torch.stack(F)

    def _tvd(self, dm, d0, dp, A0, A1, Delta, h):
        """D = G dX_{k+1/2} at each interface (all inputs per interface)."""
        def dot(u, v):
            return ((u[0] * v[0] + u[1] * v[1]) + u[2] * v[2]) + u[3] * v[3]
        if self.tvd_form == TVD_OFF:
            return torch.zeros_like(d0)
        sp, sm, dd = dot(dm, d0), dot(d0, dp), dot(d0, d0)
        if self.frozen_phi:
            sp, sm, dd = sp.detach(), sm.detach(), dd.detach()
        zero = dd == 0.0
        safe = torch.where(zero, torch.ones_like(dd), dd)
        rp, rm = sp / safe, sm / safe
        Amax = torch.where(A0 >= A1, A0, A1)
        Co = Delta * Amax / h
        C = torch.where(Co <= 0.5, Co * (1.0 - Co), torch.full_like(Co, 0.25))

        def phi(r):
            r2 = 2.0 * r
            return torch.where(r2 <= 0.0, torch.zeros_like(r2), torch.where(r2 >= 1.0, torch.ones_like(r2), r2))
        if self.tvd_form == TVD_SPLIT:
            G = 0.5 * C * (1.0 - phi(rp)) + 0.5 * C * (1.0 - phi(rm))
        else:
            G = 0.5 * C * (1.0 - phi(rp + rm))
        G = torch.where(zero, torch.zeros_like(G), G)
        return G * d0

    def sweep_z(self, X, Delta, mu, kth):
        K, hz, hx = self.K, self.hz, self.hx
        st = self.stretched
        # Delta / w on the interior planes and on the two plate half cells
        lam = Delta / self.w[1:K] if st else Delta / hz
        lam_b = Delta / self.w[0, 0] if st else 2.0 * (Delta / hz)
        lam_t = Delta / self.w[K, 0] if st else 2.0 * (Delta / hz)
        ux, uz, T, p = self.prims(X, self.z)
        A = torch.abs(uz) + torch.sqrt(self.cs2 * T)

        def dxc(f):
            return (torch.roll(f, -1, -1) - torch.roll(f, 1, -1)) / (2.0 * hx)

        def dzf(f):  # forward along z on planes 0..K-1 (= backward on 1..K)
            return (f[1:] - f[:-1]) / (self.hp if st else hz)
        # F^n on planes 0..K-1
        F = self._flux(X[:, :K], uz[:K], ux[:K], p[:K], dzf(uz), dzf(ux), dzf(T), dxc(uz)[:K], dxc(ux)[:K], True,
                       mu, kth)
        S = torch.zeros_like(X[:, 1:K])
        S = torch.stack([S[0], S[1], -self.g * X[0, 1:K], S[3]])
        XPi = X[:, 1:K] - lam * (F[:, 1:K] - F[:, 0:K - 1]) + Delta * S
        r0 = X[0, 0] - lam_b * F[0, 0]
        rK = X[0, K] + lam_t * F[0, K - 1]
        zr = torch.zeros_like(r0)
        P0 = torch.stack([r0, zr, zr, r0 * self.e_bot])[:, None]
        PK = torch.stack([rK, zr, zr, rK * self.e_top])[:, None]
        XP = torch.cat([P0, XPi, PK], dim=1)
        uxp, uzp, Tp, pp = self.prims(XP, self.z)
        # F^P on planes 1..K
        FP = self._flux(XP[:, 1:], uzp[1:], uxp[1:], pp[1:], dzf(uzp), dzf(uxp), dzf(Tp), dxc(uzp)[1:],
                        dxc(uxp)[1:], True, mu, kth)
        SP = torch.stack([S[0], S[1], -self.g * XP[0, 1:K], S[3]])
        XC = X[:, 1:K] - lam * (FP[:, 1:K] - FP[:, 0:K - 1]) + Delta * SP
        Y1 = (XPi + XC) / 2.0
        y0 = (XP[0, 0] + (X[0, 0] - lam_b * FP[0, 0])) / 2.0
        yK = (XP[0, K] + X[0, K]) / 2.0
        # TVD fluxes at interfaces k + 1/2, k = 1..K-2 (zero at the plate-adjacent ones)
        dm = X[:, 1:K - 1] - X[:, 0:K - 2]
        d0 = X[:, 2:K] - X[:, 1:K - 1]
        dp = X[:, 3:K + 1] - X[:, 2:K]
        Dk = self._tvd(dm, d0, dp, A[1:K - 1], A[2:K], Delta, self.hp[1:K - 1] if st else hz)
        zrow = torch.zeros_like(X[:, :1])
        Dall = torch.cat([zrow, Dk, zrow], dim=1)  # interfaces 0..K-1
        if st:
            Yi = Y1 + (self.rp * Dall[:, 1:K] - self.rm * Dall[:, 0:K - 1])
        else:
            Yi = Y1 + (Dall[:, 1:K] - Dall[:, 0:K - 1])
        B0 = torch.stack([y0, zr, zr, y0 * self.e_bot])[:, None]
        BK = torch.stack([yK, zr, zr, yK * self.e_top])[:, None]
        return torch.cat([B0, Yi, BK], dim=1)

    def sweep_x(self, X, Delta, mu, kth):
        K, hz, hx = self.K, self.hz, self.hx
        lam = Delta / hx
        ux, uz, T, p = self.prims(X, self.z)
        A = torch.abs(ux) + torch.sqrt(self.cs2 * T)
        Xi = X[:, 1:K]

        def dzc(f):  # central along z on rows 1..K-1
            return (f[2:] - f[:-2]) / (self.sc if self.stretched else 2.0 * hz)

        def dxf(f):
            return (torch.roll(f, -1, -1) - f) / hx

        def dxb(f):
            return (f - torch.roll(f, 1, -1)) / hx
        F = self._flux(Xi, ux[1:K], uz[1:K], p[1:K], dxf(ux[1:K]), dxf(uz[1:K]), dxf(T[1:K]), dzc(ux), dzc(uz),
                       False, mu, kth)
        XPi = Xi - lam * (F - torch.roll(F, 1, -1))
        XP = torch.cat([X[:, :1], XPi, X[:, K:]], dim=1)
        uxp, uzp, Tp, pp = self.prims(XP, self.z)
        FP = self._flux(XPi, uxp[1:K], uzp[1:K], pp[1:K], dxb(uxp[1:K]), dxb(uzp[1:K]), dxb(Tp[1:K]), dzc(uxp),
                        dzc(uzp), False, mu, kth)
        XC = Xi - lam * (torch.roll(FP, -1, -1) - FP)
        Y1 = (XPi + XC) / 2.0
        dm = Xi - torch.roll(Xi, 1, -1)
        d0 = torch.roll(Xi, -1, -1) - Xi
        dp = torch.roll(Xi, -2, -1) - torch.roll(Xi, -1, -1)
        Ai = A[1:K]
        D = self._tvd(dm, d0, dp, Ai, torch.roll(Ai, -1, -1), Delta, hx)
        Yi = Y1 + (D - torch.roll(D, 1, -1))
        return torch.cat([X[:, :1], Yi, X[:, K:]], dim=1)

    def step(self, X, dt, mu, kth):
        """X^{n+1} = L_x L_z L_x L_z X^n, every sweep at dt/2 (Eq. time_step)."""
        D = 0.5 * dt
        for _ in range(2):
            X = self.sweep_x(self.sweep_z(X, D, mu, kth), D, mu, kth)
        return X

    def nu_bar(self, X):
        """(Nu_0 + Nu_1)/2 of Eq. mean_Nu: second-order one-sided plate
        differences of the x-mean temperature minus 1 - D z."""
        _, _, T, _ = self.prims(X, self.z)
        K, dz = self.K, self.hz
        if self.stretched:
            z = self.z[:, 0]
            f = [T[q].sum() / self.nx - (1.0 - self.D * z[q]) for q in range(3)]
            g = [T[K - q].sum() / self.nx - (1.0 - self.D * z[K - q]) for q in range(3)]

            def d3(v, h1, h2):  # derivative at the first of three planes h1, h1 + h2 apart
                return (-(2.0 * h1 + h2) / (h1 * (h1 + h2)) * v[0] + (h1 + h2) / (h1 * h2) * v[1]
                        - h1 / (h2 * (h1 + h2)) * v[2])
            nb = -(1.0 / self.eps) * d3(f, z[1] - z[0], z[2] - z[1])
            nt = (1.0 / self.eps) * d3(g, z[K] - z[K - 1], z[K - 1] - z[K - 2])
            return (nb + nt) / 2.0
        f = [T[q].sum() / self.nx - (1.0 - self.D * (q / K)) for q in range(3)]
        g = [T[K - q].sum() / self.nx - (1.0 - self.D * ((K - q) / K)) for q in range(3)]
        nb = -(1.0 / self.eps) * (-3.0 * f[0] + 4.0 * f[1] - f[2]) / (2.0 * dz)
        nt = -(1.0 / self.eps) * (3.0 * g[0] - 4.0 * g[1] + g[2]) / (2.0 * dz)
        return (nb + nt) / 2.0

    def objective(self, X0, Ra, dts, win_begin):
        """J = mean of Nu_bar(X^n) over n = win_begin..len(dts) (1-based steps)."""
        mu, kth = self.coefs(Ra)
        X, acc, cnt = X0, 0.0, 0
        for n, dt in enumerate(dts, start=1):
            X = self.step(X, dt, mu, kth)
            if n >= win_begin:
                acc = acc + self.nu_bar(X)
                cnt += 1
        return acc / cnt

    def states(self, X0, Ra, dts):
        mu, kth = self.coefs(Ra)
        X, out = X0, []
        for dt in dts:
            X = self.step(X, dt, mu, kth)
            out.append(X)
        return out


def isobaric_state(model: Model, T, p, ux=None, uz=None):
    """State (rho, m_x, m_z, E) from temperature T and pressure p (fields or
    profiles broadcast to (nz, nx)), velocity zero unless given."""
    T = torch.as_tensor(T, dtype=torch.float64)
    rho = p / (model.a * T)
    ux = torch.zeros_like(rho) if ux is None else ux
    uz = torch.zeros_like(rho) if uz is None else uz
    E = rho * (0.5 * (ux * ux + uz * uz) + T / model.b + model.g * model.z)
    return torch.stack([rho, rho * ux, rho * uz, E])

