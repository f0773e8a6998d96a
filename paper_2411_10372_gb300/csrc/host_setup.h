// host_setup.h -- host-side set-up shared by the single-solver and the batch
// contexts: coefficients of the nondimensional equations (Sec. 2) in the
// state precision, and the conduction / hydrostatic profile of constant K.
#pragma once
#include <cmath>
#include <vector>

#include "../../include/cm.h"
#include "cm_device.cuh"

namespace cm {

// a = (gamma-1)/(gamma eps D) (p = a rho T), b = gamma eps D, g = gravity/eps, cs2 = gamma a
struct Closure {
    double a, b, g, cs2;
    Closure(double gamma, const cm_params& P)
        : a((gamma - 1.0) / (gamma * P.eps * P.D)), b(gamma * P.eps * P.D), g(P.gravity / P.eps),
          cs2(gamma * ((gamma - 1.0) / (gamma * P.eps * P.D)))
    {
    }
};

template <class R>
void fill_coef(Coef<R>& C, const cm_grid& G, int ny, int pitch, long long fstride, double Ra, double Pr,
               const Closure& K, const cm_params& P)
{
    const double dx = G.aspect / G.nx, dy = G.aspect / ny, dz = 1.0 / (G.nz - 1);
    C.a = (R)K.a;
    C.b = (R)K.b;
    C.g = (R)K.g;
    C.mu = (R)std::sqrt(Pr / Ra);
    C.kth = (R)(1.0 / (P.eps * P.D * std::sqrt(Ra * Pr)));
    C.cs2 = (R)K.cs2;
    C.stokes = (R)P.stokes;
    C.inv_dx = (R)(1.0 / dx);
    C.inv_dy = (R)(1.0 / dy);
    C.inv_dz = (R)(1.0 / dz);
    C.inv_2dx = (R)(1.0 / (2.0 * dx));
    C.inv_2dy = (R)(1.0 / (2.0 * dy));
    C.inv_2dz = (R)(1.0 / (2.0 * dz));
    C.hx = (R)dx;
    C.hy = (R)dy;
    C.hz = (R)dz;
    C.h2x = (R)(2.0 * dx);
    C.h2y = (R)(2.0 * dy);
    C.h2z = (R)(2.0 * dz);
    C.ebot = (R)(P.t_bot / K.b + K.g * 0.0);
    C.etop = (R)(P.t_top / K.b + K.g * 1.0);
    C.dx = dx;
    C.dy = dy;
    C.dz = dz;
    C.cfl = P.cfl;
    C.dt_fixed = P.dt_fixed;
    C.nx = G.nx;
    C.ny = ny;
    C.nz = G.nz;
    C.pitch = pitch;
    C.fstride = fstride;
    C.tvd_form = P.tvd_form;
    C.ndim = G.ndim;
}

// conduction / hydrostatic profile of constant K, FP64 (nz values):
// T linear between the plate temperatures, dp/dz = -g rho, p = a rho T, rho(0) = 1
struct Profile {
    std::vector<double> z, Tc, pc;
    double rho_min;
    Profile(int nz, const cm_params& P, const Closure& K) : z(nz), Tc(nz), pc(nz), rho_min(1e300)
    {
        const double Lam = P.t_bot - P.t_top;
        for (int k = 0; k < nz; ++k) {
            z[k] = (double)k / (double)(nz - 1);
            Tc[k] = P.t_bot - Lam * z[k];
            if (Lam != 0.0) pc[k] = K.a * P.t_bot * std::pow(Tc[k] / P.t_bot, K.g / (K.a * Lam));
            else pc[k] = K.a * P.t_bot * std::exp(-K.g * z[k] / (K.a * P.t_bot));
            rho_min = std::fmin(rho_min, pc[k] / (K.a * Tc[k]));
        }
    }
};

int pitch_of(int nx, int prec);

}  // namespace cm
