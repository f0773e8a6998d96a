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
    C.layout_exact = P.layout_exact;
    C.zp = nullptr;
}

// Plane heights of the z-grid: uniform (k/K), the tanh grid of Sec. 3 with
// stretching beta = G.zstretch,
//   z_k = (1 + tanh(beta (2k/K - 1)) / tanh(beta)) / 2,
// or the planes G.znodes given by the caller.  Returns false (with a reason)
// for an invalid request.
inline bool make_planes(const cm_grid& G, std::vector<double>& z, const char** why)
{
    const int nz = G.nz, K = nz - 1;
    z.assign(nz, 0.0);
    if (G.znodes) {
        for (int k = 0; k < nz; ++k) z[k] = G.znodes[k];
        if (z[0] != 0.0 || z[K] != 1.0) { *why = "znodes must start at exactly 0 and end at exactly 1"; return false; }
        for (int k = 0; k < K; ++k)
            if (!(z[k + 1] > z[k]) || !std::isfinite(z[k + 1])) { *why = "znodes must be finite and strictly increasing"; return false; }
        return true;
    }
    if (!(G.zstretch >= 0.0) || !std::isfinite(G.zstretch) || G.zstretch > 20.0) {
        *why = "zstretch must be in [0, 20]";
        return false;
    }
    for (int k = 0; k < nz; ++k) {
        if (G.zstretch == 0.0) z[k] = (double)k / (double)K;
        else if (k == 0) z[k] = 0.0;
        else if (k == K) z[k] = 1.0;
        else {
            const double s = 2.0 * k / K - 1.0;
            z[k] = 0.5 * (1.0 + std::tanh(G.zstretch * s) / std::tanh(G.zstretch));
        }
    }
    for (int k = 0; k < K; ++k)
        if (!(z[k + 1] > z[k])) { *why = "zstretch too large for nz: two planes coincide in FP64"; return false; }
    return true;
}

inline bool stretched(const cm_grid& G) { return G.znodes != nullptr || G.zstretch != 0.0; }

// per-plane metric of the planes z (see Plane), FP64 values rounded once to R
template <class R>
void plane_table(const std::vector<double>& z, std::vector<Plane<R>>& t)
{
    const int nz = (int)z.size(), K = nz - 1;
    std::vector<double> hp(nz);
    for (int k = 0; k < K; ++k) hp[k] = z[k + 1] - z[k];
    hp[K] = hp[K - 1];
    t.assign(nz, Plane<R>{});
    for (int k = 0; k < nz; ++k) {
        const double hm = k > 0 ? hp[k - 1] : hp[0];
        const double w = k == 0 ? hp[0] / 2.0 : (k == K ? hp[K - 1] / 2.0 : (hp[k - 1] + hp[k]) / 2.0);
        const double sc = (k > 0 && k < K) ? hp[k - 1] + hp[k] : 2.0 * hp[k];
        const double hmin = k == 0 ? hp[0] : (k == K ? hp[K - 1] : std::fmin(hp[k - 1], hp[k]));
        Plane<R>& P = t[k];
        P.hp = (R)hp[k];
        P.ihp = (R)(1.0 / hp[k]);
        P.w = (R)w;
        P.iw = (R)(1.0 / w);
        P.rp = (R)(hp[k] / w);
        P.rm = (R)(hm / w);
        P.sc = (R)sc;
        P.isc = (R)(1.0 / sc);
        P.hmin = (R)hmin;
        P.ihmin = (R)(1.0 / hmin);
        P.z = (R)z[k];
        P.pad = R(0);
    }
}

// conduction / hydrostatic profile of constant K, FP64 (nz values):
// T linear between the plate temperatures, dp/dz = -g rho, p = a rho T, rho(0) = 1
struct Profile {
    std::vector<double> z, Tc, pc;
    double rho_min;
    Profile(int nz, const cm_params& P, const Closure& K) : Profile(uniform(nz), P, K) {}
    Profile(const std::vector<double>& planes, const cm_params& P, const Closure& K)
        : z(planes), Tc(planes.size()), pc(planes.size()), rho_min(1e300)
    {
        const int nz = (int)planes.size();
        const double Lam = P.t_bot - P.t_top;
        for (int k = 0; k < nz; ++k) {
            Tc[k] = P.t_bot - Lam * z[k];
            if (Lam != 0.0) pc[k] = K.a * P.t_bot * std::pow(Tc[k] / P.t_bot, K.g / (K.a * Lam));
            else pc[k] = K.a * P.t_bot * std::exp(-K.g * z[k] / (K.a * P.t_bot));
            rho_min = std::fmin(rho_min, pc[k] / (K.a * Tc[k]));
        }
    }
    static std::vector<double> uniform(int nz)
    {
        std::vector<double> u(nz);
        for (int k = 0; k < nz; ++k) u[k] = (double)k / (double)(nz - 1);
        return u;
    }
};

// Diffusion number of the explicit viscous / conduction terms at step dt:
// nu = max(4/3 mu, K b) / min rho over the smallest spacing h (x or z),
// nu (dt/2) / h^2 (each sweep advances by dt/2).  Above 0.5 the explicit
// sweeps are unstable.
inline double diffusion_number(const cm_grid& G, const std::vector<double>& planes, double Ra, double Pr,
                               const cm_params& P, const Closure& K, double rho_min, double dt)
{
    const double mu = std::sqrt(Pr / Ra), kth = 1.0 / (P.eps * P.D * std::sqrt(Ra * Pr));
    const double nu = std::fmax(4.0 / 3.0 * mu, kth * K.b) / rho_min;
    double hz = 1.0 / (double)(planes.size() - 1);
    for (size_t k = 0; k + 1 < planes.size(); ++k) hz = std::fmin(hz, planes[k + 1] - planes[k]);
    const double hh = std::fmin(G.aspect / G.nx, hz);
    return nu * 0.5 * dt / (hh * hh);
}

int pitch_of(int nx, int prec);

}  // namespace cm
