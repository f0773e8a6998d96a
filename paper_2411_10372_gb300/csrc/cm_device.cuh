// cm_device.cuh -- device-side building blocks of the MacCormack-TVD sweeps.
//
// Physics (arXiv 2411.10372, Sec. 2, nondimensional form):
//   p = a rho T,  a = (gamma-1)/(gamma eps D)
//   E = rho (u^2/2 + T/b + g z),  b = gamma eps D,  g = (gravity factor)/eps
//   tau_ij = mu (d_j u_i + d_i u_j + s (div u) delta_ij),  mu = sqrt(Pr/Ra), s = -2/3
//   heat flux -K grad T,  K = 1/(eps D sqrt(Ra Pr))
// Scheme (Sec. 3.1): flux F_alpha = [m_alpha; m_i u_alpha - tau_{i alpha} + p delta_{i alpha};
//   u_alpha (E + p) - K dT/dx_alpha - u_b tau_{b alpha}], source -g rho in the z momentum.
//
// Rounding: the FP64 instantiation evaluates every formula as a fixed
// sequence of IEEE operations -- true divisions by the grid spacings and by
// rho, no FMA contraction (its translation unit is built with --fmad=false),
// sums in the order the formulas are written -- so the FP64 path is
// reproducible bit for bit (the flow amplifies a one-ulp change at one node
// to ~1e-6 in 1000 steps at Ra = 1e6, so nothing looser is testable).  The
// FP32 instantiation multiplies by precomputed reciprocals instead.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <type_traits>

namespace cm {

// Coefficients of one solver instance in the state precision R (the dt rule
// stays in FP64).
// Metric of one z plane of a non-uniform grid (the tanh grid of Sec. 3, or
// any given planes), in the state precision.  hp: spacing to the plane
// above, z_{k+1} - z_k; w: width of the plane's cell, (hp_{k-1} + hp_k)/2
// (hp/2 on the plates); rp, rm: hp_k / w_k and hp_{k-1} / w_k, the weights of
// the TVD fluxes above and below; sc: hp_{k-1} + hp_k, the span of a central
// difference; hmin: the smaller spacing next to the plane (CFL); i*: the
// reciprocals; z: the height.  Plate rows hold harmless values where a
// quantity does not exist.
template <class R>
struct alignas(16) Plane {
    R hp, ihp, w, iw;
    R rp, rm, sc, isc;
    R hmin, ihmin, z, pad;
};

template <class R>
struct Coef {
    R a, b, g, mu, kth, cs2, stokes;   // closures; cs2 = gamma a (c^2 = cs2 T)
    R inv_dx, inv_dy, inv_dz;          // 1/h
    R inv_2dx, inv_2dy, inv_2dz;       // 1/(2h)
    R hx, hy, hz, h2x, h2y, h2z;       // h and 2h (FP64 path divides by these)
    R ebot, etop;                      // E/rho on the plates: T_w/b + g z_w
    double dx, dy, dz, cfl, dt_fixed;
    int nx, ny, nz, pitch;             // nodes; row pitch in elements
    long long fstride;                 // elements between two fields
    int tvd_form, ndim;
    const Plane<R>* zp;                // per-plane metric of a stretched z-grid; nullptr = uniform planes
    int layout_exact;                  // FP32 2D: layout-independent sweeps (cm_params.layout_exact)
    int pad_;
};

// Device control block: dt slots (raw min of h/(|u|+c) as IEEE bits, so that
// an unsigned 64-bit atomicMin orders them), simulated time, completed steps,
// sticky status.
struct DevCtl {
    unsigned long long dt_slot[2];
    double t;
    double steps;
    int status;   // bit 0: non-finite value met
    int pad;
};

struct SweepCtl {
    DevCtl* ctl;
    int slot_in;      // dt slot this step reads
    int first;        // first sweep of a step: reset the other slot, advance t
    int last;         // last sweep of a step: reduce dt of the new state
    double Delta;     // > 0: use this Delta (single-sweep calls); else dt/2 from the slot
};


// ---- launch geometry and argument blocks shared by host and device code ----
constexpr int kWarpsPerBlock = 4;
constexpr int kOutW = 28;  // output columns per warp strip
constexpr int kDiagQ = 8;  // per-plane sums: rho, E, rho uz Tsa, rho uz u^2, u^2, rho u^2/2, T, max Mach
constexpr int kDiagThreads = 256;


struct InitArgs {
    const double* Tc;   // conduction temperature of each plane
    const double* pc;   // conduction pressure of each plane
    const double* zt;   // z of each plane
    double a, b, g, amp;
    unsigned long long seed;
    const double* Tfield = nullptr;  // dense [nz][ny][nx] interior temperatures replacing Tc + amp xi (or NULL)
};

struct DiagArgs {
    const double* zt;
    double a, b, g, D, cs2;
};

struct DiagFinal {
    double Ra, Pr, eps, D, cfl, dt_fixed;
    double cells;       // nx * ny
    int nz;
    int slot;           // dt slot of the next step
    const Plane<double>* zp;  // stretched z-grid (trapezoid weights, plate derivatives); nullptr = uniform
};

// extended diagnostics (force terms of the z momentum equation, C(Ra),
// K_e/I_e histogram), FP64
constexpr int kExtMaxBins = 1024;
struct ExtArgs {
    const double* zt;                // plane heights
    double a, b, g, D, mu, stokes;   // closures and the Stokes coefficient
    double dx, dy;
    double lo, bw;                   // histogram of log10 r: lower edge and bin width
    int nbins;
    unsigned long long* hist;        // nbins counts (device; the caller zeroes it)
};

template <class R> struct St { R r, mx, mz, E; };       // 2D conserved state
template <class R> struct St3 { R r, mx, my, mz, E; };  // 3D conserved state

__device__ __forceinline__ float shup(float v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ float shdn(float v) { return __shfl_down_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shup(double v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shdn(double v) { return __shfl_down_sync(0xffffffffu, v, 1); }

template <class R> __device__ __forceinline__ St<R> shup(const St<R>& q) { return {shup(q.r), shup(q.mx), shup(q.mz), shup(q.E)}; }
template <class R> __device__ __forceinline__ St<R> shdn(const St<R>& q) { return {shdn(q.r), shdn(q.mx), shdn(q.mz), shdn(q.E)}; }

__device__ __forceinline__ float rsqrt_(float v) { return sqrtf(v); }
__device__ __forceinline__ double rsqrt_(double v) { return sqrt(v); }

// Programmatic dependent launch between the sweeps of a stream: wait until
// the previous kernel has finished and its writes are visible (before this
// kernel reads anything it wrote, dt slots included), then allow the next
// kernel to be scheduled while this one runs.  For a launch without the
// programmatic-serialization attribute both are no-ops.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}
// the wait alone (a second wait returns at once)
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

// dt as the kernels see it: fixed, or CFL times the slot's minimum
__device__ __forceinline__ double step_dt(const DevCtl* c, int slot, double cfl, double dt_fixed)
{
    if (dt_fixed > 0.0) return dt_fixed;
    return cfl * __longlong_as_double((long long)c->dt_slot[slot]);
}

template <class R> constexpr bool kExact = std::is_same<R, double>::value;

// (a - b) / span: a one-sided (span = h) or central (span = 2h) difference
template <class R>
__device__ __forceinline__ R diff(R a, R b, R span, R inv_span)
{
    if constexpr (kExact<R>) return (a - b) / span;
    else return (a - b) * inv_span;
}

// primitive variables from the conserved state (closures of Sec. 2)
template <class R>
__device__ __forceinline__ void prims(const St<R>& q, R z, const Coef<R>& C, R& ux, R& uz, R& T, R& p)
{
    if constexpr (kExact<R>) {
        ux = q.mx / q.r;
        uz = q.mz / q.r;
        T = C.b * (q.E / q.r - R(0.5) * (ux * ux + uz * uz) - C.g * z);
    } else {
        R ri = R(1) / q.r;
        ux = q.mx * ri;
        uz = q.mz * ri;
        T = C.b * (q.E * ri - R(0.5) * (ux * ux + uz * uz) - C.g * z);
    }
    p = C.a * q.r * T;
}

// local Courant number of an interface: (dt/2) max(|u|+c over its nodes) / h
template <class R>
__device__ __forceinline__ R courant(double Delta, R lam, R A0, R A1, R h)
{
    if constexpr (kExact<R>) return (R)Delta * fmax(A0, A1) / h;
    else return lam * fmax(A0, A1);
}

// F_z at one node; dz_* one-sided along z, dx_* central across
template <class R>
__device__ __forceinline__ St<R> flux_z(const St<R>& q, R ux, R uz, R p, R dz_ux, R dz_uz, R dz_T,
                                        R dx_ux, R dx_uz, const Coef<R>& C)
{
    R div = dx_ux + dz_uz;
    R tx = C.mu * (dz_ux + dx_uz);
    R tz = C.mu * ((dz_uz + dz_uz) + C.stokes * div);
    St<R> F;
    F.r = q.mz;
    F.mx = q.mx * uz - tx;
    F.mz = (q.mz * uz - tz) + p;
    F.E = (uz * (q.E + p) - C.kth * dz_T) - (ux * tx + uz * tz);
    return F;
}

// F_x at one node; dx_* one-sided along x, dz_* central across
template <class R>
__device__ __forceinline__ St<R> flux_x(const St<R>& q, R ux, R uz, R p, R dx_ux, R dx_uz, R dx_T,
                                        R dz_ux, R dz_uz, const Coef<R>& C)
{
    R div = dx_ux + dz_uz;
    R tx = C.mu * ((dx_ux + dx_ux) + C.stokes * div);
    R tz = C.mu * (dx_uz + dz_ux);
    St<R> F;
    F.r = q.mx;
    F.mx = (q.mx * ux - tx) + p;
    F.mz = q.mz * ux - tz;
    F.E = (ux * (q.E + p) - C.kth * dx_T) - (ux * tx + uz * tz);
    return F;
}

// minmod limiter phi(s/dd) = max(0, min(2 s/dd, 1)), dividing only where the
// result is strictly between 0 and 1 (dd = 0 implies s = 0, so phi = 0)
template <class R>
__device__ __forceinline__ R phi_of(R s, R dd)
{
    R s2 = s + s;
    return (s <= R(0)) ? R(0) : ((s2 >= dd) ? R(1) : s2 / dd);
}

// coefficient G of the TVD flux G * dX_{k+1/2}:
//   Davis form G(r+_k) + G(r-_{k+1}),  printed form G(r+_k + r-_{k+1}),
//   G(r) = C (1 - phi(r)) / 2,  C = Co (1 - Co) for Co <= 1/2, else 1/4,
//   r+_k = sp/dd, r-_{k+1} = sm/dd (dd = |dX_{k+1/2}|^2; dd = 0 means dX = 0,
//   where the flux vanishes whatever G is)
template <class R>
__device__ __forceinline__ R tvd_G(R sp, R sm, R dd, R Co, int form)
{
    R C = (Co <= R(0.5)) ? Co * (R(1) - Co) : R(0.25);
    if (form == 2) return R(0);
    if constexpr (kExact<R>) {
        if (dd == R(0)) return R(0);
        const R rp = sp / dd, rm = sm / dd;
        auto phi = [](R r) { return fmax(R(0), fmin(R(2) * r, R(1))); };
        if (form == 0) return R(0.5) * C * (R(1) - phi(rp)) + R(0.5) * C * (R(1) - phi(rm));
        return R(0.5) * C * (R(1) - phi(rp + rm));
    } else {
        if (form == 0) return R(0.5) * C * (R(1) - phi_of(sp, dd)) + R(0.5) * C * (R(1) - phi_of(sm, dd));
        return R(0.5) * C * (R(1) - phi_of(sp + sm, dd));
    }
}

template <class R>
__device__ __forceinline__ R dot4(const St<R>& a, const St<R>& b)
{
    return ((a.r * b.r + a.mx * b.mx) + a.mz * b.mz) + a.E * b.E;
}

// warp-wide min of a double and OR of a flag
__device__ __forceinline__ double warp_min(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// block reduction of the dt candidate and of the non-finite flag, then one
// atomic per block; every thread of the block must call it
__device__ __forceinline__ void block_dt_reduce(double v, int bad, DevCtl* ctl, int slot)
{
    __shared__ double sm[32];
    __shared__ int sb[32];
    v = warp_min(v);
    bad = __any_sync(0xffffffffu, bad);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { sm[w] = v; sb[w] = bad; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = sm[0];
        int b = sb[0];
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) { m = fmin(m, sm[i]); b |= sb[i]; }
        if (m < __longlong_as_double(0x7FF0000000000000LL))
            atomicMin(&ctl->dt_slot[slot], (unsigned long long)__double_as_longlong(m));
        if (b) atomicOr(&ctl->status, 1);
    }
}

}  // namespace cm
