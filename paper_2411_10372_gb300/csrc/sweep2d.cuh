// sweep2d.cuh -- fused 2D sweep kernels L_z(Delta) and L_x(Delta) of Sec. 3.1.
//
// One warp owns a strip of 32 columns and marches along z through a segment
// of rows, keeping the rows in flight in registers.  Lanes 2..29 produce the
// strip's 28 output columns; lanes 0,1,30,31 are the halo the x-stencil and
// the cross derivatives need (outputs of the neighbouring strips, recomputed).
// Columns are periodic, so lane columns wrap modulo nx.  Neighbour values
// across x travel by warp shuffle: no shared memory, no block barrier in the
// march.  Per node and sweep the kernel reads the input state once and
// writes the output state once (2 nf w bytes, the algorithmic minimum of a
// sweep); everything in between -- primitives, F^n, predictor, plate fill,
// F^P, corrector, average, TVD term, plate values -- stays in registers.
#pragma once
#include "cm_device.cuh"

namespace cm {


template <class R>
struct SweepIO {
    const R* in;
    R* out;
    const R* zt;     // z of each plane, in R
    int seg_rows;    // rows per warp segment
    int nstrips;     // ceil(nx / kOutW)
};

template <class R>
__device__ __forceinline__ St<R> load_row(const R* __restrict__ base, long long fs, int row, int pitch, int ic)
{
    const R* s = base + (size_t)row * pitch + ic;
    return {__ldg(s), __ldg(s + fs), __ldg(s + 2 * fs), __ldg(s + 3 * fs)};
}

template <class R>
__device__ __forceinline__ void store_row(R* __restrict__ base, long long fs, int row, int pitch, int i, const St<R>& q)
{
    R* d = base + (size_t)row * pitch + i;
    d[0] = q.r;
    d[fs] = q.mx;
    d[2 * fs] = q.mz;
    d[3 * fs] = q.E;
}

// dt candidate of one node of the new state, FP64 path: min over x, z of
// h/(|u|+c), evaluated as the CFL rule is written; hz: the node's z step
__device__ __forceinline__ double dt_candidate(const St<double>& q, double z, double hz, const Coef<double>& C, int& bad)
{
    double ux, uz, T, p;
    prims(q, z, C, ux, uz, T, p);
    const double c = sqrt(C.cs2 * T);
    const double v = fmin(C.dx / (fabs(ux) + c), hz / (fabs(uz) + c));
    if (!(v > 0.0) || !(v < 1e300)) bad = 1;
    return v;
}

// FP32 path: the largest rate (|u|+c)/h of a node; the block turns its max
// into min h/(|u|+c) with one FP64 reciprocal; ihz: 1 / the node's z step
__device__ __forceinline__ float dt_rate(const St<float>& q, float z, float ihz, const Coef<float>& C, int& bad)
{
    float ux, uz, T, p;
    prims(q, z, C, ux, uz, T, p);
    const float c = sqrtf(C.cs2 * T);
    const float r = fmaxf((fabsf(ux) + c) * C.inv_dx, (fabsf(uz) + c) * ihz);
    if (!(r > 0.f) || !(r < 1e30f)) bad = 1;
    return r;
}

__device__ __forceinline__ int clamp_row(int j, int nz) { return min(max(j, 0), nz - 1); }

// Delta / w_k of a stretched plane: the flux-difference factor of its cell
// (FP64: the division as written; FP32: times the stored reciprocal)
template <class R>
__device__ __forceinline__ R lam_cell(double Delta, const Plane<R>& P)
{
    if constexpr (kExact<R>) return Delta / P.w;
    else return (R)Delta * P.iw;
}

constexpr int kPrefetch = 3;  // rows loaded ahead of the one being consumed

// L_z(Delta): predictor with backward flux differences, plate fill of X^P,
// corrector with forward differences of F^P, average, TVD term from the
// input state, plate values.  Row pipeline at step j (row j just loaded):
//   F^n_{j-1}, X^P_{j-1}, F^P_{j-1}, average at j-2, TVD flux at (j-2,j-1),
//   output row j-2.
// ST: stretched z-grid (C.zp): the flux differences of plane k are divided by
// its cell width w_k, the one-sided derivatives by the spacing they span, the
// TVD fluxes weighted by spacing over width (conservative form on uneven
// planes; on uniform planes every factor reduces to the constant one).
template <class R, bool ST>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
sweep_z2d(SweepIO<R> io, Coef<R> C, SweepCtl sc)
{
    pdl_enter();
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const int strip = gw % io.nstrips;
    const int ks = (gw / io.nstrips) * io.seg_rows;
    const int nz = C.nz, nx = C.nx, pitch = C.pitch;
    const long long fs = C.fstride;
    const int ke = min(ks + io.seg_rows, nz);
    const int i = strip * kOutW - 2 + lane;
    int ic = i % nx;
    if (ic < 0) ic += nx;
    const bool own = lane >= 2 && lane < 2 + kOutW && i < nx;

    const double dt = step_dt(sc.ctl, sc.slot_in, C.cfl, C.dt_fixed);
    const double Delta = sc.Delta > 0.0 ? sc.Delta : 0.5 * dt;
    const R lam = (R)(Delta / C.dz);
    const R Dl = (R)Delta;
    R lam_bot = R(2) * lam, lam_top = R(2) * lam;  // half cells on the plates: Delta / w
    if constexpr (ST) {
        lam_bot = lam_cell(Delta, C.zp[0]);
        lam_top = lam_cell(Delta, C.zp[nz - 1]);
    }

    if (sc.first && blockIdx.x == 0 && threadIdx.x == 0) {
        sc.ctl->dt_slot[sc.slot_in ^ 1] = 0x7FF0000000000000ULL;
        sc.ctl->t += dt;
        sc.ctl->steps += 1.0;
    }
    if (ks >= nz) return;  // warp-uniform; this kernel has no block barrier

    // pipeline registers, primed with the first row so nothing is undefined
    St<R> Xm2 = load_row(io.in, fs, max(ks - 4, 0), pitch, ic);
    St<R> Xm1 = Xm2;
    R ux1, uz1, T1, p1;
    prims(Xm1, io.zt[max(ks - 4, 0)], C, ux1, uz1, T1, p1);
    R A2 = R(0), A1 = R(0), dxux1 = R(0), dxuz1 = R(0);
    St<R> F2 = {R(0), R(0), R(0), R(0)};
    St<R> XP2 = Xm2;
    R ppux2 = ux1, ppuz2 = uz1, ppT2 = T1;
    St<R> FP2 = F2, d1 = F2, Dm = F2;
    R dd1 = R(0), ss2 = R(0);

    St<R> pf[kPrefetch];
#pragma unroll
    for (int q = 0; q < kPrefetch; ++q) pf[q] = load_row(io.in, fs, clamp_row(ks - 2 + q, nz), pitch, ic);

    for (int j = ks - 2; j <= ke + 1; ++j) {
        const int jr = clamp_row(j, nz);
        // row j: primitives, wave speed |u_z| + c, cross derivatives d/dx
        const St<R> X0 = pf[0];
#pragma unroll
        for (int q = 0; q < kPrefetch - 1; ++q) pf[q] = pf[q + 1];
        pf[kPrefetch - 1] = load_row(io.in, fs, clamp_row(j + kPrefetch, nz), pitch, ic);
        R ux0, uz0, T0, p0;
        prims(X0, io.zt[jr], C, ux0, uz0, T0, p0);
        const R A0 = fabs(uz0) + rsqrt_(C.cs2 * T0);
        const R dxux0 = diff(shdn(ux0), shup(ux0), C.h2x, C.inv_2dx);
        const R dxuz0 = diff(shdn(uz0), shup(uz0), C.h2x, C.inv_2dx);

        // predictor flux F^n_{j-1} (forward z-differences inside F)
        const int m = j - 1;
        R hf = C.hz, ihf = C.inv_dz, hb = C.hz, ihb = C.inv_dz, lam_m = lam;
        if constexpr (ST) {
            const Plane<R>& Pm = C.zp[clamp_row(m, nz)];
            const Plane<R>& Pb = C.zp[clamp_row(m - 1, nz)];
            hf = Pm.hp; ihf = Pm.ihp;  // spacing above plane m
            hb = Pb.hp; ihb = Pb.ihp;  // spacing below plane m
            lam_m = lam_cell(Delta, Pm);
        }
        const St<R> F1 = flux_z(Xm1, ux1, uz1, p1, diff(ux0, ux1, hf, ihf), diff(uz0, uz1, hf, ihf),
                                diff(T0, T1, hf, ihf), dxux1, dxuz1, C);
        // predictor X^P_{j-1}; plates as half cells with zero wall flux, m = 0, T = T_w
        St<R> XP1;
        if (m >= 1 && m <= nz - 2) {
            XP1.r = Xm1.r - lam_m * (F1.r - F2.r);
            XP1.mx = Xm1.mx - lam_m * (F1.mx - F2.mx);
            XP1.mz = (Xm1.mz - lam_m * (F1.mz - F2.mz)) + Dl * (-C.g * Xm1.r);
            XP1.E = Xm1.E - lam_m * (F1.E - F2.E);
        } else if (m <= 0) {
            XP1.r = Xm1.r - lam_bot * F1.r;
            XP1.mx = R(0); XP1.mz = R(0);
            XP1.E = XP1.r * C.ebot;
        } else {
            XP1.r = Xm1.r + lam_top * F2.r;
            XP1.mx = R(0); XP1.mz = R(0);
            XP1.E = XP1.r * C.etop;
        }
        R ppux1, ppuz1, ppT1, ppp1;
        prims(XP1, io.zt[min(max(m, 0), nz - 1)], C, ppux1, ppuz1, ppT1, ppp1);
        const R dxppux1 = diff(shdn(ppux1), shup(ppux1), C.h2x, C.inv_2dx);
        const R dxppuz1 = diff(shdn(ppuz1), shup(ppuz1), C.h2x, C.inv_2dx);
        // corrector flux F^P_{j-1} (backward z-differences inside F)
        const St<R> FP1 = flux_z(XP1, ppux1, ppuz1, ppp1, diff(ppux1, ppux2, hb, ihb),
                                 diff(ppuz1, ppuz2, hb, ihb), diff(ppT1, ppT2, hb, ihb), dxppux1,
                                 dxppuz1, C);

        // corrector X^C_{j-2} and the average (X^P + X^C)/2
        const int c = j - 2;
        R lam_c = lam, hc = C.hz, lamh_c = lam, rp_c = R(1), rm_c = R(1);
        if constexpr (ST) {
            const Plane<R>& Pc = C.zp[clamp_row(c, nz)];
            lam_c = lam_cell(Delta, Pc);
            hc = Pc.hp;                  // spacing of interface (c, c+1)
            lamh_c = (R)Delta * Pc.ihp;  // FP32 Courant factor of that interface
            rp_c = Pc.rp;
            rm_c = Pc.rm;
        }
        St<R> Xa;
        if (c >= 1 && c <= nz - 2) {
            const R xcr = Xm2.r - lam_c * (FP1.r - FP2.r);
            const R xcmx = Xm2.mx - lam_c * (FP1.mx - FP2.mx);
            const R xcmz = (Xm2.mz - lam_c * (FP1.mz - FP2.mz)) + Dl * (-C.g * XP2.r);
            const R xcE = Xm2.E - lam_c * (FP1.E - FP2.E);
            Xa.r = (XP2.r + xcr) * R(0.5);
            Xa.mx = (XP2.mx + xcmx) * R(0.5);
            Xa.mz = (XP2.mz + xcmz) * R(0.5);
            Xa.E = (XP2.E + xcE) * R(0.5);
        } else if (c <= 0) {
            Xa.r = (XP2.r + (Xm2.r - lam_bot * FP1.r)) * R(0.5);
            Xa.mx = Xa.mz = Xa.E = R(0);
        } else {
            Xa.r = (XP2.r + Xm2.r) * R(0.5);  // F^P on the top plate is m_z = 0
            Xa.mx = Xa.mz = Xa.E = R(0);
        }

        // TVD: differences of the input state across interfaces j-1/2
        const St<R> d0 = {X0.r - Xm1.r, X0.mx - Xm1.mx, X0.mz - Xm1.mz, X0.E - Xm1.E};
        const R dd0 = dot4(d0, d0);
        const R ss1 = dot4(d1, d0);
        St<R> Dn = {R(0), R(0), R(0), R(0)};
        if (c >= 1 && c <= nz - 3) {  // interface (j-2, j-1); zero next to the plates
            const R G = tvd_G(ss2, ss1, dd1, courant(Delta, lamh_c, A2, A1, hc), C.tvd_form);
            Dn = {G * d1.r, G * d1.mx, G * d1.mz, G * d1.E};
        }

        // output row j-2
        if (c >= ks && c < ke) {
            St<R> Xn;
            if (c >= 1 && c <= nz - 2) {
                if constexpr (ST) {
                    Xn.r = Xa.r + (rp_c * Dn.r - rm_c * Dm.r);
                    Xn.mx = Xa.mx + (rp_c * Dn.mx - rm_c * Dm.mx);
                    Xn.mz = Xa.mz + (rp_c * Dn.mz - rm_c * Dm.mz);
                    Xn.E = Xa.E + (rp_c * Dn.E - rm_c * Dm.E);
                } else {
                    Xn.r = Xa.r + (Dn.r - Dm.r);
                    Xn.mx = Xa.mx + (Dn.mx - Dm.mx);
                    Xn.mz = Xa.mz + (Dn.mz - Dm.mz);
                    Xn.E = Xa.E + (Dn.E - Dm.E);
                }
            } else {
                Xn.r = Xa.r;
                Xn.mx = R(0); Xn.mz = R(0);
                Xn.E = Xa.r * (c == 0 ? C.ebot : C.etop);
            }
            if (own) store_row(io.out, fs, c, pitch, i, Xn);
        }

        // advance the pipeline
        Xm2 = Xm1; Xm1 = X0;
        ux1 = ux0; uz1 = uz0; T1 = T0; p1 = p0;
        A2 = A1; A1 = A0;
        dxux1 = dxux0; dxuz1 = dxuz0;
        F2 = F1; XP2 = XP1;
        ppux2 = ppux1; ppuz2 = ppuz1; ppT2 = ppT1;
        FP2 = FP1;
        d1 = d0; dd1 = dd0; ss2 = ss1; Dm = Dn;
    }
}

// L_x(Delta) on the interior rows (plate rows pass through).  Row pipeline at
// step j: F^n_{j-1} and X^P_{j-1} (needs rows j, j-2 for d/dz), then F^P_{j-2}
// (needs X^P rows j-1, j-3), corrector, average, TVD along x, output row j-2.
// ST: stretched z-grid: the central z-differences divide by the distance of
// the two planes they use, and the CFL z step is the plane's smaller spacing.
template <class R, bool ST>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
sweep_x2d(SweepIO<R> io, Coef<R> C, SweepCtl sc)
{
    pdl_enter();
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const int strip = gw % io.nstrips;
    const int ks = (gw / io.nstrips) * io.seg_rows;
    const int nz = C.nz, nx = C.nx, pitch = C.pitch;
    const long long fs = C.fstride;
    const int ke = min(ks + io.seg_rows, nz);
    const int i = strip * kOutW - 2 + lane;
    int ic = i % nx;
    if (ic < 0) ic += nx;
    const bool own = lane >= 2 && lane < 2 + kOutW && i < nx;

    const double dt = step_dt(sc.ctl, sc.slot_in, C.cfl, C.dt_fixed);
    const double Delta = sc.Delta > 0.0 ? sc.Delta : 0.5 * dt;
    const R lam = (R)(Delta / C.dx);

    if (sc.first && blockIdx.x == 0 && threadIdx.x == 0) {
        sc.ctl->dt_slot[sc.slot_in ^ 1] = 0x7FF0000000000000ULL;
        sc.ctl->t += dt;
        sc.ctl->steps += 1.0;
    }

    double vmin = 1e308;  // FP64 path: min h/(|u|+c) over the nodes of this thread
    R rmax = R(0);        // FP32 path: max (|u|+c)/h
    int bad = 0;
    if (ks < nz) {
        St<R> Xm2 = load_row(io.in, fs, max(ks - 4, 0), pitch, ic);
        St<R> Xm1 = Xm2;
        R ux1, uz1, T1, p1;
        prims(Xm1, io.zt[max(ks - 4, 0)], C, ux1, uz1, T1, p1);
        R ux2 = ux1, uz2 = uz1, T2 = T1, p2 = p1;
        St<R> XP2 = Xm2;
        R ppux2 = ux1, ppuz2 = uz1, ppT2 = T1, ppp2 = p1;
        R ppux3 = ux1, ppuz3 = uz1;

        St<R> pf[kPrefetch];
#pragma unroll
        for (int q = 0; q < kPrefetch; ++q) pf[q] = load_row(io.in, fs, clamp_row(ks - 2 + q, nz), pitch, ic);

        for (int j = ks - 2; j <= ke + 1; ++j) {
            const int jr = clamp_row(j, nz);
            const St<R> X0 = pf[0];
#pragma unroll
            for (int q = 0; q < kPrefetch - 1; ++q) pf[q] = pf[q + 1];
            pf[kPrefetch - 1] = load_row(io.in, fs, clamp_row(j + kPrefetch, nz), pitch, ic);
            R ux0, uz0, T0, p0;
            prims(X0, io.zt[jr], C, ux0, uz0, T0, p0);

            // row m = j-1: F^n with forward x-differences, central z-differences
            const int m = j - 1;
            R scm = C.h2z, iscm = C.inv_2dz;
            if constexpr (ST) {
                const Plane<R>& Pm = C.zp[clamp_row(m, nz)];
                scm = Pm.sc; iscm = Pm.isc;
            }
            const St<R> F1 = flux_x(Xm1, ux1, uz1, p1, diff(shdn(ux1), ux1, C.hx, C.inv_dx),
                                    diff(shdn(uz1), uz1, C.hx, C.inv_dx), diff(shdn(T1), T1, C.hx, C.inv_dx),
                                    diff(ux0, ux2, scm, iscm), diff(uz0, uz2, scm, iscm), C);
            const St<R> Fl = shup(F1);
            St<R> XP1 = Xm1;
            if (m >= 1 && m <= nz - 2) {
                XP1.r = Xm1.r - lam * (F1.r - Fl.r);
                XP1.mx = Xm1.mx - lam * (F1.mx - Fl.mx);
                XP1.mz = Xm1.mz - lam * (F1.mz - Fl.mz);
                XP1.E = Xm1.E - lam * (F1.E - Fl.E);
            }
            R ppux1, ppuz1, ppT1, ppp1;
            prims(XP1, io.zt[min(max(m, 0), nz - 1)], C, ppux1, ppuz1, ppT1, ppp1);

            // row c = j-2: F^P with backward x-differences, corrector, average
            const int c = j - 2;
            R scc = C.h2z, iscc = C.inv_2dz;
            double hzc = C.dz;
            R ihzc = C.inv_dz;
            if constexpr (ST) {
                const Plane<R>& Pc = C.zp[clamp_row(c, nz)];
                scc = Pc.sc; iscc = Pc.isc;
                hzc = (double)Pc.hmin; ihzc = Pc.ihmin;
            }
            const St<R> FP = flux_x(XP2, ppux2, ppuz2, ppp2, diff(ppux2, shup(ppux2), C.hx, C.inv_dx),
                                    diff(ppuz2, shup(ppuz2), C.hx, C.inv_dx), diff(ppT2, shup(ppT2), C.hx, C.inv_dx),
                                    diff(ppux1, ppux3, scc, iscc), diff(ppuz1, ppuz3, scc, iscc), C);
            const St<R> FPr = shdn(FP);
            St<R> Xa;
            Xa.r = (XP2.r + (Xm2.r - lam * (FPr.r - FP.r))) * R(0.5);
            Xa.mx = (XP2.mx + (Xm2.mx - lam * (FPr.mx - FP.mx))) * R(0.5);
            Xa.mz = (XP2.mz + (Xm2.mz - lam * (FPr.mz - FP.mz))) * R(0.5);
            Xa.E = (XP2.E + (Xm2.E - lam * (FPr.E - FP.E))) * R(0.5);

            // TVD along x from the input state of row c
            const St<R> Xr = shdn(Xm2);
            const St<R> d0 = {Xr.r - Xm2.r, Xr.mx - Xm2.mx, Xr.mz - Xm2.mz, Xr.E - Xm2.E};
            const R dd = dot4(d0, d0);
            const St<R> dl = shup(d0);
            const R sp = dot4(dl, d0);
            const R sm = shdn(sp);
            const R A = fabs(ux2) + rsqrt_(C.cs2 * T2);
            const R G = tvd_G(sp, sm, dd, courant(Delta, lam, A, shdn(A), C.hx), C.tvd_form);
            const St<R> Dn = {G * d0.r, G * d0.mx, G * d0.mz, G * d0.E};
            const St<R> Dlf = shup(Dn);

            if (c >= ks && c < ke) {
                St<R> Xn = Xm2;  // plate rows pass through
                if (c >= 1 && c <= nz - 2) {
                    Xn.r = Xa.r + (Dn.r - Dlf.r);
                    Xn.mx = Xa.mx + (Dn.mx - Dlf.mx);
                    Xn.mz = Xa.mz + (Dn.mz - Dlf.mz);
                    Xn.E = Xa.E + (Dn.E - Dlf.E);
                }
                if (own) {
                    store_row(io.out, fs, c, pitch, i, Xn);
                    if (sc.last) {
                        if constexpr (kExact<R>) vmin = fmin(vmin, dt_candidate(Xn, io.zt[c], hzc, C, bad));
                        else rmax = fmax(rmax, dt_rate(Xn, io.zt[c], ihzc, C, bad));
                    }
                }
            }

            Xm2 = Xm1; Xm1 = X0;
            ux2 = ux1; uz2 = uz1; T2 = T1; p2 = p1;
            ux1 = ux0; uz1 = uz0; T1 = T0; p1 = p0;
            ppux3 = ppux2; ppuz3 = ppuz2;
            XP2 = XP1;
            ppux2 = ppux1; ppuz2 = ppuz1; ppT2 = ppT1; ppp2 = ppp1;
        }
    }
    if (sc.last) {
        if constexpr (!kExact<R>) vmin = rmax > R(0) ? 1.0 / (double)rmax : 1e308;
        block_dt_reduce(vmin, bad, sc.ctl, sc.slot_in ^ 1);
    }
}

}  // namespace cm
