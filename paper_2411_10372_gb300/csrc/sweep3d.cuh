// sweep3d.cuh -- fused 3D sweeps L_z, L_y (march kernel) and L_x (lane
// kernel) of Sec. 3.1, templated on the state precision.
//
// Geometry (a 2.5D march).  Lanes span x (a strip of 32 columns, 28 output
// columns, periodic).  The NW warps of a block span the third direction W
// (y for the z and x sweeps, z for the y sweep), one row each; the block's
// outer two warps on each side are halo and alone the inner NW-4 store.
// Every warp marches along the march direction M (z for the z and x sweeps,
// y for the y sweep) through a segment of rows, keeping rows in flight in
// registers as the 2D kernels do, with the next row's state loaded one
// iteration ahead.  Cross derivatives along x come from lane shuffles, along
// M from the register pipeline, and along W from one shared-memory exchange
// per row (double-buffered by row parity, so one block barrier per row) of
// the velocity components the fluxes need, of X at the newest row and of
// X^P one row behind.
//
// Halo roles: the outermost warps (role 0) only supply primitives of X; the
// next ones (role 1) also compute F^n, X^P and its primitives, which the
// output warps' F^P cross derivatives read; output warps (role 2) run the
// whole pipeline.
#pragma once
#include "sweep3d_common.cuh"

namespace cm {

template <class R>
struct Sweep3IO {
    const R* in;
    R* out;
    const R* zt;   // z of each plane, in R
    int seg;       // rows per march segment
    int nstrips;   // x strips of kOutW columns
    int nmarch;    // rows along the march direction (nz or ny)
    int nw;        // rows along W (ny or nz)
};

// state index of (plane k, row jy, column ic)
__device__ __forceinline__ long long off3(int k, int jy, int ny, int pitch, int ic)
{
    return ((long long)k * ny + jy) * pitch + ic;
}

__device__ __forceinline__ int wrap(int a, int n)
{
    a %= n;
    return a < 0 ? a + n : a;
}

// Stretched z-grid: the per-plane metric of the planes a block's segment
// touches (ks - 4 .. ke, clamped), copied once into shared memory so that
// every row reads it by broadcast (all warps of a block march the same
// rows).  NV values per plane; entry e holds plane clamp(ks - 4 + e).
constexpr int kPlaneBack = 4;
template <class R, int NV>
__device__ __forceinline__ void fill_planes(R* pz, const Coef<R>& C, int ks, int ke, bool march_z)
{
    const int n = ke - ks + kPlaneBack + 1;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const Plane<R>& P = C.zp[min(max(ks - kPlaneBack + e, 0), C.nz - 1)];
        if (march_z) {
            // FP64: the spacings (the exact path divides); FP32: reciprocals
            pz[e * NV + 0] = kExact<R> ? P.hp : P.ihp;
            pz[e * NV + 1] = kExact<R> ? P.w : P.iw;
            pz[e * NV + 2] = P.rp;
            pz[e * NV + 3] = P.rm;
        } else {
            pz[e * NV + 0] = kExact<R> ? P.sc : P.isc;
            pz[e * NV + 1] = kExact<R> ? P.hmin : P.ihmin;
        }
    }
    __syncthreads();
}
template <class R>
inline size_t plane_cache_bytes(int seg, int nv) { return (size_t)(seg + kPlaneBack + 1) * nv * sizeof(R); }

template <int NW>
__device__ __forceinline__ int halo_role(int w)
{
    return (w == 0 || w == NW - 1) ? 0 : ((w == 1 || w == NW - 2) ? 1 : 2);
}

// L_z (AL = 2: march z, W = y) or L_y (AL = 1: march y, W = z).  ST: a
// stretched z-grid (C.zp): for L_z the flux differences of plane k divide by
// its cell width, the one-sided derivatives by the spacing they span and the
// TVD fluxes are weighted by spacing over width (as in the 2D z sweep); for
// L_y the central z-differences across W divide by the distance of the two
// planes next to the warp's plane.
// Row pipeline at step j (row j of the march just taken from the prefetch),
// as in sweep_z2d: F^n_{j-1}, X^P_{j-1}, F^P_{j-1}, average at j-2, TVD flux
// across (j-2, j-1), output row j-2.  Plates: for L_z at the ends of the
// march (half-cell density, m = 0, T = T_w); for L_y the plate planes are
// rows of W and pass through unchanged.
template <class R, int AL, int NW, bool ST = false>
__global__ void __launch_bounds__(NW * 32)
sweep3d_march(Sweep3IO<R> io, Coef<R> C, SweepCtl sc)
{
    pdl_enter();
    extern __shared__ unsigned char pz_raw[];
    R* pz = reinterpret_cast<R*>(pz_raw);  // stretched L_z: plane cache (fill_planes)
    constexpr int WD = (AL == 2) ? 1 : 2;  // direction of the warps
    // [row parity][u_AL, u_W of X at row j; u_AL, u_W of X^P at row j-1][warp][lane]
    __shared__ R xs[2][4][NW][32];

    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int role = halo_role<NW>(w);
    const int strip = blockIdx.x;
    const int cw = blockIdx.y * (NW - 4) - 2 + w;      // W coordinate of this warp
    const int ks = blockIdx.z * io.seg;                 // first output row of the segment
    const int nz = C.nz, ny = C.ny, nx = C.nx, pitch = C.pitch;
    const long long fs = C.fstride;
    const int nm = io.nmarch;
    const int ke = min(ks + io.seg, nm);
    const int i = strip * kOutW - 2 + lane;
    const int ic = wrap(i, nx);
    // W row this warp reads: periodic in y, clamped in z (out-of-range warps compute unused values)
    const int cwr = (WD == 1) ? wrap(cw, ny) : min(max(cw, 0), nz - 1);
    const bool w_out = w >= 2 && w < NW - 2 && cw < io.nw && cw >= 0;
    const bool own = lane >= 2 && lane < 2 + kOutW && i < nx && w_out;
    // L_y leaves the plate planes unchanged
    const bool passthru = (AL == 1) && (cwr == 0 || cwr == nz - 1);

    const double dt = step_dt(sc.ctl, sc.slot_in, C.cfl, C.dt_fixed);
    const double Delta = sc.Delta > 0.0 ? sc.Delta : 0.5 * dt;
    const R h = (AL == 2) ? C.hz : C.hy;
    const R lam = (R)(Delta / ((AL == 2) ? C.dz : C.dy));
    const R Dl = (R)Delta;
    const R lam2 = R(2) * lam;
    // stretched grid: plate half cells (L_z) and the warp plane's central z span (L_y)
    R lam_bot = lam2, lam_top = lam2, wsc = C.h2z, iwsc = C.inv_2dz;
    if constexpr (ST) {
        if (AL == 2) {
            lam_bot = lam_cell(Delta, C.zp[0]);
            lam_top = lam_cell(Delta, C.zp[nz - 1]);
        } else {
            const Plane<R>& Pw = C.zp[cwr];
            wsc = Pw.sc;
            iwsc = Pw.isc;
        }
    }
    if (sc.first && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0) {
        sc.ctl->dt_slot[sc.slot_in ^ 1] = 0x7FF0000000000000ULL;
        sc.ctl->t += dt;
        sc.ctl->steps += 1.0;
    }

    if constexpr (ST && AL == 2) fill_planes<R, 4>(pz, C, ks, ke, true);
    auto pl = [&](int k, int q) -> R { return pz[(k - (ks - kPlaneBack)) * 4 + q]; };

    // memory offset of march row j: plane clamp(j) of row cwr (L_z), row
    // wrap(j) of plane cwr (L_y); rows are taken in order from j0 - 1 on
    const long long colbase = (AL == 2) ? (long long)cwr * pitch + ic : (long long)cwr * ny * pitch + ic;
    const long long rstride = (AL == 2) ? (long long)ny * pitch : (long long)pitch;
    const int j0 = ks - 2;
    int jl = j0 - 1;                             // next row to load
    int jw = (AL == 1) ? wrap(jl, ny) : 0;      // its wrapped index (L_y)
    const R zc = io.zt[cwr];
    auto load_next = [&](S3<R>& X, R& z) {
        const int r = (AL == 2) ? min(max(jl, 0), nz - 1) : jw;
        X = s3_load(io.in, fs, colbase + r * rstride);
        z = (AL == 2) ? io.zt[r] : zc;
        ++jl;
        if (AL == 1) jw = (jw + 1 == ny) ? 0 : jw + 1;
    };
    auto row_off = [&](int j) -> long long {
        return colbase + (long long)((AL == 2) ? min(max(j, 0), nz - 1) : wrap(j, ny)) * rstride;
    };

    S3<R> Xm1, Xpre;
    R zm1, zpre;
    load_next(Xm1, zm1);
    load_next(Xpre, zpre);
    S3<R> Xm2 = Xm1;
    R u1[3], T1, p1;
    prims3(Xm1, zm1, C, u1, T1, p1);
    R A1 = R(0), A2 = R(0), dxux1 = R(0), dxua1 = R(0), dwua1 = R(0), dwuw1 = R(0);
    const S3<R> zero = {R(0), {R(0), R(0), R(0)}, R(0)};
    S3<R> F2 = zero, XP2 = Xm1, FP2 = zero, d1 = zero, Dm = zero;
    R ppu2[3] = {u1[0], u1[1], u1[2]}, ppT2 = T1;
    R dd1 = R(0), ss2 = R(0);

    for (int j = j0; j <= ke + 1; ++j) {
        const S3<R> X0 = Xpre;
        const R z0 = zpre;
        if (j <= ke) load_next(Xpre, zpre);  // row j+1, used next iteration
        R u0[3], T0, p0;
        prims3(X0, z0, C, u0, T0, p0);
        R A0 = R(0), dxux0 = R(0), dxua0 = R(0);

        // row m = j-1: F^n (forward along the march), X^P and its primitives
        const int m = j - 1;
        // spacings along the march (stretched L_z: per plane) and the cell factor of row m
        R hf = h, ihf = (AL == 2) ? C.inv_dz : C.inv_dy, hb = hf, ihb = ihf, lam_m = lam;
        if constexpr (ST && AL == 2) {
            // spacing above m and below m, and Delta / w_m (FP64: spacings; FP32: reciprocals)
            if constexpr (kExact<R>) {
                hf = pl(m, 0);
                hb = pl(m - 1, 0);
                lam_m = Delta / pl(m, 1);
            } else {
                ihf = pl(m, 0);
                ihb = pl(m - 1, 0);
                lam_m = (R)Delta * pl(m, 1);
            }
        }
        S3<R> F1 = zero, XP1 = Xm1;
        R ppu1[3] = {u1[0], u1[1], u1[2]}, ppT1 = T1, ppp1 = p1;
        if (role >= 1) {
            A0 = fabs(u0[AL]) + rsqrt_(C.cs2 * T0);
            dxux0 = d3(shdn(u0[0]), shup(u0[0]), C, 0, true);
            dxua0 = d3(shdn(u0[AL]), shup(u0[AL]), C, 0, true);
            R du[3][3] = {{R(0), R(0), R(0)}, {R(0), R(0), R(0)}, {R(0), R(0), R(0)}};
#pragma unroll
            for (int c = 0; c < 3; ++c) du[c][AL] = diff(u0[c], u1[c], hf, ihf);
            du[0][0] = dxux1;
            du[AL][0] = dxua1;
            du[WD][WD] = dwuw1;
            du[AL][WD] = dwua1;
            F1 = flux3<AL>(Xm1, u1, p1, du, diff(T0, T1, hf, ihf), C);
            if (AL == 2) {
                if (m >= 1 && m <= nz - 2) {
                    XP1.r = Xm1.r - lam_m * (F1.r - F2.r);
                    XP1.m[0] = Xm1.m[0] - lam_m * (F1.m[0] - F2.m[0]);
                    XP1.m[1] = Xm1.m[1] - lam_m * (F1.m[1] - F2.m[1]);
                    XP1.m[2] = (Xm1.m[2] - lam_m * (F1.m[2] - F2.m[2])) + Dl * (-C.g * Xm1.r);
                    XP1.E = Xm1.E - lam_m * (F1.E - F2.E);
                } else {
                    XP1.r = (m <= 0) ? Xm1.r - lam_bot * F1.r : Xm1.r + lam_top * F2.r;
                    XP1.m[0] = XP1.m[1] = XP1.m[2] = R(0);
                    XP1.E = XP1.r * ((m <= 0) ? C.ebot : C.etop);
                }
            } else if (!passthru) {
                XP1.r = Xm1.r - lam * (F1.r - F2.r);
#pragma unroll
                for (int c = 0; c < 3; ++c) XP1.m[c] = Xm1.m[c] - lam * (F1.m[c] - F2.m[c]);
                XP1.E = Xm1.E - lam * (F1.E - F2.E);
            }
            prims3(XP1, zm1, C, ppu1, ppT1, ppp1);
        }

        // exchange across W: u of X at row j and of X^P at row m
        R(*buf)[NW][32] = xs[j & 1];
        buf[0][w][lane] = u0[AL];
        buf[1][w][lane] = u0[WD];
        buf[2][w][lane] = ppu1[AL];
        buf[3][w][lane] = ppu1[WD];
        __syncthreads();
        const int wu = min(w + 1, NW - 1), wd = max(w - 1, 0);
        // central differences across W (W = z for L_y: the warp plane's span)
        auto dw = [&](R a, R b) { return (WD == 2) ? diff(a, b, wsc, iwsc) : d3(a, b, C, WD, true); };
        const R dwua0 = dw(buf[0][wu][lane], buf[0][wd][lane]);
        const R dwuw0 = dw(buf[1][wu][lane], buf[1][wd][lane]);

        S3<R> FP1 = zero, Dn = zero, d0 = zero;
        R dd0 = R(0), ss1 = R(0);
        if (role == 2) {
            const R dwppa1 = dw(buf[2][wu][lane], buf[2][wd][lane]);
            const R dwppw1 = dw(buf[3][wu][lane], buf[3][wd][lane]);
            R dq[3][3] = {{R(0), R(0), R(0)}, {R(0), R(0), R(0)}, {R(0), R(0), R(0)}};
#pragma unroll
            for (int c = 0; c < 3; ++c) dq[c][AL] = diff(ppu1[c], ppu2[c], hb, ihb);
            dq[0][0] = d3(shdn(ppu1[0]), shup(ppu1[0]), C, 0, true);
            dq[AL][0] = d3(shdn(ppu1[AL]), shup(ppu1[AL]), C, 0, true);
            dq[WD][WD] = dwppw1;
            dq[AL][WD] = dwppa1;
            FP1 = flux3<AL>(XP1, ppu1, ppp1, dq, diff(ppT1, ppT2, hb, ihb), C);

            // row c = j-2: corrector X^C and the average (X^P + X^C)/2
            const int c = j - 2;
            R lam_c = lam, hc = h, lamh_c = lam, rp_c = R(1), rm_c = R(1);
            if constexpr (ST && AL == 2) {
                if constexpr (kExact<R>) {
                    hc = pl(c, 0);
                    lam_c = Delta / pl(c, 1);
                } else {
                    lamh_c = (R)Delta * pl(c, 0);
                    lam_c = (R)Delta * pl(c, 1);
                }
                rp_c = pl(c, 2);
                rm_c = pl(c, 3);
            }
            S3<R> Xa = Xm2;
            if (AL == 2) {
                if (c >= 1 && c <= nz - 2) {
                    Xa.r = (XP2.r + (Xm2.r - lam_c * (FP1.r - FP2.r))) * R(0.5);
                    Xa.m[0] = (XP2.m[0] + (Xm2.m[0] - lam_c * (FP1.m[0] - FP2.m[0]))) * R(0.5);
                    Xa.m[1] = (XP2.m[1] + (Xm2.m[1] - lam_c * (FP1.m[1] - FP2.m[1]))) * R(0.5);
                    Xa.m[2] = (XP2.m[2] + ((Xm2.m[2] - lam_c * (FP1.m[2] - FP2.m[2])) + Dl * (-C.g * XP2.r))) * R(0.5);
                    Xa.E = (XP2.E + (Xm2.E - lam_c * (FP1.E - FP2.E))) * R(0.5);
                } else {
                    Xa.r = (c <= 0) ? (XP2.r + (Xm2.r - lam_bot * FP1.r)) * R(0.5) : (XP2.r + Xm2.r) * R(0.5);
                }
            } else if (!passthru) {
                Xa.r = (XP2.r + (Xm2.r - lam * (FP1.r - FP2.r))) * R(0.5);
#pragma unroll
                for (int q = 0; q < 3; ++q)
                    Xa.m[q] = (XP2.m[q] + (Xm2.m[q] - lam * (FP1.m[q] - FP2.m[q]))) * R(0.5);
                Xa.E = (XP2.E + (Xm2.E - lam * (FP1.E - FP2.E))) * R(0.5);
            }

            // TVD flux across (j-2, j-1) from the input state
            d0 = s3_sub(X0, Xm1);
            dd0 = s3_dot(d0, d0);
            ss1 = s3_dot(d1, d0);
            const bool tvd_on = (AL == 2) ? (c >= 1 && c <= nz - 3) : !passthru;
            if (tvd_on) {
                const R G = tvd_G(ss2, ss1, dd1, courant(Delta, lamh_c, A2, A1, hc), C.tvd_form);
                Dn = {G * d1.r, {G * d1.m[0], G * d1.m[1], G * d1.m[2]}, G * d1.E};
            }

            if (c >= ks && c < ke && own) {
                S3<R> Xn = Xa;
                const bool interior = (AL == 2) ? (c >= 1 && c <= nz - 2) : !passthru;
                if (interior) {
                    if constexpr (ST && AL == 2) {
                        Xn.r = Xa.r + (rp_c * Dn.r - rm_c * Dm.r);
#pragma unroll
                        for (int q = 0; q < 3; ++q) Xn.m[q] = Xa.m[q] + (rp_c * Dn.m[q] - rm_c * Dm.m[q]);
                        Xn.E = Xa.E + (rp_c * Dn.E - rm_c * Dm.E);
                    } else {
                        Xn.r = Xa.r + (Dn.r - Dm.r);
#pragma unroll
                        for (int q = 0; q < 3; ++q) Xn.m[q] = Xa.m[q] + (Dn.m[q] - Dm.m[q]);
                        Xn.E = Xa.E + (Dn.E - Dm.E);
                    }
                } else if (AL == 2) {
                    Xn.m[0] = Xn.m[1] = Xn.m[2] = R(0);
                    Xn.E = Xa.r * (c == 0 ? C.ebot : C.etop);
                }
                s3_store(io.out, fs, row_off(c), Xn);
            }
        }

        Xm2 = Xm1;
        Xm1 = X0;
        zm1 = z0;
        u1[0] = u0[0]; u1[1] = u0[1]; u1[2] = u0[2];
        T1 = T0;
        p1 = p0;
        A2 = A1;
        A1 = A0;
        dxux1 = dxux0; dxua1 = dxua0; dwua1 = dwua0; dwuw1 = dwuw0;
        F2 = F1;
        XP2 = XP1;
        ppu2[0] = ppu1[0]; ppu2[1] = ppu1[1]; ppu2[2] = ppu1[2];
        ppT2 = ppT1;
        FP2 = FP1;
        d1 = d0;
        dd1 = dd0;
        ss2 = ss1;
        Dm = Dn;
    }
}

// L_x in 3D: march z, warps span y, the x stencil across lanes (as
// sweep_x2d); plate planes pass through.  Row pipeline at step j: F^n and X^P
// of row j-1 (d/dz from rows j, j-2; d/dy from the exchange of row j-1 one
// iteration earlier), then F^P (d/dz of X^P from rows j-1, j-3; d/dy from
// the exchange of row j-2), corrector, average and TVD along x of row j-2,
// output row j-2.  One exchange per row carries u_x, u_y of X at row j and
// of X^P at row j-1, both read in the next iteration.  ST: stretched z-grid:
// central z-differences over the distance of the two planes next to the
// row, CFL z step the row plane's smaller spacing.
template <class R, int NW, bool ST = false>
__global__ void __launch_bounds__(NW * 32)
sweep3d_x(Sweep3IO<R> io, Coef<R> C, SweepCtl sc)
{
    pdl_enter();
    __shared__ R xs[2][4][NW][32];
    extern __shared__ unsigned char pz_raw[];
    R* pz = reinterpret_cast<R*>(pz_raw);  // stretched grid: plane cache (fill_planes)
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int role = halo_role<NW>(w);
    const int cw = blockIdx.y * (NW - 4) - 2 + w;  // y row of this warp
    const int ks = blockIdx.z * io.seg;
    const int nz = C.nz, ny = C.ny, nx = C.nx, pitch = C.pitch;
    const long long fs = C.fstride;
    const int ke = min(ks + io.seg, nz);
    const int i = blockIdx.x * kOutW - 2 + lane;
    const int ic = wrap(i, nx);
    const int cwr = wrap(cw, ny);
    const bool own = lane >= 2 && lane < 2 + kOutW && i < nx && w >= 2 && w < NW - 2 && cw < ny;

    const double dt = step_dt(sc.ctl, sc.slot_in, C.cfl, C.dt_fixed);
    const double Delta = sc.Delta > 0.0 ? sc.Delta : 0.5 * dt;
    const R lam = (R)(Delta / C.dx);
    if (sc.first && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0) {
        sc.ctl->dt_slot[sc.slot_in ^ 1] = 0x7FF0000000000000ULL;
        sc.ctl->t += dt;
        sc.ctl->steps += 1.0;
    }
    if constexpr (ST) fill_planes<R, 2>(pz, C, ks, ke, false);
    auto pl = [&](int k, int q) -> R { return pz[(k - (ks - kPlaneBack)) * 2 + q]; };
    const long long colbase = (long long)cwr * pitch + ic, rstride = (long long)ny * pitch;
    auto offk = [&](int k) { return colbase + (long long)min(max(k, 0), nz - 1) * rstride; };
    auto zk = [&](int k) { return io.zt[min(max(k, 0), nz - 1)]; };

    double vmin = 1e308;
    R rmax = R(0);
    int bad = 0;
    const int j0 = ks - 2;
    S3<R> Xm1 = s3_load(io.in, fs, offk(j0 - 1)), Xm2 = Xm1;
    S3<R> Xpre = s3_load(io.in, fs, offk(j0));
    R zm1 = zk(j0 - 1), zpre = zk(j0);
    R u1[3], T1, p1;
    prims3(Xm1, zm1, C, u1, T1, p1);
    R u2[3] = {u1[0], u1[1], u1[2]}, T2 = T1;
    R dwx1 = R(0), dwy1 = R(0);          // d/dy of u_x, u_y of row j-1
    S3<R> XP2 = Xm1;
    R pp2[3] = {u1[0], u1[1], u1[2]}, ppT2 = T1, ppp2 = p1;
    R pp3[3] = {u1[0], u1[1], u1[2]};
    R dwpx2 = R(0), dwpy2 = R(0);        // d/dy of X^P u_x, u_y of row j-2

    for (int j = j0; j <= ke + 1; ++j) {
        const S3<R> X0 = Xpre;
        const R z0 = zpre;
        if (j <= ke) {  // row j+1, used next iteration
            Xpre = s3_load(io.in, fs, offk(j + 1));
            zpre = zk(j + 1);
        }
        R u0[3], T0, p0;
        prims3(X0, z0, C, u0, T0, p0);

        // row m = j-1: F^n with forward x-differences, X^P and its primitives
        const int m = j - 1;
        R scm = C.h2z, iscm = C.inv_2dz;  // central z span at row m
        if constexpr (ST) {
            if constexpr (kExact<R>) scm = pl(m, 0);
            else iscm = pl(m, 0);
        }
        S3<R> XP1 = Xm1;
        R pp1[3] = {u1[0], u1[1], u1[2]}, ppT1 = T1, ppp1 = p1;
        if (role >= 1) {
            R du[3][3] = {{R(0), R(0), R(0)}, {R(0), R(0), R(0)}, {R(0), R(0), R(0)}};
#pragma unroll
            for (int c = 0; c < 3; ++c) du[c][0] = d3(shdn(u1[c]), u1[c], C, 0, false);
            du[0][1] = dwx1;
            du[1][1] = dwy1;
            du[0][2] = diff(u0[0], u2[0], scm, iscm);
            du[2][2] = diff(u0[2], u2[2], scm, iscm);
            const S3<R> F1 = flux3<0>(Xm1, u1, p1, du, d3(shdn(T1), T1, C, 0, false), C);
            const S3<R> Fl = {shup(F1.r), {shup(F1.m[0]), shup(F1.m[1]), shup(F1.m[2])}, shup(F1.E)};
            if (m >= 1 && m <= nz - 2) {
                XP1.r = Xm1.r - lam * (F1.r - Fl.r);
#pragma unroll
                for (int c = 0; c < 3; ++c) XP1.m[c] = Xm1.m[c] - lam * (F1.m[c] - Fl.m[c]);
                XP1.E = Xm1.E - lam * (F1.E - Fl.E);
            }
            prims3(XP1, zm1, C, pp1, ppT1, ppp1);
        }

        // exchange across y: u of X at row j and of X^P at row j-1
        R(*buf)[NW][32] = xs[j & 1];
        buf[0][w][lane] = u0[0];
        buf[1][w][lane] = u0[1];
        buf[2][w][lane] = pp1[0];
        buf[3][w][lane] = pp1[1];
        __syncthreads();
        const int wu = min(w + 1, NW - 1), wd = max(w - 1, 0);
        const R dwx0 = d3(buf[0][wu][lane], buf[0][wd][lane], C, 1, true);
        const R dwy0 = d3(buf[1][wu][lane], buf[1][wd][lane], C, 1, true);
        const R dwpx1 = d3(buf[2][wu][lane], buf[2][wd][lane], C, 1, true);
        const R dwpy1 = d3(buf[3][wu][lane], buf[3][wd][lane], C, 1, true);

        if (role == 2) {
            // row c = j-2: F^P with backward x-differences, corrector, average, TVD along x
            const int c = j - 2;
            R scc = C.h2z, iscc = C.inv_2dz, hzc = C.hz, ihzc = C.inv_dz;
            if constexpr (ST) {
                if constexpr (kExact<R>) {
                    scc = pl(c, 0);
                    hzc = pl(c, 1);
                } else {
                    iscc = pl(c, 0);
                    ihzc = pl(c, 1);
                }
            }
            R dq[3][3] = {{R(0), R(0), R(0)}, {R(0), R(0), R(0)}, {R(0), R(0), R(0)}};
#pragma unroll
            for (int q = 0; q < 3; ++q) dq[q][0] = d3(pp2[q], shup(pp2[q]), C, 0, false);
            dq[0][1] = dwpx2;
            dq[1][1] = dwpy2;
            dq[0][2] = diff(pp1[0], pp3[0], scc, iscc);
            dq[2][2] = diff(pp1[2], pp3[2], scc, iscc);
            const S3<R> FP = flux3<0>(XP2, pp2, ppp2, dq, d3(ppT2, shup(ppT2), C, 0, false), C);
            const S3<R> FPr = {shdn(FP.r), {shdn(FP.m[0]), shdn(FP.m[1]), shdn(FP.m[2])}, shdn(FP.E)};
            S3<R> Xa;
            Xa.r = (XP2.r + (Xm2.r - lam * (FPr.r - FP.r))) * R(0.5);
#pragma unroll
            for (int q = 0; q < 3; ++q) Xa.m[q] = (XP2.m[q] + (Xm2.m[q] - lam * (FPr.m[q] - FP.m[q]))) * R(0.5);
            Xa.E = (XP2.E + (Xm2.E - lam * (FPr.E - FP.E))) * R(0.5);
            const S3<R> Xr = {shdn(Xm2.r), {shdn(Xm2.m[0]), shdn(Xm2.m[1]), shdn(Xm2.m[2])}, shdn(Xm2.E)};
            const S3<R> d0 = s3_sub(Xr, Xm2);
            const R dd = s3_dot(d0, d0);
            const S3<R> dl = {shup(d0.r), {shup(d0.m[0]), shup(d0.m[1]), shup(d0.m[2])}, shup(d0.E)};
            const R sp = s3_dot(dl, d0);
            const R sm = shdn(sp);
            const R A = fabs(u2[0]) + rsqrt_(C.cs2 * T2);
            const R G = tvd_G(sp, sm, dd, courant(Delta, lam, A, shdn(A), C.hx), C.tvd_form);
            const S3<R> Dn = {G * d0.r, {G * d0.m[0], G * d0.m[1], G * d0.m[2]}, G * d0.E};
            const S3<R> Dl = {shup(Dn.r), {shup(Dn.m[0]), shup(Dn.m[1]), shup(Dn.m[2])}, shup(Dn.E)};

            if (c >= ks && c < ke && own) {
                S3<R> Xn = Xm2;  // plate planes pass through
                if (c >= 1 && c <= nz - 2) {
                    Xn.r = Xa.r + (Dn.r - Dl.r);
#pragma unroll
                    for (int q = 0; q < 3; ++q) Xn.m[q] = Xa.m[q] + (Dn.m[q] - Dl.m[q]);
                    Xn.E = Xa.E + (Dn.E - Dl.E);
                }
                s3_store(io.out, fs, offk(c), Xn);
                if (sc.last) {
                    R un[3], Tn, pn;
                    prims3(Xn, zk(c), C, un, Tn, pn);
                    if constexpr (kExact<R>) {
                        const double cs = sqrt(C.cs2 * Tn);
                        double v = C.dx / (fabs(un[0]) + cs);
                        v = fmin(v, C.dy / (fabs(un[1]) + cs));
                        v = fmin(v, (ST ? (double)hzc : C.dz) / (fabs(un[2]) + cs));
                        if (!(v > 0.0) || !(v < 1e300)) bad = 1;
                        vmin = fmin(vmin, v);
                    } else {
                        const R cs = rsqrt_(C.cs2 * Tn);
                        const R r = fmax(fmax((fabs(un[0]) + cs) * C.inv_dx, (fabs(un[1]) + cs) * C.inv_dy),
                                         (fabs(un[2]) + cs) * ihzc);
                        if (!(r > R(0)) || !(r < R(1e30))) bad = 1;
                        rmax = fmax(rmax, r);
                    }
                }
            }
        }

        Xm2 = Xm1;
        Xm1 = X0;
        zm1 = z0;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            u2[q] = u1[q];
            u1[q] = u0[q];
            pp3[q] = pp2[q];
            pp2[q] = pp1[q];
        }
        T2 = T1;
        T1 = T0;
        p1 = p0;
        dwx1 = dwx0;
        dwy1 = dwy0;
        XP2 = XP1;
        ppT2 = ppT1;
        ppp2 = ppp1;
        dwpx2 = dwpx1;
        dwpy2 = dwpy1;
    }
    if (sc.last) {
        if constexpr (!kExact<R>) vmin = rmax > R(0) ? 1.0 / (double)rmax : 1e308;
        block_dt_reduce(vmin, bad, sc.ctl, sc.slot_in ^ 1);
    }
}

}  // namespace cm
