// sweep3d_x2.cuh -- FP32 3D sweeps with two columns per lane (even nx;
// uniform or, with ST, stretched z-grid): L_z and L_y (march kernel) and L_x
// of Sec. 3.1.
//
// The 2.5D geometry of sweep3d.cuh -- lanes across x, the warps of a block
// across the third direction W (y for L_z and L_x, z for L_y), all marching
// together along M (z for L_z and L_x, y for L_y) -- with the packed
// arithmetic of sweep2d_x2.cuh: every lane carries two adjacent columns as
// float2 and updates both with one FFMA2/FMUL2/FADD2, so a warp covers 64
// columns, of which lanes 1..30 store 60.  Neighbour columns come from one
// shuffle per exchanged quantity; cross derivatives along W from one
// shared-memory exchange per row (double-buffered by row parity: one block
// barrier per row) of the velocity components the fluxes need, of X at the
// newest row and of X^P one row behind.  The outer two warps on each side of
// a block are halo (role 0: primitives of X; role 1: also F^n, X^P and its
// primitives); the inner ones store.  Rows are staged by a per-thread
// cp.async ring in shared memory, kRing3 rows deep.
//
// The march kernel carries the average across rows:
//   H_c = (X^P + X + Delta S^P)_c / 2 - D_{c-1/2},
//   X_new_c = H_c - (lambda/2) (F^P_{c+1} - F^P_c) + D_{c+1/2},
// which is the average (X^P + X^C)/2 plus the TVD term of Sec. 3.1.  The
// corrector's flux difference is formed first, as the scheme writes it, so
// that equal fluxes cancel exactly (y-independent data keep m_y = 0 through
// L_y, whose y-momentum flux holds the pressure).
//
// Stretched z-grid (ST): the conservative metric form of the one-column
// kernels.  L_z: flux differences of plane k over its cell width w_k, the
// one-sided derivatives over the spacing they span, the TVD flux through
// (k, k+1) weighted by its spacing over w_k and its Courant number over that
// spacing; L_y: the central z span of the warp's plane; L_x: the central z
// span of each row's plane and its CFL step 1/h_min.  The block copies the
// metric of its segment's planes after the row ring once (fill_planes).
#pragma once
#include "sweep2d_x2.cuh"
#include "sweep3d.cuh"

namespace cm {

constexpr int kRing3 = 4;                      // rows in flight per thread
// warps per block (2 halo each side): 12 warps of 168 registers run spill-free
// (measured 3.48 ms per 512 x 512 x 128 step); 16 warps would cap a thread at 128
// registers and spill ~290 bytes in the march kernel (5.95 ms)
constexpr int kNW3pDefault = 12;
// ring bytes of a block of NW warps
__host__ __device__ constexpr size_t ring3_bytes(int NW) { return (size_t)kRing3 * 5 * NW * 32 * sizeof(float2); }

// 3D state of two columns: (rho, m_x, m_y, m_z, E)
struct P5 {
    f2 r, m[3], E;
};

__device__ __forceinline__ P5 p5_right(const P5& q)
{
    return {right_of(q.r), {right_of(q.m[0]), right_of(q.m[1]), right_of(q.m[2])}, right_of(q.E)};
}
__device__ __forceinline__ P5 p5_left(const P5& q)
{
    return {left_of(q.r), {left_of(q.m[0]), left_of(q.m[1]), left_of(q.m[2])}, left_of(q.E)};
}
__device__ __forceinline__ P5 p5_sub(const P5& a, const P5& b)
{
    return {sub2f(a.r, b.r), {sub2f(a.m[0], b.m[0]), sub2f(a.m[1], b.m[1]), sub2f(a.m[2], b.m[2])}, sub2f(a.E, b.E)};
}
__device__ __forceinline__ f2 p5_dot(const P5& a, const P5& b)
{
    return fma2f(a.E, b.E, fma2f(a.m[2], b.m[2], fma2f(a.m[1], b.m[1], fma2f(a.m[0], b.m[0], mul2f(a.r, b.r)))));
}
__device__ __forceinline__ P5 p5_scale(f2 g, const P5& d)
{
    return {mul2f(g, d.r), {mul2f(g, d.m[0]), mul2f(g, d.m[1]), mul2f(g, d.m[2])}, mul2f(g, d.E)};
}
__device__ __forceinline__ P5 p5_zero()
{
    const f2 z = bc(0.f);
    return {z, {z, z, z}, z};
}
__device__ __forceinline__ P5 ld5(const float* __restrict__ base, int fs, int off)
{
    const float* s = base + off;
    return {__ldg(reinterpret_cast<const f2*>(s)),
            {__ldg(reinterpret_cast<const f2*>(s + fs)), __ldg(reinterpret_cast<const f2*>(s + 2 * fs)),
             __ldg(reinterpret_cast<const f2*>(s + 3 * fs))},
            __ldg(reinterpret_cast<const f2*>(s + 4 * fs))};
}
__device__ __forceinline__ void st5(float* __restrict__ base, int fs, int off, const P5& q)
{
    float* d = base + off;
    *reinterpret_cast<f2*>(d) = q.r;
    *reinterpret_cast<f2*>(d + fs) = q.m[0];
    *reinterpret_cast<f2*>(d + 2 * fs) = q.m[1];
    *reinterpret_cast<f2*>(d + 3 * fs) = q.m[2];
    *reinterpret_cast<f2*>(d + 4 * fs) = q.E;
}

__device__ __forceinline__ void cp_async_wait_ring3()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(kRing3 - 1) : "memory");
}

// per-thread ring [kRing3 slots][5 fields][NT threads] of float2; a thread
// reads back only what it copied itself
template <int NT>
struct Ring5 {
    static constexpr int kThreads3p = NT;
    f2* mine;
    __device__ __forceinline__ void request(int slot, const float* __restrict__ g, int fs) const
    {
        f2* d = mine + slot * 5 * kThreads3p;
        cp_async8(d, g);
        cp_async8(d + kThreads3p, g + fs);
        cp_async8(d + 2 * kThreads3p, g + 2 * fs);
        cp_async8(d + 3 * kThreads3p, g + 3 * fs);
        cp_async8(d + 4 * kThreads3p, g + 4 * fs);
        cp_async_commit();
    }
    __device__ __forceinline__ P5 take(int slot) const
    {
        const f2* d = mine + slot * 5 * kThreads3p;
        return {d[0], {d[kThreads3p], d[2 * kThreads3p], d[3 * kThreads3p]}, d[4 * kThreads3p]};
    }
};

// primitives (Sec. 2 closures): u = m/rho, T = b (E/rho - u^2/2 - g z), p = a rho T; gz = -g z
__device__ __forceinline__ void prims5(const P5& q, f2 gz, const Coef<float>& C, f2 (&u)[3], f2& T, f2& p)
{
    const f2 ri = rcp2(q.r);
    u[0] = mul2f(q.m[0], ri);
    u[1] = mul2f(q.m[1], ri);
    u[2] = mul2f(q.m[2], ri);
    const f2 ke = fma2f(u[2], u[2], fma2f(u[1], u[1], mul2f(u[0], u[0])));
    const f2 e = fma2f(q.E, ri, fma2f(ke, bc(-0.5f), gz));
    T = mul2f(bc(C.b), e);
    p = mul2f(mul2f(bc(C.a), q.r), T);
}

// F_AL of Sec. 3.1 for two columns, from the derivatives it uses:
//   g[c] = d u_c / d x_AL and gT = dT / d x_AL (one-sided along the sweep),
//   ca[d] = d u_AL / d x_d and cb[d] = d u_d / d x_d for d != AL (central across);
//   tau_{i AL} = mu (g[i] + ca[i]) (i != AL), tau_{AL AL} = mu (2 g[AL] + s div)
template <int AL>
__device__ __forceinline__ P5 flux5(const P5& q, const f2 (&u)[3], f2 p, const f2 (&g)[3], f2 gT, const f2 (&ca)[3],
                                    const f2 (&cb)[3], const Coef<float>& C)
{
    constexpr int B1 = AL == 0 ? 1 : 0, B2 = AL == 2 ? 1 : 2;  // the two directions across
    const f2 div = add2f(g[AL], add2f(cb[B1], cb[B2]));
    const f2 mu = bc(C.mu);
    f2 tau[3];
    tau[AL] = mul2f(mu, fma2f(bc(C.stokes), div, add2f(g[AL], g[AL])));
    tau[B1] = mul2f(mu, add2f(g[B1], ca[B1]));
    tau[B2] = mul2f(mu, add2f(g[B2], ca[B2]));
    P5 F;
    F.r = q.m[AL];
#pragma unroll
    for (int i = 0; i < 3; ++i) F.m[i] = fnma2f(bc(1.f), tau[i], mul2f(q.m[i], u[AL]));
    F.m[AL] = add2f(F.m[AL], p);
    const f2 work = fma2f(u[2], tau[2], fma2f(u[1], tau[1], mul2f(u[0], tau[0])));
    F.E = sub2f(fnma2f(bc(C.kth), gT, mul2f(u[AL], add2f(q.E, p))), work);
    return F;
}

// L_z (AL = 2: march z, W = y) or L_y (AL = 1: march y, W = z).  Row
// pipeline at step j (row j of the march just taken from the ring):
// F^n_{j-1} (forward along the march, central across x from shuffles and
// across W from the exchange of row j-1 one step earlier), X^P_{j-1} and its
// primitives; exchange; F^P_{j-1} (backward along the march); the TVD flux
// across (j-2, j-1) from the input state; output row j-2; H_{j-1}.  Plates:
// for L_z at the ends of the march (half-cell density, m = 0, T = T_w); for
// L_y the plate planes are W rows that pass through unchanged.
template <int AL, int kNW3p, bool ST = false>
__global__ void __launch_bounds__(kNW3p * 32, 1)
sweep3d_march_x2(Sweep3IO<float> io, const __grid_constant__ Coef<float> C, SweepCtl sc)
{
    pdl_enter();
    extern __shared__ f2 ring3_mem[];
    // [row parity][u_AL, u_W of X at row j; u_AL, u_W of X^P at row j-1][warp][lane]
    __shared__ f2 xs[2][4][kNW3p][32];
    constexpr int WD = (AL == 2) ? 1 : 2;  // direction across the warps

    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int role = halo_role<kNW3p>(w);
    const int cw = blockIdx.y * (kNW3p - 4) - 2 + w;  // W coordinate of this warp
    const int ks = blockIdx.z * io.seg;               // first output row of the segment
    const int nz = C.nz, ny = C.ny, nx = C.nx, pitch = C.pitch;
    const int fs = (int)C.fstride;
    const int ke = min(ks + io.seg, io.nmarch);
    const int i = blockIdx.x * kOutW2 - 2 + 2 * lane;  // first of the lane's two columns (even)
    int ic = i % nx;
    if (ic < 0) ic += nx;
    // W row this warp reads: periodic in y, clamped in z (out-of-range warps compute unused values)
    const int cwr = (WD == 1) ? wrap(cw, ny) : min(max(cw, 0), nz - 1);
    const bool own = lane >= 1 && lane <= 30 && i < nx && w >= 2 && w < kNW3p - 2 && cw >= 0 && cw < io.nw;
    const bool passthru = (AL == 1) && (cwr == 0 || cwr == nz - 1);  // L_y leaves the plate planes unchanged

    const float Df = sweep_delta_f32(sc, C);  // Delta = dt/2
    const float lamf = Df * ((AL == 2) ? C.inv_dz : C.inv_dy);
    const f2 lam = bc(lamf), hlam = bc(0.5f * lamf), lam2 = bc(2.f * lamf);
    const f2 mDg = bc(-Df * C.g);  // Delta times the source per unit density (L_z)
    const f2 half = bc(0.5f), z0 = bc(0.f);
    const f2 ia = bc((AL == 2) ? C.inv_dz : C.inv_dy), i2dx = bc(C.inv_2dx);
    // across W: uniform y (L_z); for L_y on a stretched grid the central span
    // of the warp's own plane
    const f2 i2dw = bc((WD == 1) ? C.inv_2dy : (ST ? C.zp[min(max(cw, 0), nz - 1)].isc : C.inv_2dz));
    // stretched L_z: plate half cells Delta / w (predictor) and Delta / (2 w) (average)
    f2 lam_bot = lam2, lam_top = lam2, hlam_bot = lam;
    if constexpr (ST && AL == 2) {
        lam_bot = bc(Df * C.zp[0].iw);
        lam_top = bc(Df * C.zp[nz - 1].iw);
        hlam_bot = bc(0.5f * Df * C.zp[0].iw);
    }

    if (sc.first && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0) step_bookkeeping(sc, C);

    // memory offset of march row j of this warp's W row
    auto row_off = [&](int j) -> int {
        if (AL == 2) return (min(max(j, 0), nz - 1) * ny + cwr) * pitch + ic;
        return (cwr * ny + wrap(j, ny)) * pitch + ic;
    };
    // -g z of march row j (L_z) or of the warp's plane (L_y)
    const f2 gzw = bc(-C.g * io.zt[(AL == 2) ? 0 : cwr]);
    auto gz_of = [&](int j) -> f2 {
        if (AL == 2) return bc(-C.g * io.zt[min(max(j, 0), nz - 1)]);
        return gzw;
    };

    const Ring5<kNW3p * 32> ring{ring3_mem + threadIdx.x};
    // stretched L_z: the block's plane cache after the ring, {1/hp, 1/w, rp, rm}
    // of planes ks - 4 .. ke (clamped); every warp marches the same rows
    float* pz = reinterpret_cast<float*>(ring3_mem + ring3_bytes(kNW3p) / sizeof(f2));
    if constexpr (ST && AL == 2) fill_planes<float, 4>(pz, C, ks, ke, true);
    auto pl = [&](int k, int q) -> float { return pz[(k - (ks - kPlaneBack)) * 4 + q]; };
    const int j0 = ks - 2;  // first step; the first stored row is ks, at step ks + 2
    for (int q = 0; q < kRing3 - 1; ++q) ring.request(q, io.in + row_off(j0 + q), fs);

    P5 Xm1 = ld5(io.in, fs, row_off(j0 - 1));  // X_{j-1}
    f2 gz1 = gz_of(j0 - 1);
    f2 u1[3], T1, p1;
    prims5(Xm1, gz1, C, u1, T1, p1);
    f2 A1 = z0, A2 = z0;        // |u_AL| + c of rows j-1, j-2
    f2 dwa1 = z0, dww1 = z0;    // d/dW of u_AL, u_W of X at row j-1 (exchanged one step earlier)
    // carried from row to row; each is replaced as soon as its new value
    // exists (which shortens what is live across the exchange)
    P5 F2 = p5_zero();   // F^n_{j-2}
    P5 FP2 = p5_zero();  // F^P_{j-2}
    P5 H = p5_zero();    // H_{j-2}
    P5 d1 = p5_zero();   // X_{j-1} - X_{j-2}
    f2 pp2[3] = {u1[0], u1[1], u1[2]}, ppT2 = T1;  // primitives of X^P_{j-2}
    f2 dd1 = z0, ss2 = z0;      // <d1, d1>, <X_{j-2} - X_{j-3}, d1>

    for (int j = j0; j <= ke + 1; ++j) {
        const int t = j - j0;
        ring.request((t + kRing3 - 1) % kRing3, io.in + row_off(j + kRing3 - 1), fs);
        cp_async_wait_ring3();
        const P5 X0 = ring.take(t % kRing3);
        const f2 gz0 = gz_of(j);
        f2 u0[3], T0, p0;
        prims5(X0, gz0, C, u0, T0, p0);
        const f2 A0 = add2f(abs2(u0[AL]), sqrt2(mul2f(bc(C.cs2), T0)));

        // row m = j-1: F^n, X^P and its primitives (roles 1, 2)
        const int m = j - 1;
        P5 XP1 = Xm1, F1 = p5_zero();
        f2 pp1[3] = {u1[0], u1[1], u1[2]}, ppT1 = T1, ppp1 = p1;
        // stretched L_z: 1/(spacing above m), 1/(spacing below m), Delta / w_m
        f2 ia_f = ia, ia_b = ia, lam_m = lam;
        if constexpr (ST && AL == 2) {
            ia_f = bc(pl(m, 0));
            ia_b = bc(pl(m - 1, 0));
            lam_m = bc(Df * pl(m, 1));
        }
        if (role >= 1) {
            f2 g[3], ca[3], cb[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) g[c] = mul2f(sub2f(u0[c], u1[c]), ia_f);
            ca[0] = mul2f(sub2f(right_of(u1[AL]), left_of(u1[AL])), i2dx);
            cb[0] = mul2f(sub2f(right_of(u1[0]), left_of(u1[0])), i2dx);
            ca[WD] = dwa1;
            cb[WD] = dww1;
            ca[AL] = cb[AL] = z0;
            F1 = flux5<AL>(Xm1, u1, p1, g, mul2f(sub2f(T0, T1), ia_f), ca, cb, C);
            if (AL == 2) {
                if (m >= 1 && m <= nz - 2) {
                    XP1.r = fnma2f(lam_m, sub2f(F1.r, F2.r), Xm1.r);
#pragma unroll
                    for (int c = 0; c < 3; ++c) XP1.m[c] = fnma2f(lam_m, sub2f(F1.m[c], F2.m[c]), Xm1.m[c]);
                    XP1.m[2] = fma2f(mDg, Xm1.r, XP1.m[2]);
                    XP1.E = fnma2f(lam_m, sub2f(F1.E, F2.E), Xm1.E);
                } else if (m <= 0) {
                    XP1.r = fnma2f(lam_bot, F1.r, Xm1.r);
                    XP1.m[0] = XP1.m[1] = XP1.m[2] = z0;
                    XP1.E = mul2f(XP1.r, bc(C.ebot));
                } else {
                    XP1.r = fma2f(lam_top, F2.r, Xm1.r);
                    XP1.m[0] = XP1.m[1] = XP1.m[2] = z0;
                    XP1.E = mul2f(XP1.r, bc(C.etop));
                }
            } else if (!passthru) {
                XP1.r = fnma2f(lam, sub2f(F1.r, F2.r), Xm1.r);
#pragma unroll
                for (int c = 0; c < 3; ++c) XP1.m[c] = fnma2f(lam, sub2f(F1.m[c], F2.m[c]), Xm1.m[c]);
                XP1.E = fnma2f(lam, sub2f(F1.E, F2.E), Xm1.E);
            }
            prims5(XP1, gz1, C, pp1, ppT1, ppp1);
            F2 = F1;
        }

        // exchange across W: u of X at row j and of X^P at row m
        f2(*buf)[kNW3p][32] = xs[j & 1];
        buf[0][w][lane] = u0[AL];
        buf[1][w][lane] = u0[WD];
        buf[2][w][lane] = pp1[AL];
        buf[3][w][lane] = pp1[WD];
        __syncthreads();
        const int wu = min(w + 1, kNW3p - 1), wd = max(w - 1, 0);
        const f2 dwa0 = mul2f(sub2f(buf[0][wu][lane], buf[0][wd][lane]), i2dw);
        const f2 dww0 = mul2f(sub2f(buf[1][wu][lane], buf[1][wd][lane]), i2dw);

        P5 d0 = p5_zero();
        f2 dd0 = z0, ss1 = z0;
        if (role == 2) {
            // F^P at row m (backward along the march)
            f2 g[3], ca[3], cb[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) g[c] = mul2f(sub2f(pp1[c], pp2[c]), ia_b);
            ca[0] = mul2f(sub2f(right_of(pp1[AL]), left_of(pp1[AL])), i2dx);
            cb[0] = mul2f(sub2f(right_of(pp1[0]), left_of(pp1[0])), i2dx);
            ca[WD] = mul2f(sub2f(buf[2][wu][lane], buf[2][wd][lane]), i2dw);
            cb[WD] = mul2f(sub2f(buf[3][wu][lane], buf[3][wd][lane]), i2dw);
            ca[AL] = cb[AL] = z0;
            const P5 FP1 = flux5<AL>(XP1, pp1, ppp1, g, mul2f(sub2f(ppT1, ppT2), ia_b), ca, cb, C);

            // TVD flux across (c, m), c = j-2, from the input state
            const int c = j - 2;
            d0 = p5_sub(X0, Xm1);
            dd0 = p5_dot(d0, d0);
            ss1 = p5_dot(d1, d0);
            P5 Dn = p5_zero();
            const bool tvd_on = (AL == 2) ? (c >= 1 && c <= nz - 3) : !passthru;
            // Courant number of interface (c, c+1): Delta over its spacing
            const f2 lamh_c = (ST && AL == 2) ? bc(Df * pl(c, 0)) : lam;
            if (tvd_on) Dn = p5_scale(tvd_G2f(ss2, ss1, dd1, mul2f(lamh_c, max2(A2, A1)), C.tvd_form), d1);
            d1 = d0;

            // output row c
            if (own && c >= ks && c < ke) {
                P5 Xn;
                const bool interior = (AL == 2) ? (c >= 1 && c <= nz - 2) : !passthru;
                if (interior) {
                    if constexpr (ST && AL == 2) {
                        // Delta / (2 w_c) on the corrector's difference; the TVD flux
                        // through (c, c+1) weighted by its spacing over w_c
                        const f2 hl = bc(0.5f * Df * pl(c, 1)), rp = bc(pl(c, 2));
                        Xn.r = fma2f(rp, Dn.r, fnma2f(hl, sub2f(FP1.r, FP2.r), H.r));
#pragma unroll
                        for (int q = 0; q < 3; ++q) Xn.m[q] = fma2f(rp, Dn.m[q], fnma2f(hl, sub2f(FP1.m[q], FP2.m[q]), H.m[q]));
                        Xn.E = fma2f(rp, Dn.E, fnma2f(hl, sub2f(FP1.E, FP2.E), H.E));
                    } else {
                        Xn.r = add2f(fnma2f(hlam, sub2f(FP1.r, FP2.r), H.r), Dn.r);
#pragma unroll
                        for (int q = 0; q < 3; ++q) Xn.m[q] = add2f(fnma2f(hlam, sub2f(FP1.m[q], FP2.m[q]), H.m[q]), Dn.m[q]);
                        Xn.E = add2f(fnma2f(hlam, sub2f(FP1.E, FP2.E), H.E), Dn.E);
                    }
                } else if (AL == 2) {
                    // plates: rho = (rho^P + rho^C)/2 with the half-cell corrector
                    Xn.r = (c == 0) ? fnma2f(hlam_bot, FP1.r, H.r) : H.r;
                    Xn.m[0] = Xn.m[1] = Xn.m[2] = z0;
                    Xn.E = mul2f(Xn.r, bc(c == 0 ? C.ebot : C.etop));
                } else {
                    Xn = H;  // plate planes of L_y: the input row
                }
                st5(io.out, fs, row_off(c), Xn);
            }

            // H of row m for the next step
            const bool interior_m = (AL == 2) ? (m >= 1 && m <= nz - 2) : !passthru;
            if (interior_m && ST && AL == 2) {
                // the TVD flux through (m-1, m) weighted by its spacing over w_m
                const f2 rm = bc(pl(m, 3));
                H.r = fnma2f(rm, Dn.r, mul2f(half, add2f(XP1.r, Xm1.r)));
                H.m[0] = fnma2f(rm, Dn.m[0], mul2f(half, add2f(XP1.m[0], Xm1.m[0])));
                H.m[1] = fnma2f(rm, Dn.m[1], mul2f(half, add2f(XP1.m[1], Xm1.m[1])));
                H.m[2] = fnma2f(rm, Dn.m[2], mul2f(half, fma2f(mDg, XP1.r, add2f(XP1.m[2], Xm1.m[2]))));
                H.E = fnma2f(rm, Dn.E, mul2f(half, add2f(XP1.E, Xm1.E)));
            } else if (interior_m) {
                H.r = sub2f(mul2f(half, add2f(XP1.r, Xm1.r)), Dn.r);
                H.m[0] = sub2f(mul2f(half, add2f(XP1.m[0], Xm1.m[0])), Dn.m[0]);
                H.m[1] = sub2f(mul2f(half, add2f(XP1.m[1], Xm1.m[1])), Dn.m[1]);
                if (AL == 2)
                    H.m[2] = sub2f(mul2f(half, fma2f(mDg, XP1.r, add2f(XP1.m[2], Xm1.m[2]))), Dn.m[2]);
                else
                    H.m[2] = sub2f(mul2f(half, add2f(XP1.m[2], Xm1.m[2])), Dn.m[2]);
                H.E = sub2f(mul2f(half, add2f(XP1.E, Xm1.E)), Dn.E);
            } else if (AL == 2) {
                H = p5_zero();
                H.r = mul2f(half, add2f(XP1.r, Xm1.r));
            } else {
                H = Xm1;
            }
            FP2 = FP1;
        }

        Xm1 = X0;
        gz1 = gz0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            u1[c] = u0[c];
            pp2[c] = pp1[c];
        }
        T1 = T0;
        p1 = p0;
        A2 = A1;
        A1 = A0;
        dwa1 = dwa0;
        dww1 = dww0;
        ppT2 = ppT1;
        dd1 = dd0;
        ss2 = ss1;
    }
    cp_async_drain();  // rows requested past the segment end
}

// L_x in 3D, march z, warps across y; the x stencil across lanes as in the
// 2D packed x sweep, plate planes pass through.  Row pipeline at step j:
// F^n of row j-1 (forward x; d/dz from rows j, j-2; d/dy from the exchange
// of row j-1 one step earlier), X^P, the TVD term along x and
//   K_{j-1} = (X^P + X)_{j-1}/2 + D_{i+1/2} - D_{i-1/2};
// exchange; then for row c = j-2, F^P (backward x; d/dz of X^P from rows j-1,
// j-3; d/dy from the exchange of row j-2) and X_new_c = K_c - (lambda/2)
// (F^P_{i+1} - F^P_i).  The last sweep of a step (sc.last) also reduces the
// next dt from the stored nodes.
template <int kNW3p, bool ST = false>
__global__ void __launch_bounds__(kNW3p * 32, 1)
sweep3d_x_x2(Sweep3IO<float> io, const __grid_constant__ Coef<float> C, SweepCtl sc)
{
    pdl_enter();
    extern __shared__ f2 ring3_mem[];
    // [row parity][u_x, u_y of X at row j; u_x, u_y of X^P at row j-1][warp][lane]
    __shared__ f2 xs[2][4][kNW3p][32];
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int role = halo_role<kNW3p>(w);
    const int cw = blockIdx.y * (kNW3p - 4) - 2 + w;  // y row of this warp
    const int ks = blockIdx.z * io.seg;
    const int nz = C.nz, ny = C.ny, nx = C.nx, pitch = C.pitch;
    const int fs = (int)C.fstride;
    const int ke = min(ks + io.seg, nz);
    const int i = blockIdx.x * kOutW2 - 2 + 2 * lane;
    int ic = i % nx;
    if (ic < 0) ic += nx;
    const int cwr = wrap(cw, ny);
    const bool own = lane >= 1 && lane <= 30 && i < nx && w >= 2 && w < kNW3p - 2 && cw < ny;
    const bool want_dt = sc.last != 0;

    const float lamf = sweep_delta_f32(sc, C) * C.inv_dx;  // Delta / dx, Delta = dt/2
    const f2 lam = bc(lamf), hlam = bc(0.5f * lamf), half = bc(0.5f), z0 = bc(0.f);
    const f2 idx_ = bc(C.inv_dx), i2dy = bc(C.inv_2dy), i2dz = bc(C.inv_2dz);
    if (sc.first && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0) step_bookkeeping(sc, C);
    auto row_off = [&](int k) -> int { return (min(max(k, 0), nz - 1) * ny + cwr) * pitch + ic; };
    auto gz_of = [&](int k) -> f2 { return bc(-C.g * io.zt[min(max(k, 0), nz - 1)]); };

    // next dt: running maxima of |u_x| + c, |u_y| + c, |u_z| + c over the
    // stored nodes (NaN-propagating), times 1/dx, 1/dy, 1/dz once at the end
    // (equal to the maximum of the per-node products: rounding is monotone)
    float ax = 0.f, ay = 0.f, az = 0.f;
    const Ring5<kNW3p * 32> ring{ring3_mem + threadIdx.x};
    // stretched grid: the block's plane cache after the ring, {1/(central z
    // span), 1/(smaller spacing)} of planes ks - 4 .. ke (clamped)
    float* pz = reinterpret_cast<float*>(ring3_mem + ring3_bytes(kNW3p) / sizeof(f2));
    if constexpr (ST) fill_planes<float, 2>(pz, C, ks, ke, false);
    auto pl = [&](int k, int q) -> float { return pz[(k - (ks - kPlaneBack)) * 2 + q]; };
    const int j0 = ks - 2;
    for (int q = 0; q < kRing3 - 1; ++q) ring.request(q, io.in + row_off(j0 + q), fs);

    P5 Xm1 = ld5(io.in, fs, row_off(j0 - 1));
    f2 gz1 = gz_of(j0 - 1), gz2 = gz1;
    f2 u1[3], T1, p1;
    prims5(Xm1, gz1, C, u1, T1, p1);
    f2 u2x = u1[0], u2z = u1[2];            // u_x, u_z of X at row j-2
    f2 dwx1 = z0, dwy1 = z0;                // d/dy of u_x, u_y of X at row j-1
    P5 XP2 = Xm1, K2 = Xm1;                 // X^P and K of row j-2
    f2 pp2[3] = {u1[0], u1[1], u1[2]}, ppT2 = T1, ppp2 = p1;  // primitives of X^P_{j-2}
    f2 pp3x = u1[0], pp3z = u1[2];          // u_x, u_z of X^P at row j-3
    f2 dwpx2 = z0, dwpy2 = z0;              // d/dy of u_x, u_y of X^P at row j-2

    for (int j = j0; j <= ke + 1; ++j) {
        const int t = j - j0;
        ring.request((t + kRing3 - 1) % kRing3, io.in + row_off(j + kRing3 - 1), fs);
        cp_async_wait_ring3();
        const P5 X0 = ring.take(t % kRing3);
        const f2 gz0 = gz_of(j);
        f2 u0[3], T0, p0;
        prims5(X0, gz0, C, u0, T0, p0);

        // row m = j-1: F^n (forward x), X^P, the TVD term along x and K
        const int m = j - 1;
        const bool interior_m = m >= 1 && m <= nz - 2;
        P5 XP1 = Xm1, K1 = Xm1;  // plate planes pass through
        f2 pp1[3] = {u1[0], u1[1], u1[2]}, ppT1 = T1, ppp1 = p1;
        if (role >= 1) {
            if (interior_m) {
                f2 g[3], ca[3], cb[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) g[c] = mul2f(sub2f(right_of(u1[c]), u1[c]), idx_);
                ca[1] = dwx1;
                cb[1] = dwy1;
                const f2 i2dz_m = ST ? bc(pl(m, 0)) : i2dz;  // 1/(central z span) of plane m
                ca[2] = mul2f(sub2f(u0[0], u2x), i2dz_m);
                cb[2] = mul2f(sub2f(u0[2], u2z), i2dz_m);
                ca[0] = cb[0] = z0;
                const P5 F1 = flux5<0>(Xm1, u1, p1, g, mul2f(sub2f(right_of(T1), T1), idx_), ca, cb, C);
                const P5 Fl = p5_left(F1);
                XP1.r = fnma2f(lam, sub2f(F1.r, Fl.r), Xm1.r);
#pragma unroll
                for (int c = 0; c < 3; ++c) XP1.m[c] = fnma2f(lam, sub2f(F1.m[c], Fl.m[c]), Xm1.m[c]);
                XP1.E = fnma2f(lam, sub2f(F1.E, Fl.E), Xm1.E);
                if (role == 2) {
                    // TVD along x on row m from the input state
                    const P5 dr = p5_sub(p5_right(Xm1), Xm1);
                    const f2 dd = p5_dot(dr, dr);
                    const f2 sp = p5_dot(p5_left(dr), dr);
                    const f2 A = add2f(abs2(u1[0]), sqrt2(mul2f(bc(C.cs2), T1)));
                    const f2 G = tvd_G2f(sp, right_of(sp), dd, mul2f(lam, max2(A, right_of(A))), C.tvd_form);
                    const P5 Dn = p5_scale(G, dr);
                    const P5 Dl = p5_left(Dn);
                    K1.r = fma2f(half, add2f(XP1.r, Xm1.r), sub2f(Dn.r, Dl.r));
#pragma unroll
                    for (int c = 0; c < 3; ++c) K1.m[c] = fma2f(half, add2f(XP1.m[c], Xm1.m[c]), sub2f(Dn.m[c], Dl.m[c]));
                    K1.E = fma2f(half, add2f(XP1.E, Xm1.E), sub2f(Dn.E, Dl.E));
                }
            }
            prims5(XP1, gz1, C, pp1, ppT1, ppp1);
        }

        // exchange across y: u_x, u_y of X at row j and of X^P at row m
        f2(*buf)[kNW3p][32] = xs[j & 1];
        buf[0][w][lane] = u0[0];
        buf[1][w][lane] = u0[1];
        buf[2][w][lane] = pp1[0];
        buf[3][w][lane] = pp1[1];
        __syncthreads();
        const int wu = min(w + 1, kNW3p - 1), wd = max(w - 1, 0);
        const f2 dwx0 = mul2f(sub2f(buf[0][wu][lane], buf[0][wd][lane]), i2dy);
        const f2 dwy0 = mul2f(sub2f(buf[1][wu][lane], buf[1][wd][lane]), i2dy);
        const f2 dwpx1 = mul2f(sub2f(buf[2][wu][lane], buf[2][wd][lane]), i2dy);
        const f2 dwpy1 = mul2f(sub2f(buf[3][wu][lane], buf[3][wd][lane]), i2dy);

        if (role == 2) {
            // row c = j-2: F^P (backward x), corrector, output
            const int c = j - 2;
            P5 Xn = K2;
            if (c >= 1 && c <= nz - 2) {
                f2 g[3], ca[3], cb[3];
#pragma unroll
                for (int q = 0; q < 3; ++q) g[q] = mul2f(sub2f(pp2[q], left_of(pp2[q])), idx_);
                ca[1] = dwpx2;
                cb[1] = dwpy2;
                const f2 i2dz_c = ST ? bc(pl(c, 0)) : i2dz;  // 1/(central z span) of plane c
                ca[2] = mul2f(sub2f(pp1[0], pp3x), i2dz_c);
                cb[2] = mul2f(sub2f(pp1[2], pp3z), i2dz_c);
                ca[0] = cb[0] = z0;
                const P5 FP = flux5<0>(XP2, pp2, ppp2, g, mul2f(sub2f(ppT2, left_of(ppT2)), idx_), ca, cb, C);
                const P5 FPr = p5_right(FP);
                Xn.r = fnma2f(hlam, sub2f(FPr.r, FP.r), K2.r);
#pragma unroll
                for (int q = 0; q < 3; ++q) Xn.m[q] = fnma2f(hlam, sub2f(FPr.m[q], FP.m[q]), K2.m[q]);
                Xn.E = fnma2f(hlam, sub2f(FPr.E, FP.E), K2.E);
            }
            const bool keep = own && c >= ks && c < ke;
            if (keep) st5(io.out, fs, row_off(c), Xn);
            if (want_dt) {
                // every lane of a storing warp evaluates; only kept nodes count
                f2 un[3], Tn, pn;
                prims5(Xn, gz2, C, un, Tn, pn);
                const f2 cs = sqrt2(mul2f(bc(C.cs2), Tn));
                const float vx = fmax_nan(fabsf(un[0].x) + cs.x, fabsf(un[0].y) + cs.y);
                const float vy = fmax_nan(fabsf(un[1].x) + cs.x, fabsf(un[1].y) + cs.y);
                float vz = fmax_nan(fabsf(un[2].x) + cs.x, fabsf(un[2].y) + cs.y);
                if constexpr (ST) vz *= pl(c, 1);  // the plane's CFL z step, 1/h_min
                if (keep) {
                    ax = fmax_nan(ax, vx);
                    ay = fmax_nan(ay, vy);
                    az = fmax_nan(az, vz);
                }
            }
        }

        Xm1 = X0;
        gz2 = gz1;
        gz1 = gz0;
        u2x = u1[0];
        u2z = u1[2];
#pragma unroll
        for (int c = 0; c < 3; ++c) u1[c] = u0[c];
        T1 = T0;
        p1 = p0;
        dwx1 = dwx0;
        dwy1 = dwy0;
        XP2 = XP1;
        K2 = K1;
        pp3x = pp2[0];
        pp3z = pp2[2];
#pragma unroll
        for (int c = 0; c < 3; ++c) pp2[c] = pp1[c];
        ppT2 = ppT1;
        ppp2 = ppp1;
        dwpx2 = dwpx1;
        dwpy2 = dwpy1;
    }
    cp_async_drain();
    if (want_dt) {
        const float r = fmax_nan(fmax_nan(ax * C.inv_dx, ay * C.inv_dy), ST ? az : az * C.inv_dz);
        block_rmax_dt(r, sc.ctl, sc.slot_in ^ 1);
    }
}

}  // namespace cm
