// sweep2d_x2.cuh -- FP32 sweeps with two columns per lane (even nx).
//
// Same scheme and row pipeline as sweep2d.cuh, but every lane carries the
// state of two adjacent columns as float2 and does the arithmetic with the
// packed FP32x2 instructions of sm_100+ (__fadd2_rn, __fmul2_rn,
// __ffma2_rn): one instruction updates both columns.  A warp covers 64
// columns; the stencil and the cross derivatives reach two columns, one
// lane, to each side, so lanes 1..30 produce 60 output columns per strip.
// Neighbour columns come from one shuffle per exchanged quantity:
//   value at c+1 = (own.y, lane+1 .x),  value at c-1 = (lane-1 .y, own.x).
// Loads and stores are 8-byte vectors (the strip origin is even).
#pragma once
#include "cm_device.cuh"
#include "sweep2d_x2_types.h"

namespace cm {


typedef float2 f2;

__device__ __forceinline__ f2 bc(float s) { return make_float2(s, s); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
// a - b, rounded once
__device__ __forceinline__ f2 sub2(f2 a, f2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
// a - s*b
__device__ __forceinline__ f2 fnma2(f2 s, f2 b, f2 a) { return __ffma2_rn(make_float2(-s.x, -s.y), b, a); }

__device__ __forceinline__ f2 right_of(f2 v) { return make_float2(v.y, __shfl_down_sync(0xffffffffu, v.x, 1)); }
__device__ __forceinline__ f2 left_of(f2 v) { return make_float2(__shfl_up_sync(0xffffffffu, v.y, 1), v.x); }

struct S2 { f2 r, mx, mz, E; };

__device__ __forceinline__ S2 right_of(const S2& q) { return {right_of(q.r), right_of(q.mx), right_of(q.mz), right_of(q.E)}; }
__device__ __forceinline__ S2 left_of(const S2& q) { return {left_of(q.r), left_of(q.mx), left_of(q.mz), left_of(q.E)}; }

__device__ __forceinline__ S2 ld2(const float* __restrict__ base, int fs, int off)
{
    const float* s = base + off;
    return {__ldg(reinterpret_cast<const f2*>(s)), __ldg(reinterpret_cast<const f2*>(s + fs)),
            __ldg(reinterpret_cast<const f2*>(s + 2 * fs)), __ldg(reinterpret_cast<const f2*>(s + 3 * fs))};
}

__device__ __forceinline__ void st2(float* __restrict__ base, int fs, int off, const S2& q)
{
    float* d = base + off;
    *reinterpret_cast<f2*>(d) = q.r;
    *reinterpret_cast<f2*>(d + fs) = q.mx;
    *reinterpret_cast<f2*>(d + 2 * fs) = q.mz;
    *reinterpret_cast<f2*>(d + 3 * fs) = q.E;
}

// reciprocal and square root on the special-function unit alone (one MUFU
// instruction each, ~1 ulp, denormals flushed): the FP32 path's tolerance
// is far above that
__device__ __forceinline__ float rcp_fast(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float sqrt_fast(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ f2 rcp2(f2 a) { return make_float2(rcp_fast(a.x), rcp_fast(a.y)); }

// primitives: u = m/rho, T = b (E/rho - u^2/2 - g z), p = a rho T
__device__ __forceinline__ void prims2(const S2& q, f2 gz, const Coef<float>& C, f2& ux, f2& uz, f2& T, f2& p)
{
    const f2 ri = rcp2(q.r);
    ux = mul2(q.mx, ri);
    uz = mul2(q.mz, ri);
    const f2 ke = fma2(ux, ux, mul2(uz, uz));
    const f2 e = fma2(q.E, ri, fma2(ke, bc(-0.5f), gz));  // gz = -g z
    T = mul2(bc(C.b), e);
    p = mul2(mul2(bc(C.a), q.r), T);
}

// F_z (one-sided d/dz inside, central d/dx across)
__device__ __forceinline__ S2 flux_z2(const S2& q, f2 ux, f2 uz, f2 p, f2 dz_ux, f2 dz_uz, f2 dz_T, f2 dx_ux, f2 dx_uz,
                                      const Coef<float>& C)
{
    const f2 div = add2(dx_ux, dz_uz);
    const f2 tx = mul2(bc(C.mu), add2(dz_ux, dx_uz));
    const f2 tz = mul2(bc(C.mu), fma2(bc(C.stokes), div, add2(dz_uz, dz_uz)));
    S2 F;
    F.r = q.mz;
    F.mx = fnma2(bc(1.f), tx, mul2(q.mx, uz));
    F.mz = add2(fnma2(bc(1.f), tz, mul2(q.mz, uz)), p);
    F.E = sub2(fnma2(bc(C.kth), dz_T, mul2(uz, add2(q.E, p))), fma2(ux, tx, mul2(uz, tz)));
    return F;
}

// F_x (one-sided d/dx inside, central d/dz across)
__device__ __forceinline__ S2 flux_x2(const S2& q, f2 ux, f2 uz, f2 p, f2 dx_ux, f2 dx_uz, f2 dx_T, f2 dz_ux, f2 dz_uz,
                                      const Coef<float>& C)
{
    const f2 div = add2(dx_ux, dz_uz);
    const f2 tx = mul2(bc(C.mu), fma2(bc(C.stokes), div, add2(dx_ux, dx_ux)));
    const f2 tz = mul2(bc(C.mu), add2(dx_uz, dz_ux));
    S2 F;
    F.r = q.mx;
    F.mx = add2(fnma2(bc(1.f), tx, mul2(q.mx, ux)), p);
    F.mz = fnma2(bc(1.f), tz, mul2(q.mz, ux));
    F.E = sub2(fnma2(bc(C.kth), dx_T, mul2(ux, add2(q.E, p))), fma2(ux, tx, mul2(uz, tz)));
    return F;
}

__device__ __forceinline__ f2 dot2(const S2& a, const S2& b)
{
    return fma2(a.E, b.E, fma2(a.mz, b.mz, fma2(a.mx, b.mx, mul2(a.r, b.r))));
}

// TVD coefficient G of the flux G dX, both columns at once:
//   C = c(1 - c), c = min(Co, 1/2);  phi(s) = clamp(2 s / dd, 0, 1)
//   Davis form: G = C (2 - phi(sp) - phi(sm)) / 2;  printed form: C (1 - phi(sp + sm)) / 2
// One reciprocal of dd serves both ratios.  dd = 0 (dX = 0) gives 0 * inf =
// NaN, which the clamp maps to 0; the flux G dX is 0 there anyway.
__device__ __forceinline__ float clamp01(float x) { return fminf(fmaxf(x, 0.f), 1.f); }

__device__ __forceinline__ f2 tvd_G2(f2 sp, f2 sm, f2 dd, f2 Co, int form)
{
    const f2 c = make_float2(fminf(Co.x, 0.5f), fminf(Co.y, 0.5f));
    const f2 hC = mul2(make_float2(0.5f, 0.5f), fma2(make_float2(-c.x, -c.y), c, c));  // C/2
    const f2 r2 = mul2(make_float2(2.f, 2.f), rcp2(dd));
    if (form == 0) {
        const f2 a = mul2(sp, r2), b = mul2(sm, r2);
        const f2 phis = make_float2(clamp01(a.x) + clamp01(b.x), clamp01(a.y) + clamp01(b.y));
        return mul2(hC, sub2(make_float2(2.f, 2.f), phis));
    }
    if (form == 1) {
        const f2 a = mul2(add2(sp, sm), r2);
        return mul2(hC, sub2(make_float2(1.f, 1.f), make_float2(clamp01(a.x), clamp01(a.y))));
    }
    return make_float2(0.f, 0.f);
}

__device__ __forceinline__ f2 abs2(f2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ f2 max2(f2 a, f2 b) { return make_float2(fmaxf(a.x, b.x), fmaxf(a.y, b.y)); }
__device__ __forceinline__ f2 sqrt2(f2 a) { return make_float2(sqrt_fast(a.x), sqrt_fast(a.y)); }
__device__ __forceinline__ S2 scale2(f2 g, const S2& d) { return {mul2(g, d.r), mul2(g, d.mx), mul2(g, d.mz), mul2(g, d.E)}; }
__device__ __forceinline__ S2 diff2(const S2& a, const S2& b) { return {sub2(a.r, b.r), sub2(a.mx, b.mx), sub2(a.mz, b.mz), sub2(a.E, b.E)}; }

struct SweepIO2 {
    const float* in;
    float* out;
    const float* zt;
    int seg_rows;
    int nstrips;  // ceil(nx / kOutW2)
};

// ---- asynchronous row loads: each lane copies its own two columns of the
// four fields into a per-thread ring in shared memory (cp.async), kRing rows
// deep, so a row is requested kRing-1 rows before it is consumed without
// holding registers.  A lane only ever reads back what it copied itself, so
// cp.async.wait_group is the only ordering needed.
constexpr int kRing = 4;

__device__ __forceinline__ void cp_async8(f2* smem, const float* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_ring() { asm volatile("cp.async.wait_group %0;\n" ::"n"(kRing - 1) : "memory"); }
__device__ __forceinline__ void cp_async_drain() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

constexpr int kThreads2 = kWarpsPerBlock * 32;  // block size of the packed kernels

// per-thread ring [kRing slots][4 fields][kThreads2] of float2 in shared
// memory; the field stride is a compile-time constant
struct RowRing {
    f2* mine;  // this thread's element of slot 0, field 0
    __device__ __forceinline__ f2* at(int slot, int f) const { return mine + (slot * 4 + f) * kThreads2; }
    __device__ __forceinline__ void request(int slot, const float* __restrict__ g, int fs) const
    {
        f2* d = mine + slot * 4 * kThreads2;
        cp_async8(d, g);
        cp_async8(d + kThreads2, g + fs);
        cp_async8(d + 2 * kThreads2, g + 2 * fs);
        cp_async8(d + 3 * kThreads2, g + 3 * fs);
        cp_async_commit();
    }
    __device__ __forceinline__ S2 take(int slot) const
    {
        const f2* d = mine + slot * 4 * kThreads2;
        return {d[0], d[kThreads2], d[2 * kThreads2], d[3 * kThreads2]};
    }
};

// Stretched z-grid: each warp copies the metric of the planes its segment
// touches (ks - 3 .. ke + 1, clamped) into its own slice of shared memory,
// after the row ring, so that every row reads it by broadcast.  NV values
// per plane; entry e holds plane clamp(ks - 3 + e).
constexpr int kPlaneBack2 = 3;
__host__ __device__ constexpr int plane_cap2(int seg_rows) { return seg_rows + kPlaneBack2 + 2; }
template <int NV>
__device__ __forceinline__ float* plane_cache2(f2* ring_mem, int seg_rows)
{
    return reinterpret_cast<float*>(ring_mem + kRing * 4 * kThreads2) + (threadIdx.x >> 5) * plane_cap2(seg_rows) * NV;
}

// A segment is "interior" when none of its pipeline rows (ks-5 .. ke+4,
// prefetch included) touches a plate or leaves the grid: its steps need no
// plate rules, no row clamping and no range tests.
__device__ __forceinline__ bool interior_segment(int ks, int ke, int nz) { return ks >= 5 && ke <= nz - 5; }

// L_z(Delta), FP32, two columns per lane.  Row pipeline at step j (row j
// just taken from the ring):
//   F^n_{j-1}, X^P_{j-1}, F^P_{j-1}; TVD flux D across (j-2, j-1);
//   output X_new_{j-2} = H_{j-2} - (lambda/2) F^P_{j-1} + D;
//   H_{j-1} = (X^P + X + Delta S^P + lambda F^P)_{j-1} / 2 - D,
// which is the average (X^P + X^C)/2 plus the TVD term of Sec. 3.1 with the
// corrector split into its two rows.
// one warp's segment of the z sweep: columns of strip `strip`, output rows
// [ks, ks + seg_rows); `lead` marks the one thread block that does the
// per-step bookkeeping of a first sweep.  ST: stretched z-grid (C.zp):
// flux differences of plane k over its cell width w_k,
// one-sided derivatives over the spacing they span, TVD fluxes weighted by
// spacing over width, Courant numbers over the interface spacing.
template <bool ST = false>
__device__ __forceinline__ void z2_body(const float* __restrict__ in, float* __restrict__ out, const Coef<float>& C,
                                        const SweepCtl& sc, int strip, int ks, int seg_rows, bool lead)
{
    extern __shared__ f2 ring_mem[];
    SweepIO2 io;
    io.in = in;
    io.out = out;
    const int lane = threadIdx.x & 31;
    const int nz = C.nz, nx = C.nx, pitch = C.pitch;
    const int fs = (int)C.fstride;
    const int ke = min(ks + seg_rows, nz);
    const int i = strip * kOutW2 - 2 + 2 * lane;  // first of the lane's two columns (even)
    int ic = i % nx;
    if (ic < 0) ic += nx;
    const bool own = lane >= 1 && lane <= 30 && i < nx;

    const double dt = step_dt(sc.ctl, sc.slot_in, C.cfl, C.dt_fixed);
    const double Delta = sc.Delta > 0.0 ? sc.Delta : 0.5 * dt;
    const float lamf = (float)(Delta / C.dz);
    const f2 lam = bc(lamf), hlam = bc(0.5f * lamf), lam2 = bc(2.f * lamf);
    const f2 mDg = bc(-(float)Delta * C.g);  // Delta * (source per unit density)
    const f2 half = bc(0.5f), idz = bc(C.inv_dz), i2dx = bc(C.inv_2dx);
    const float Df = (float)Delta;
    // plate half cells: Delta / w (predictor) and Delta / (2 w) (corrector average)
    f2 lam_bot = lam2, lam_top = lam2, hlam_bot = lam;
    if constexpr (ST) {
        lam_bot = bc(Df * C.zp[0].iw);
        lam_top = bc(Df * C.zp[nz - 1].iw);
        hlam_bot = bc(0.5f * Df * C.zp[0].iw);
    }

    if (sc.first && lead && threadIdx.x == 0) {
        sc.ctl->dt_slot[sc.slot_in ^ 1] = 0x7FF0000000000000ULL;
        sc.ctl->t += dt;
        sc.ctl->steps += 1.0;
    }
    if (ks >= nz) return;  // warp-uniform; no block barrier in this sweep

    const RowRing ring{ring_mem + threadIdx.x};
    auto row_off = [&](int j) { return min(max(j, 0), nz - 1) * pitch + ic; };
    // stretched: this warp's plane cache {1/hp, 1/w, rp, rm, z}
    float* pc = ST ? plane_cache2<5>(ring_mem, seg_rows) : nullptr;
    if constexpr (ST) {
        for (int e = lane; e < ke - ks + kPlaneBack2 + 2; e += 32) {
            const Plane<float>& P = C.zp[min(max(ks - kPlaneBack2 + e, 0), nz - 1)];
            pc[e * 5 + 0] = P.ihp;
            pc[e * 5 + 1] = P.iw;
            pc[e * 5 + 2] = P.rp;
            pc[e * 5 + 3] = P.rm;
            pc[e * 5 + 4] = P.z;
        }
        __syncwarp();
    }
    auto pv = [&](int k, int q) { return pc[(k - (ks - kPlaneBack2)) * 5 + q]; };
    auto gz_of = [&](int j) {
        if constexpr (ST) return bc(-C.g * pv(j, 4));
        else return bc(-C.g * ((float)min(max(j, 0), nz - 1) * C.hz));
    };
    // the first step is j0 = ks - 1 (primed with row ks - 2): no output row
    // >= ks uses anything an earlier step would produce
    const int j0 = ks - 1;

    for (int q = 0; q < kRing - 1; ++q) ring.request(q, io.in + row_off(j0 + q), fs);

    const f2 z0 = bc(0.f);
    S2 Xm1 = ld2(io.in, fs, row_off(j0 - 1));  // X_{j-1} (primed with row j0-1)
    f2 ux1, uz1, T1, p1;                       // primitives of X_{j-1}
    f2 gz1 = gz_of(j0 - 1);                    // -g z of row j-1
    prims2(Xm1, gz1, C, ux1, uz1, T1, p1);
    f2 A1 = z0, A2 = z0;                       // |u_z| + c of rows j-1, j-2
    S2 F2 = {z0, z0, z0, z0};
    f2 ppux2 = ux1, ppuz2 = uz1, ppT2 = T1;    // primitives of X^P_{j-2}
    S2 H = {z0, z0, z0, z0};                   // H_{j-2}
    S2 d1 = {z0, z0, z0, z0};
    f2 dd1 = z0, ss2 = z0;
    const float* gnext = io.in + row_off(j0 + kRing - 1);  // next row to request (interior path)
    float* gout = io.out + (long long)(j0 - 2) * pitch + i;  // output row of the current step (used only when it exists)

    // one step of the pipeline; edge: plate rules and range tests; store: the
    // step has an output row; ramp 1 / 2: the first / second step of an
    // interior segment, which skip what no stored row uses (1: X^P, F^P, the
    // TVD coefficient and H; 2: F^P, the TVD coefficient and H)
    auto row_step = [&](const int j, auto edge_tag, auto store_tag, auto ramp_tag) {
        constexpr bool edge = decltype(edge_tag)::value;
        constexpr bool store = decltype(store_tag)::value;
        constexpr int ramp = decltype(ramp_tag)::value;
        const int t = j - j0;
        if (edge) {
            ring.request((t + kRing - 1) % kRing, io.in + row_off(j + kRing - 1), fs);
        } else {
            ring.request((t + kRing - 1) % kRing, gnext, fs);
            gnext += pitch;
        }
        cp_async_wait_ring();
        const S2 X0 = ring.take(t % kRing);
        f2 gz0;
        if constexpr (ST) gz0 = gz_of(j);
        else gz0 = edge ? gz_of(j) : bc(-C.g * ((float)j * C.hz));

        f2 ux0, uz0, T0, p0;
        prims2(X0, gz0, C, ux0, uz0, T0, p0);
        const f2 A0 = add2(abs2(uz0), sqrt2(mul2(bc(C.cs2), T0)));

        // row m = j-1: F^n (forward z, central x), X^P, F^P (backward z)
        const int m = j - 1;
        // stretched: planes m and c = m - 1 from the warp's cache
        f2 lam_m = lam, idz_f = idz, idz_b = idz;  // Delta/w_m, 1/(spacing above m), 1/(spacing below m)
        if constexpr (ST) {
            lam_m = bc(Df * pv(m, 1));
            idz_f = bc(pv(m, 0));
            idz_b = bc(pv(m - 1, 0));
        }
        const f2 dxux1 = mul2(sub2(right_of(ux1), left_of(ux1)), i2dx);
        const f2 dxuz1 = mul2(sub2(right_of(uz1), left_of(uz1)), i2dx);
        const S2 F1 = flux_z2(Xm1, ux1, uz1, p1, mul2(sub2(ux0, ux1), idz_f), mul2(sub2(uz0, uz1), idz_f),
                              mul2(sub2(T0, T1), idz_f), dxux1, dxuz1, C);
        S2 XP1 = Xm1;
        const bool interior_m = !edge || (m >= 1 && m <= nz - 2);
        if (ramp == 1) {
        } else if (interior_m) {
            XP1.r = fnma2(lam_m, sub2(F1.r, F2.r), Xm1.r);
            XP1.mx = fnma2(lam_m, sub2(F1.mx, F2.mx), Xm1.mx);
            XP1.mz = fma2(mDg, Xm1.r, fnma2(lam_m, sub2(F1.mz, F2.mz), Xm1.mz));
            XP1.E = fnma2(lam_m, sub2(F1.E, F2.E), Xm1.E);
        } else if (m <= 0) {
            XP1.r = fnma2(lam_bot, F1.r, Xm1.r);
            XP1.mx = z0; XP1.mz = z0;
            XP1.E = mul2(XP1.r, bc(C.ebot));
        } else {
            XP1.r = fma2(lam_top, F2.r, Xm1.r);
            XP1.mx = z0; XP1.mz = z0;
            XP1.E = mul2(XP1.r, bc(C.etop));
        }
        f2 ppux1 = z0, ppuz1 = z0, ppT1 = z0, ppp1 = z0;
        if (ramp != 1) prims2(XP1, gz1, C, ppux1, ppuz1, ppT1, ppp1);
        S2 FP1 = {z0, z0, z0, z0};
        if (ramp == 0) {
            const f2 dxppux1 = mul2(sub2(right_of(ppux1), left_of(ppux1)), i2dx);
            const f2 dxppuz1 = mul2(sub2(right_of(ppuz1), left_of(ppuz1)), i2dx);
            FP1 = flux_z2(XP1, ppux1, ppuz1, ppp1, mul2(sub2(ppux1, ppux2), idz_b), mul2(sub2(ppuz1, ppuz2), idz_b),
                          mul2(sub2(ppT1, ppT2), idz_b), dxppux1, dxppuz1, C);
        }

        // TVD flux across (j-2, j-1) from the input state
        const S2 d0 = diff2(X0, Xm1);
        const f2 dd0 = dot2(d0, d0);
        const f2 ss1 = ramp == 1 ? z0 : dot2(d1, d0);
        const int c = j - 2;
        S2 Dn = {z0, z0, z0, z0};
        if (ramp == 0 && (!edge || (c >= 1 && c <= nz - 3))) {
            const f2 lamh_c = ST ? bc(Df * pv(c, 0)) : lam;  // Delta / (spacing of interface c, c+1)
            Dn = scale2(tvd_G2(ss2, ss1, dd1, mul2(lamh_c, max2(A2, A1)), C.tvd_form), d1);
        }

        // output row c = j-2
        if (store) {
            S2 Xn;
            if (!edge || (c >= 1 && c <= nz - 2)) {
                if constexpr (ST) {
                    const f2 hl = bc(0.5f * Df * pv(c, 1)), rp = bc(pv(c, 2));
                    Xn.r = fma2(rp, Dn.r, fnma2(hl, FP1.r, H.r));
                    Xn.mx = fma2(rp, Dn.mx, fnma2(hl, FP1.mx, H.mx));
                    Xn.mz = fma2(rp, Dn.mz, fnma2(hl, FP1.mz, H.mz));
                    Xn.E = fma2(rp, Dn.E, fnma2(hl, FP1.E, H.E));
                } else {
                    Xn.r = add2(fnma2(hlam, FP1.r, H.r), Dn.r);
                    Xn.mx = add2(fnma2(hlam, FP1.mx, H.mx), Dn.mx);
                    Xn.mz = add2(fnma2(hlam, FP1.mz, H.mz), Dn.mz);
                    Xn.E = add2(fnma2(hlam, FP1.E, H.E), Dn.E);
                }
            } else {
                // plates: rho = (rho^P + rho^C)/2 with the half-cell corrector
                Xn.r = (c == 0) ? fnma2(hlam_bot, FP1.r, H.r) : H.r;
                Xn.mx = z0; Xn.mz = z0;
                Xn.E = mul2(Xn.r, bc(c == 0 ? C.ebot : C.etop));
            }
            if (own) st2(gout, fs, 0, Xn);
        }
        gout += pitch;

        // H of row m for the next step
        if (ramp != 0) {
        } else if (interior_m) {
            if constexpr (ST) {
                const f2 rm = bc(pv(m, 3));
                H.r = fnma2(rm, Dn.r, mul2(half, fma2(lam_m, FP1.r, add2(XP1.r, Xm1.r))));
                H.mx = fnma2(rm, Dn.mx, mul2(half, fma2(lam_m, FP1.mx, add2(XP1.mx, Xm1.mx))));
                H.mz = fnma2(rm, Dn.mz, mul2(half, fma2(lam_m, FP1.mz, fma2(mDg, XP1.r, add2(XP1.mz, Xm1.mz)))));
                H.E = fnma2(rm, Dn.E, mul2(half, fma2(lam_m, FP1.E, add2(XP1.E, Xm1.E))));
            } else {
                H.r = sub2(mul2(half, fma2(lam, FP1.r, add2(XP1.r, Xm1.r))), Dn.r);
                H.mx = sub2(mul2(half, fma2(lam, FP1.mx, add2(XP1.mx, Xm1.mx))), Dn.mx);
                H.mz = sub2(mul2(half, fma2(lam, FP1.mz, fma2(mDg, XP1.r, add2(XP1.mz, Xm1.mz)))), Dn.mz);
                H.E = sub2(mul2(half, fma2(lam, FP1.E, add2(XP1.E, Xm1.E))), Dn.E);
            }
        } else {
            H.r = mul2(half, add2(XP1.r, Xm1.r));
            H.mx = z0; H.mz = z0; H.E = z0;
        }

        Xm1 = X0;
        ux1 = ux0; uz1 = uz0; T1 = T0; p1 = p0;
        gz1 = gz0;
        A2 = A1; A1 = A0;
        F2 = F1;
        ppux2 = ppux1; ppuz2 = ppuz1; ppT2 = ppT1;
        d1 = d0; dd1 = dd0; ss2 = ss1;
    };

    // steps j0 .. ke+1: three that only fill the pipeline, then one output row
    // per step.  Segments clear of the plates and of the grid ends run a
    // specialised step without plate rules, clamping or range tests, two
    // steps per trip so the pipeline registers swap roles instead of being
    // copied.  (The specialisations round alike to within FP32 noise, not bit
    // for bit, so FP32 results may differ at that level between segment
    // lengths; for a fixed launch configuration they are reproducible.)
    const std::true_type yes;
    const std::false_type no;
    const std::integral_constant<int, 0> full;
    const std::integral_constant<int, 1> ramp1;
    const std::integral_constant<int, 2> ramp2;
    if (interior_segment(ks, ke, nz)) {
        row_step(j0, no, no, ramp1);      // j0 = ks - 1
        row_step(j0 + 1, no, no, ramp2);  // ks
        row_step(j0 + 2, no, no, full);   // ks + 1
        int j = ks + 2;
        for (; j + 1 <= ke + 1; j += 2) {
            row_step(j, no, yes, full);
            row_step(j + 1, no, yes, full);
        }
        if (j <= ke + 1) row_step(j, no, yes, full);
    } else {
        for (int j = j0; j <= ke + 1; ++j) {
            if (j >= ks + 2) row_step(j, yes, yes, full);
            else row_step(j, yes, no, full);
        }
    }
    cp_async_drain();  // rows requested past the segment end
}

__global__ void __launch_bounds__(kThreads2, 4)
sweep_z2d_x2(SweepIO2 io, const __grid_constant__ Coef<float> C, SweepCtl sc)
{
    pdl_enter();
    const int gw = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    z2_body(io.in, io.out, C, sc, gw % io.nstrips, (gw / io.nstrips) * io.seg_rows, io.seg_rows, blockIdx.x == 0);
}

// L_x(Delta) on the interior rows (plate rows pass through), FP32, two
// columns per lane.  Row pipeline at step j: for row m = j-1, F^n (forward
// x, central z from rows j and j-2), X^P, the TVD term along x and
// K_m = (X^P + X)_m/2 + D_{i+1/2} - D_{i-1/2}; then for row c = j-2, F^P
// (backward x, central z from X^P rows j-1 and j-3) and
// X_new_c = K_c - (lambda/2)(F^P_{i+1} - F^P_i).
// one warp's segment of the x sweep (see z2_body); every thread of the block
// must call it when it reduces the next dt: DT = 1 always, 0 never, -1 when
// sc.last is set (the reduction needs a block barrier).  ST:
// stretched z-grid: central z-differences over the distance of the two planes
// they use, CFL z step of a plane its smaller spacing.
template <bool ST = false, int DT = -1>
__device__ __forceinline__ void x2_body(const float* __restrict__ in, float* __restrict__ out, const Coef<float>& C,
                                        const SweepCtl& sc, int strip, int ks, int seg_rows, bool lead)
{
    const bool want_dt = DT < 0 ? sc.last != 0 : DT == 1;
    extern __shared__ f2 ring_mem[];
    SweepIO2 io;
    io.in = in;
    io.out = out;
    const int lane = threadIdx.x & 31;
    const int nz = C.nz, nx = C.nx, pitch = C.pitch;
    const int fs = (int)C.fstride;
    const int ke = min(ks + seg_rows, nz);
    const int i = strip * kOutW2 - 2 + 2 * lane;
    int ic = i % nx;
    if (ic < 0) ic += nx;
    const bool own = lane >= 1 && lane <= 30 && i < nx;

    const double dt = step_dt(sc.ctl, sc.slot_in, C.cfl, C.dt_fixed);
    const double Delta = sc.Delta > 0.0 ? sc.Delta : 0.5 * dt;
    const float lamf = (float)(Delta / C.dx);
    const f2 lam = bc(lamf), hlam = bc(0.5f * lamf);
    const f2 half = bc(0.5f);

    if (sc.first && lead && threadIdx.x == 0) {
        sc.ctl->dt_slot[sc.slot_in ^ 1] = 0x7FF0000000000000ULL;
        sc.ctl->t += dt;
        sc.ctl->steps += 1.0;
    }

    float rmax = 0.f;
    int bad = 0;
    if (ks < nz) {
        const RowRing ring{ring_mem + threadIdx.x};
        auto row_off = [&](int j) { return min(max(j, 0), nz - 1) * pitch + ic; };
        // stretched: this warp's plane cache {1/sc, z}
        float* pc = ST ? plane_cache2<2>(ring_mem, seg_rows) : nullptr;
        if constexpr (ST) {
            for (int e = lane; e < ke - ks + kPlaneBack2 + 2; e += 32) {
                const Plane<float>& P = C.zp[min(max(ks - kPlaneBack2 + e, 0), nz - 1)];
                pc[e * 2 + 0] = P.isc;
                pc[e * 2 + 1] = P.z;
            }
            __syncwarp();
        }
        auto pv = [&](int k, int q) { return pc[(k - (ks - kPlaneBack2)) * 2 + q]; };
        auto gz_of = [&](int j) {
            if constexpr (ST) return bc(-C.g * pv(j, 1));
            else return bc(-C.g * ((float)min(max(j, 0), nz - 1) * C.hz));
        };
        const f2 idx_ = bc(C.inv_dx), i2dz = bc(C.inv_2dz);
        const f2 z0 = bc(0.f);

        // the first step is j0 = ks - 1 (primed with row ks - 2), as in z2_body
        const int j0 = ks - 1;
        for (int q = 0; q < kRing - 1; ++q) ring.request(q, io.in + row_off(j0 + q), fs);

        S2 Xm1 = ld2(io.in, fs, row_off(j0 - 1));
        f2 gz1 = gz_of(j0 - 1);
        f2 ux1, uz1, T1, p1;
        prims2(Xm1, gz1, C, ux1, uz1, T1, p1);
        f2 ux2 = ux1, uz2 = uz1;
        S2 XP2 = Xm1, K2 = Xm1;
        f2 ppux2 = ux1, ppuz2 = uz1, ppT2 = T1, ppp2 = p1;
        f2 ppux3 = ux1, ppuz3 = uz1;
        f2 gz2 = gz1;  // -g z of row j-2
        const float* gnext = io.in + row_off(j0 + kRing - 1);
        float* gout = io.out + (long long)(j0 - 2) * pitch + i;  // used only when the row exists

        // ramp 1: the first step of an interior segment, which skips what no
        // stored row uses (F^n, X^P, the TVD term and K of row ks - 2)
        auto row_step = [&](const int j, auto edge_tag, auto store_tag, auto ramp_tag) {
            constexpr bool edge = decltype(edge_tag)::value;
            constexpr bool store = decltype(store_tag)::value;
            constexpr int ramp = decltype(ramp_tag)::value;
            const int t = j - j0;
            if (edge) {
                ring.request((t + kRing - 1) % kRing, io.in + row_off(j + kRing - 1), fs);
            } else {
                ring.request((t + kRing - 1) % kRing, gnext, fs);
                gnext += pitch;
            }
            cp_async_wait_ring();
            const S2 X0 = ring.take(t % kRing);
            f2 gz0;
            if constexpr (ST) gz0 = gz_of(j);
            else gz0 = edge ? gz_of(j) : bc(-C.g * ((float)j * C.hz));
            f2 ux0, uz0, T0, p0;
            prims2(X0, gz0, C, ux0, uz0, T0, p0);

            // row m = j-1
            const int m = j - 1;
            f2 i2dz_m = i2dz, i2dz_c = i2dz;  // 1/(central z span) of planes m and c = m - 1
            if constexpr (ST) {
                i2dz_m = bc(pv(m, 0));
                i2dz_c = bc(pv(m - 1, 0));
            }
            S2 XP1 = Xm1, K1 = Xm1;  // plate rows pass through
            if (ramp != 1 && (!edge || (m >= 1 && m <= nz - 2))) {
                const S2 F1 = flux_x2(Xm1, ux1, uz1, p1, mul2(sub2(right_of(ux1), ux1), idx_),
                                      mul2(sub2(right_of(uz1), uz1), idx_), mul2(sub2(right_of(T1), T1), idx_),
                                      mul2(sub2(ux0, ux2), i2dz_m), mul2(sub2(uz0, uz2), i2dz_m), C);
                const S2 Fl = left_of(F1);
                XP1.r = fnma2(lam, sub2(F1.r, Fl.r), Xm1.r);
                XP1.mx = fnma2(lam, sub2(F1.mx, Fl.mx), Xm1.mx);
                XP1.mz = fnma2(lam, sub2(F1.mz, Fl.mz), Xm1.mz);
                XP1.E = fnma2(lam, sub2(F1.E, Fl.E), Xm1.E);
            }
            if (ramp == 0 && (!edge || (m >= 1 && m <= nz - 2))) {
                // TVD along x on row m from the input state
                const S2 d0 = diff2(right_of(Xm1), Xm1);
                const f2 dd = dot2(d0, d0);
                const f2 sp = dot2(left_of(d0), d0);
                const f2 A = add2(abs2(ux1), sqrt2(mul2(bc(C.cs2), T1)));
                const f2 G = tvd_G2(sp, right_of(sp), dd, mul2(lam, max2(A, right_of(A))), C.tvd_form);
                const S2 Dn = scale2(G, d0);
                const S2 Dl = left_of(Dn);
                K1.r = fma2(half, add2(XP1.r, Xm1.r), sub2(Dn.r, Dl.r));
                K1.mx = fma2(half, add2(XP1.mx, Xm1.mx), sub2(Dn.mx, Dl.mx));
                K1.mz = fma2(half, add2(XP1.mz, Xm1.mz), sub2(Dn.mz, Dl.mz));
                K1.E = fma2(half, add2(XP1.E, Xm1.E), sub2(Dn.E, Dl.E));
            }
            f2 ppux1 = z0, ppuz1 = z0, ppT1 = z0, ppp1 = z0;
            if (ramp != 1) prims2(XP1, gz1, C, ppux1, ppuz1, ppT1, ppp1);

            // row c = j-2: F^P (backward x, central z) and the corrector
            if (store) {
                const int c = j - 2;
                S2 Xn = K2;
                if (!edge || (c >= 1 && c <= nz - 2)) {
                    const S2 FP = flux_x2(XP2, ppux2, ppuz2, ppp2, mul2(sub2(ppux2, left_of(ppux2)), idx_),
                                          mul2(sub2(ppuz2, left_of(ppuz2)), idx_), mul2(sub2(ppT2, left_of(ppT2)), idx_),
                                          mul2(sub2(ppux1, ppux3), i2dz_c), mul2(sub2(ppuz1, ppuz3), i2dz_c), C);
                    const S2 FPr = right_of(FP);
                    Xn.r = fnma2(hlam, sub2(FPr.r, FP.r), K2.r);
                    Xn.mx = fnma2(hlam, sub2(FPr.mx, FP.mx), K2.mx);
                    Xn.mz = fnma2(hlam, sub2(FPr.mz, FP.mz), K2.mz);
                    Xn.E = fnma2(hlam, sub2(FPr.E, FP.E), K2.E);
                }
                if (own) {
                    st2(gout, fs, 0, Xn);
                    if (want_dt) {
                        f2 ux, uz, T, p;
                        prims2(Xn, gz2, C, ux, uz, T, p);
                        const f2 cs = sqrt2(mul2(bc(C.cs2), T));
                        const f2 rx = mul2(add2(abs2(ux), cs), idx_);
                        const f2 rz = mul2(add2(abs2(uz), cs), bc(ST ? __ldg(&C.zp[c].ihmin) : C.inv_dz));
                        const float r = fmaxf(fmaxf(rx.x, rx.y), fmaxf(rz.x, rz.y));
                        if (!(r > 0.f) || !(r < 1e30f)) bad = 1;
                        rmax = fmaxf(rmax, r);
                    }
                }
            }
            gout += pitch;

            Xm1 = X0;
            ux2 = ux1; uz2 = uz1;
            ux1 = ux0; uz1 = uz0; T1 = T0; p1 = p0;
            gz2 = gz1; gz1 = gz0;
            ppux3 = ppux2; ppuz3 = ppuz2;
            XP2 = XP1; K2 = K1;
            ppux2 = ppux1; ppuz2 = ppuz1; ppT2 = ppT1; ppp2 = ppp1;
        };

        // steps j0 .. ke+1: three that only fill the pipeline, then one output row
        // per step.  Segments clear of the plates and of the grid ends run a
        // specialised step without plate rules, clamping or range tests, two
        // steps per trip so the pipeline registers swap roles instead of being
        // copied.  (The specialisations round alike to within FP32 noise, not bit
        // for bit, so FP32 results may differ at that level between segment
        // lengths; for a fixed launch configuration they are reproducible.)
        const std::true_type yes;
        const std::false_type no;
        const std::integral_constant<int, 0> full;
        const std::integral_constant<int, 1> ramp1;
        if (interior_segment(ks, ke, nz)) {
            row_step(j0, no, no, ramp1);      // j0 = ks - 1
            row_step(j0 + 1, no, no, full);   // ks
            row_step(j0 + 2, no, no, full);   // ks + 1
            int j = ks + 2;
            for (; j + 1 <= ke + 1; j += 2) {
                row_step(j, no, yes, full);
                row_step(j + 1, no, yes, full);
            }
            if (j <= ke + 1) row_step(j, no, yes, full);
        } else {
            for (int j = j0; j <= ke + 1; ++j) {
                if (j >= ks + 2) row_step(j, yes, yes, full);
                else row_step(j, yes, no, full);
            }
        }
        cp_async_drain();  // rows requested past the segment end
    }
    if (want_dt) block_dt_reduce(rmax > 0.f ? 1.0 / (double)rmax : 1e308, bad, sc.ctl, sc.slot_in ^ 1);
}

// the x sweep without (sc.last unset) and with (_dt) the next step's dt reduction
__global__ void __launch_bounds__(kThreads2, 4)
sweep_x2d_x2(SweepIO2 io, const __grid_constant__ Coef<float> C, SweepCtl sc)
{
    pdl_enter();
    const int gw = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    x2_body<false, 0>(io.in, io.out, C, sc, gw % io.nstrips, (gw / io.nstrips) * io.seg_rows, io.seg_rows,
                      blockIdx.x == 0);
}

__global__ void __launch_bounds__(kThreads2, 4)
sweep_x2d_x2_dt(SweepIO2 io, const __grid_constant__ Coef<float> C, SweepCtl sc)
{
    pdl_enter();
    const int gw = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    x2_body<false, 1>(io.in, io.out, C, sc, gw % io.nstrips, (gw / io.nstrips) * io.seg_rows, io.seg_rows,
                      blockIdx.x == 0);
}

// the same two sweeps on a stretched z-grid (C.zp set)
__global__ void __launch_bounds__(kThreads2, 4)
sweep_z2d_x2s(SweepIO2 io, const __grid_constant__ Coef<float> C, SweepCtl sc)
{
    pdl_enter();
    const int gw = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    z2_body<true>(io.in, io.out, C, sc, gw % io.nstrips, (gw / io.nstrips) * io.seg_rows, io.seg_rows, blockIdx.x == 0);
}

__global__ void __launch_bounds__(kThreads2, 4)
sweep_x2d_x2s(SweepIO2 io, const __grid_constant__ Coef<float> C, SweepCtl sc)
{
    pdl_enter();
    const int gw = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    x2_body<true, 0>(io.in, io.out, C, sc, gw % io.nstrips, (gw / io.nstrips) * io.seg_rows, io.seg_rows,
                     blockIdx.x == 0);
}

__global__ void __launch_bounds__(kThreads2, 4)
sweep_x2d_x2s_dt(SweepIO2 io, const __grid_constant__ Coef<float> C, SweepCtl sc)
{
    pdl_enter();
    const int gw = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    x2_body<true, 1>(io.in, io.out, C, sc, gw % io.nstrips, (gw / io.nstrips) * io.seg_rows, io.seg_rows,
                     blockIdx.x == 0);
}

// ---- batched ensemble: many independent boxes in one launch per sweep -----
// Each warp takes one work item (box, strip, first row of its segment); the
// four warps of a block always belong to the same box.  Boxes step in
// lockstep (same sweep, same dt slot parity) but each has its own dt, time
// and state buffers.  Batches of up to kConstBoxes boxes read each box's
// coefficients from constant memory with a block-uniform index (no per-thread
// registers for them); larger batches stage them in shared memory.
__constant__ Coef<float> c_box[kConstBoxes];

__device__ __forceinline__ const BatchWork& batch_item(const BatchLaunch& L, SweepCtl& sc, const float*& in,
                                                       float*& out, int& box)
{
    const BatchWork& w = L.work[blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5)];
    box = L.work[blockIdx.x * kWarpsPerBlock].box;
    const BoxDesc& B = L.boxes[box];
    sc.ctl = B.ctl;
    sc.slot_in = L.slot;
    sc.first = L.first;
    sc.last = L.last;
    sc.Delta = L.Delta;
    in = B.buf[L.cur];
    out = B.buf[L.cur ^ 1];
    return w;
}

// one batched sweep (Z: the z sweep, else x) with each box's coefficients in
// constant memory; ST: stretched z-grids (every box's C.zp set)
template <bool Z, bool ST>
__device__ __forceinline__ void batch_sweep_const(const BatchLaunch& L)
{
    SweepCtl sc;
    const float* in;
    float* out;
    int box;
    const BatchWork& w = batch_item(L, sc, in, out, box);
    box = __shfl_sync(0xffffffffu, box, 0);  // warp-uniform index into the constant bank
    if constexpr (Z) z2_body<ST>(in, out, c_box[box], sc, w.strip, w.ks, w.seg_rows, w.lead != 0);
    else x2_body<ST, -1>(in, out, c_box[box], sc, w.strip, w.ks, w.seg_rows, w.lead != 0);
}

// the same for batches of more than kConstBoxes boxes: the block stages its
// box's coefficients in shared memory (sC)
template <bool Z, bool ST>
__device__ __forceinline__ void batch_sweep_smem(const BatchLaunch& L, Coef<float>& sC)
{
    SweepCtl sc;
    const float* in;
    float* out;
    int box;
    const BatchWork& w = batch_item(L, sc, in, out, box);
    if (threadIdx.x == 0) sC = L.boxes[box].C;
    __syncthreads();
    if constexpr (Z) z2_body<ST>(in, out, sC, sc, w.strip, w.ks, w.seg_rows, w.lead != 0);
    else x2_body<ST, -1>(in, out, sC, sc, w.strip, w.ks, w.seg_rows, w.lead != 0);
}

__global__ void __launch_bounds__(kThreads2, 4) sweep_z2d_batch(const __grid_constant__ BatchLaunch L)
{
    batch_sweep_const<true, false>(L);
}

__global__ void __launch_bounds__(kThreads2, 4) sweep_x2d_batch(const __grid_constant__ BatchLaunch L)
{
    batch_sweep_const<false, false>(L);
}

__global__ void __launch_bounds__(kThreads2, 4) sweep_z2d_batch_smem(const __grid_constant__ BatchLaunch L)
{
    __shared__ Coef<float> sC;
    batch_sweep_smem<true, false>(L, sC);
}

__global__ void __launch_bounds__(kThreads2, 4) sweep_x2d_batch_smem(const __grid_constant__ BatchLaunch L)
{
    __shared__ Coef<float> sC;
    batch_sweep_smem<false, false>(L, sC);
}

// batches with stretched z-grids: each warp's plane cache follows the row
// ring in dynamic shared memory, sized for segments of up to kBatchSegMax rows
__global__ void __launch_bounds__(kThreads2, 4) sweep_z2d_batch_s(const __grid_constant__ BatchLaunch L)
{
    batch_sweep_const<true, true>(L);
}

__global__ void __launch_bounds__(kThreads2, 4) sweep_x2d_batch_s(const __grid_constant__ BatchLaunch L)
{
    batch_sweep_const<false, true>(L);
}

__global__ void __launch_bounds__(kThreads2, 4) sweep_z2d_batch_smem_s(const __grid_constant__ BatchLaunch L)
{
    __shared__ Coef<float> sC;
    batch_sweep_smem<true, true>(L, sC);
}

__global__ void __launch_bounds__(kThreads2, 4) sweep_x2d_batch_smem_s(const __grid_constant__ BatchLaunch L)
{
    __shared__ Coef<float> sC;
    batch_sweep_smem<false, true>(L, sC);
}

// shared memory of the row ring for a block
constexpr size_t kRingBytes = (size_t)kRing * 4 * kThreads2 * sizeof(f2);

}  // namespace cm
