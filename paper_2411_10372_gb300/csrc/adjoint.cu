// adjoint.cu -- reverse mode of the 2D FP64 MacCormack-TVD sweeps (Sec. 3.1)
// for gradients of the time-averaged plate Nusselt number (Eq. mean_Nu).
//
// One sweep Y = L_al(Delta) X is differentiated in stages, each a kernel with
// one thread per node.  First the sweep's intermediates are recomputed from X
// (primitives, F^n, X^P and its primitives).  The quantities that decide the
// limiter's and C(Co)'s branches (primitives, wave speeds, the differences of
// X and their dot products, the ratios and Co) are rounded exactly as in the
// forward kernels (explicit intrinsics); everything else may use multiply-add
// contraction.  Then the adjoint
// runs the stages backwards: TVD term, corrector and average, F^P, X^P,
// predictor, F^n, primitives.  Every stage whose forward reads neighbours is
// written as a gather: a node collects the contributions it made to its
// neighbours' outputs, so no atomics are used and the result is
// deterministic.  Non-smooth points take fixed one-sided derivatives:
// phi'(r) = 2 on 0 < 2r < 1 and 0 elsewhere, d|u|/du = 0 at u = 0, the
// Co(1 - Co) branch for Co <= 1/2, and on a tie of max(A_k, A_k+1) the first
// argument.  dt of each step is a constant (the recorded one).
//
// The limiter's ratio r = <dX_-, dX_+> / <dX_+, dX_+> of the vector TVD term
// is not Lipschitz in X: where dX_+ -> 0 with dX_- not parallel to it, the
// exact derivative of phi(r) dX_+ grows like |dX_-| / |dX_+|.  The tangent map
// of a long run then grows without bound although the run itself stays
// bounded.  AdjWork::frozen_phi = 1 drops the derivative through r (phi' = 0
// everywhere: the limiter's switch values held fixed, C(Co) still
// differentiated), which keeps the reverse pass bounded.
//
// Stretched z-grid (C.zp set): the spans and factors follow the forward
// sweeps' conservative form.  Along z, the flux differences of plane k scale
// with Delta / w_k (the plate half cells with Delta / w_0, Delta / w_K), the
// one-sided derivatives of a flux at plane j divide by h_j (F^n) or h_{j-1}
// (F^P), the TVD flux of interface (s, s+1) enters Y_s with weight rp_s and
// Y_{s+1} with rm_{s+1} and its Courant number divides by h_s; the x sweep's
// central z-differences at plane k divide by sc_k = h_{k-1} + h_k.
#include <cuda_runtime.h>

#include <cstring>

#include "adjoint.h"

namespace cm {
namespace {

constexpr int kAdjThreads = 256;

__device__ __forceinline__ int wrapx(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// node (i, k) <-> index k * pitch + i; neighbours along the sweep (AL = 2: z,
// AL = 0: x, periodic) and across it
template <int AL>
__device__ __forceinline__ long long nb_al(const Coef<double>& C, int i, int k, int s)
{
    return AL == 2 ? (long long)(k + s) * C.pitch + i : (long long)k * C.pitch + wrapx(i + s, C.nx);
}
template <int AL>
__device__ __forceinline__ long long nb_ac(const Coef<double>& C, int i, int k, int s)
{
    return AL == 2 ? (long long)k * C.pitch + wrapx(i + s, C.nx) : (long long)(k + s) * C.pitch + i;
}

// nodes that carry a flux: F^n (FWD) along z on planes 0..K-1, F^P along z on
// 1..K; along x the interior rows 1..K-1 only
template <int AL, bool FWD>
__device__ __forceinline__ bool has_flux(const Coef<double>& C, int k)
{
    const int K = C.nz - 1;
    if (AL == 2) return FWD ? (k >= 0 && k <= K - 1) : (k >= 1 && k <= K);
    return k >= 1 && k <= K - 1;
}

__device__ __forceinline__ bool interior_row(const Coef<double>& C, int k) { return k >= 1 && k <= C.nz - 2; }

struct Q4 {
    double v[4];
};

__device__ __forceinline__ Q4 ld4(const double* X, long long fs, long long n)
{
    return {{X[n], X[fs + n], X[2 * fs + n], X[3 * fs + n]}};
}

__device__ __forceinline__ void st4(double* X, long long fs, long long n, const Q4& q)
{
    X[n] = q.v[0];
    X[fs + n] = q.v[1];
    X[2 * fs + n] = q.v[2];
    X[3 * fs + n] = q.v[3];
}

// primitives in the forward kernels' operation order (Sec. 2 closures), each
// operation rounded on its own (explicit intrinsics: this unit contracts
// multiply-adds elsewhere), so that T and the wave speed that decide the
// limiter's branches equal the forward run's bit for bit
__device__ __forceinline__ void prims_of(const Q4& q, double z, const Coef<double>& C, double& ux, double& uz,
                                         double& T, double& p)
{
    ux = q.v[1] / q.v[0];
    uz = q.v[2] / q.v[0];
    const double ke = __dmul_rn(0.5, __dadd_rn(__dmul_rn(ux, ux), __dmul_rn(uz, uz)));
    T = __dmul_rn(C.b, __dsub_rn(__dsub_rn(q.v[3] / q.v[0], ke), __dmul_rn(C.g, z)));
    p = __dmul_rn(__dmul_rn(C.a, q.v[0]), T);
}

// grid-stride loop over the nodes; each iteration defines i, k and the index n = k * pitch + i
#define FOR_NODES(C)                                                                                    \
    for (long long t_ = blockIdx.x * (long long)blockDim.x + threadIdx.x; t_ < (long long)(C).nx * (C).nz; \
         t_ += (long long)gridDim.x * blockDim.x)
#define NODE(C)                                                                                         \
    const int k = (int)(t_ / (C).nx), i = (int)(t_ % (C).nx);                                          \
    const long long n = (long long)k * (C).pitch + i;                                                   \
    (void)i;                                                                                            \
    (void)n

template <int AL>
__global__ void k_prims(const double* __restrict__ X, const double* __restrict__ zt, Coef<double> C, AdjWork w)
{
    FOR_NODES(C)
    {
        NODE(C);
        double ux, uz, T, p;
        prims_of(ld4(X, w.fs, n), zt[k], C, ux, uz, T, p);
        w.U0[n] = ux;
        w.U1[n] = uz;
        w.T[n] = T;
        w.P[n] = p;
        w.A[n] = __dadd_rn(fabs(AL == 2 ? uz : ux), __dsqrt_rn(__dmul_rn(C.cs2, T)));
    }
}

// the derivatives a flux at node (i, k) uses: along the sweep one-sided
// (forward for F^n, backward for F^P), across central.  d[0..2] = along
// (u_al, u_across, T), d[3..4] = across (u_al, u_across).
template <int AL, bool FWD>
__device__ __forceinline__ void flux_derivs(const Coef<double>& C, const double* Ux, const double* Uz,
                                            const double* Tt, int i, int k, long long n, double (&d)[5])
{
    const double* Ua = AL == 2 ? Uz : Ux;
    const double* Uc = AL == 2 ? Ux : Uz;
    const double ha = AL == 2 ? C.hz : C.hx, h2c = AL == 2 ? C.h2x : C.h2z;
    const long long np = FWD ? nb_al<AL>(C, i, k, 1) : n, nm = FWD ? n : nb_al<AL>(C, i, k, -1);
    // no branch of the reverse pass depends on these, so reciprocal spans suffice
    double ia = 1.0 / ha, ic = 1.0 / h2c;
    if (C.zp) {
        if (AL == 2) ia = C.zp[FWD ? k : k - 1].ihp;  // spacing spanned by the one-sided difference
        else ic = C.zp[k].isc;                        // distance of planes k-1 and k+1
    }
    d[0] = (Ua[np] - Ua[nm]) * ia;
    d[1] = (Uc[np] - Uc[nm]) * ia;
    d[2] = (Tt[np] - Tt[nm]) * ia;
    const long long cp = nb_ac<AL>(C, i, k, 1), cm_ = nb_ac<AL>(C, i, k, -1);
    d[3] = (Ua[cp] - Ua[cm_]) * ic;
    d[4] = (Uc[cp] - Uc[cm_]) * ic;
}

// F_al of Sec. 3.1 in 2D, by components along (a) and across (c) the sweep:
//   [m_a ; m_a u_a - tau_a + p ; m_c u_a - tau_c ; u_a (E + p) - K dT_a - (u_x tau_x + u_z tau_z)]
//   tau_a = mu (2 d_a u_a + s div), tau_c = mu (d_a u_c + d_c u_a), div = d_a u_a + d_c u_c
template <int AL>
__device__ __forceinline__ Q4 flux_of(const Q4& q, double ux, double uz, double p, const double (&d)[5],
                                      const Coef<double>& C)
{
    constexpr int fa = AL == 2 ? 2 : 1, fc = AL == 2 ? 1 : 2;
    const double ua = AL == 2 ? uz : ux;
    const double div = d[0] + d[4];
    const double ta = C.mu * ((d[0] + d[0]) + C.stokes * div);
    const double tc = C.mu * (d[1] + d[3]);
    const double tx = AL == 2 ? tc : ta, tz = AL == 2 ? ta : tc;
    Q4 F;
    F.v[0] = q.v[fa];
    F.v[fa] = (q.v[fa] * ua - ta) + p;
    F.v[fc] = q.v[fc] * ua - tc;
    F.v[3] = (ua * (q.v[3] + p) - C.kth * d[2]) - (ux * tx + uz * tz);
    return F;
}

template <int AL, bool FWD>
__global__ void k_flux(const double* __restrict__ Xq, const double* Ux, const double* Uz, const double* Tt,
                       const double* Pp, double* Fout, Coef<double> C, long long fs)
{
    FOR_NODES(C)
    {
        NODE(C);
        if (!has_flux<AL, FWD>(C, k)) continue;
        double d[5];
        flux_derivs<AL, FWD>(C, Ux, Uz, Tt, i, k, n, d);
        st4(Fout, fs, n, flux_of<AL>(ld4(Xq, fs, n), Ux[n], Uz[n], Pp[n], d, C));
    }
}

// X^P (predictor, plate half cells for L_z, plate rows unchanged for L_x) and its primitives
template <int AL>
__global__ void k_pred(const double* __restrict__ X, const double* __restrict__ zt, Coef<double> C, AdjWork w,
                       double Delta)
{
    const double lam = Delta / (AL == 2 ? C.dz : C.dx);
    FOR_NODES(C)
    {
        NODE(C);
        const Q4 x = ld4(X, w.fs, n);
        Q4 xp = x;
        if (interior_row(C, k)) {
            const double lk = (AL == 2 && C.zp) ? Delta / C.zp[k].w : lam;
            const Q4 f0 = ld4(w.F, w.fs, n), f1 = ld4(w.F, w.fs, nb_al<AL>(C, i, k, -1));
            for (int c = 0; c < 4; ++c) xp.v[c] = x.v[c] - lk * (f0.v[c] - f1.v[c]);
            if (AL == 2) xp.v[2] = xp.v[2] + Delta * (-C.g * x.v[0]);
        } else if (AL == 2) {
            const double lpl = C.zp ? Delta / C.zp[k].w : 2.0 * lam;  // plate half cell
            xp.v[0] = (k == 0) ? x.v[0] - lpl * w.F[n] : x.v[0] + lpl * w.F[nb_al<AL>(C, i, k, -1)];
            xp.v[1] = xp.v[2] = 0.0;
            xp.v[3] = xp.v[0] * (k == 0 ? C.ebot : C.etop);
        }
        st4(w.XP, w.fs, n, xp);
        double ux, uz, T, p;
        prims_of(xp, zt[k], C, ux, uz, T, p);
        w.UP0[n] = ux;
        w.UP1[n] = uz;
        w.TP[n] = T;
        w.PP[n] = p;
    }
}

// ---- reverse stages -------------------------------------------------------

// dot product in the forward kernels' order, every operation rounded on its own
__device__ __forceinline__ double dot4q(const Q4& a, const Q4& b)
{
    return __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(a.v[0], b.v[0]), __dmul_rn(a.v[1], b.v[1])),
                               __dmul_rn(a.v[2], b.v[2])),
                     __dmul_rn(a.v[3], b.v[3]));
}

__device__ __forceinline__ double phi_r(double r) { return fmax(0.0, fmin(2.0 * r, 1.0)); }
__device__ __forceinline__ double dphi_r(double r) { return (2.0 * r > 0.0 && 2.0 * r < 1.0) ? 2.0 : 0.0; }

// reverse of the TVD flux D = G dX_{s+1/2} of one interface (nodes x[0..3] =
// s-1, s, s+1, s+2 along the sweep, wave speeds A0 at s, A1 at s+1) for the
// adjoint Db of D: contributions cx[role] to the adjoints of the four nodes
// and ca[0], ca[1] to those of A0, A1
struct TvdAdj {
    Q4 cx[4];
    double ca[2];
};

__device__ TvdAdj tvd_iface_adj(const Q4 (&x)[4], double A0, double A1, const Q4& Db, double Delta, double h,
                                int form, int frozen_phi)
{
    TvdAdj r;
    for (int q = 0; q < 4; ++q)
        for (int c = 0; c < 4; ++c) r.cx[q].v[c] = 0.0;
    r.ca[0] = r.ca[1] = 0.0;
    Q4 dm, d0, dp;
    for (int c = 0; c < 4; ++c) {
        dm.v[c] = x[1].v[c] - x[0].v[c];
        d0.v[c] = x[2].v[c] - x[1].v[c];
        dp.v[c] = x[3].v[c] - x[2].v[c];
    }
    const double sp = dot4q(dm, d0), sm = dot4q(d0, dp), dd = dot4q(d0, d0);
    if (form == 2 || dd == 0.0) return r;
    const double rp = sp / dd, rm = sm / dd;
    const double Co = __dmul_rn(Delta, fmax(A0, A1)) / h;
    const double Cc = Co <= 0.5 ? Co * (1.0 - Co) : 0.25;
    const double dC = Co <= 0.5 ? 1.0 - 2.0 * Co : 0.0;
    const double Gb = dot4q(Db, d0);
    double G, Cb, rpb, rmb;
    if (form == 0) {
        const double pp = phi_r(rp), pm = phi_r(rm);
        G = 0.5 * Cc * (1.0 - pp) + 0.5 * Cc * (1.0 - pm);
        Cb = Gb * 0.5 * ((1.0 - pp) + (1.0 - pm));
        rpb = -Gb * 0.5 * Cc * dphi_r(rp);
        rmb = -Gb * 0.5 * Cc * dphi_r(rm);
    } else {
        const double rs = rp + rm;
        G = 0.5 * Cc * (1.0 - phi_r(rs));
        Cb = Gb * 0.5 * (1.0 - phi_r(rs));
        rpb = rmb = -Gb * 0.5 * Cc * dphi_r(rs);
    }
    if (frozen_phi) rpb = rmb = 0.0;
    const double spb = rpb / dd, smb = rmb / dd, ddb = -(rpb * rp + rmb * rm) / dd;
    for (int c = 0; c < 4; ++c) {
        const double dmb = spb * d0.v[c];
        const double dpb = smb * d0.v[c];
        const double d0b = G * Db.v[c] + spb * dm.v[c] + smb * dp.v[c] + 2.0 * ddb * d0.v[c];
        r.cx[0].v[c] = -dmb;
        r.cx[1].v[c] = dmb - d0b;
        r.cx[2].v[c] = d0b - dpb;
        r.cx[3].v[c] = dpb;
    }
    const double Ab = Cb * dC * Delta / h;
    if (A0 >= A1) r.ca[0] = Ab;
    else r.ca[1] = Ab;
    return r;
}

// stage 1 of the reverse: the TVD terms, in two kernels.  r_tvd_iface: each
// interface s+1/2 (stored at node s) takes the reverse of its flux once and
// stores the adjoints of its three differences dX_{s-1/2}, dX_{s+1/2},
// dX_{s+3/2} (DVm, DV0, DVp) and of the wave speeds A_s, A_s+1 (DVA); zero where
// there is no TVD flux.  r_tvd_gather: node m sums what the four interfaces
// s = m+1, m, m-1, m-2 give it (X_m enters dX_{s-1/2} with -1 for s = m+1,
// +1 for s = m; dX_{s+1/2} with -1 for s = m, +1 for s = m-1; dX_{s+3/2} with
// -1 for s = m-1, +1 for s = m-2).  D_{s+1/2} enters Y_s with + and Y_{s+1}
// with -.
template <int AL>
__global__ void __launch_bounds__(kAdjThreads) r_tvd_iface(const double* __restrict__ X,
                                                           const double* __restrict__ Ybar, Coef<double> C,
                                                           AdjWork w, double Delta)
{
    const double h = AL == 2 ? C.hz : C.hx;
    const int K = C.nz - 1;
    FOR_NODES(C)
    {
        NODE(C);
        TvdAdj t;
        for (int q = 0; q < 4; ++q)
            for (int c = 0; c < 4; ++c) t.cx[q].v[c] = 0.0;
        t.ca[0] = t.ca[1] = 0.0;
        const bool on = C.tvd_form != 2 && (AL == 2 ? (k >= 1 && k <= K - 2) : interior_row(C, k));
        if (on) {
            Q4 xs[4];
            for (int q = 0; q < 4; ++q) xs[q] = ld4(X, w.fs, nb_al<AL>(C, i, k, q - 1));
            const long long s1 = nb_al<AL>(C, i, k, 1);
            const Q4 y0 = ld4(Ybar, w.fs, n), y1 = ld4(Ybar, w.fs, s1);
            Q4 Db;
            if (AL == 2 && C.zp) {
                const double wp = C.zp[k].rp, wm = C.zp[k + 1].rm;
                for (int c = 0; c < 4; ++c) Db.v[c] = wp * y0.v[c] - wm * y1.v[c];
                t = tvd_iface_adj(xs, w.A[n], w.A[s1], Db, Delta, C.zp[k].hp, C.tvd_form, w.frozen_phi);
            } else {
                for (int c = 0; c < 4; ++c) Db.v[c] = y0.v[c] - y1.v[c];
                t = tvd_iface_adj(xs, w.A[n], w.A[s1], Db, Delta, h, C.tvd_form, w.frozen_phi);
            }
        }
        // cx[0] = -dm_b, cx[3] = dp_b, cx[1] = dm_b - d0_b  ->  d0_b = -cx[0] - cx[1]
        Q4 tm, t0, tp;
        for (int c = 0; c < 4; ++c) {
            tm.v[c] = -t.cx[0].v[c];
            t0.v[c] = -t.cx[0].v[c] - t.cx[1].v[c];
            tp.v[c] = t.cx[3].v[c];
        }
        st4(w.DVm, w.fs, n, tm);
        st4(w.DV0, w.fs, n, t0);
        st4(w.DVp, w.fs, n, tp);
        w.DVA[n] = t.ca[0];
        w.DVA[w.fs + n] = t.ca[1];
    }
}

template <int AL>
__global__ void __launch_bounds__(kAdjThreads) r_tvd_gather(double* __restrict__ Xbar, Coef<double> C, AdjWork w)
{
    const int K = C.nz - 1;
    FOR_NODES(C)
    {
        NODE(C);
        Q4 acc = {{0.0, 0.0, 0.0, 0.0}};
        double ab = 0.0;
        // interface at node m + d along the sweep exists (in the arrays) for these d
        auto ok = [&](int d) { return AL == 0 || (k + d >= 0 && k + d <= K); };
        if (ok(1)) {
            const Q4 a = ld4(w.DVm, w.fs, nb_al<AL>(C, i, k, 1));
            for (int c = 0; c < 4; ++c) acc.v[c] -= a.v[c];
        }
        {
            const Q4 a = ld4(w.DVm, w.fs, n), b = ld4(w.DV0, w.fs, n);
            for (int c = 0; c < 4; ++c) acc.v[c] += a.v[c] - b.v[c];
            ab += w.DVA[n];
        }
        if (ok(-1)) {
            const long long nm = nb_al<AL>(C, i, k, -1);
            const Q4 a = ld4(w.DV0, w.fs, nm), b = ld4(w.DVp, w.fs, nm);
            for (int c = 0; c < 4; ++c) acc.v[c] += a.v[c] - b.v[c];
            ab += w.DVA[w.fs + nm];
        }
        if (ok(-2)) {
            const Q4 a = ld4(w.DVp, w.fs, nb_al<AL>(C, i, k, -2));
            for (int c = 0; c < 4; ++c) acc.v[c] += a.v[c];
        }
        st4(Xbar, w.fs, n, acc);
        w.AB[n] = ab;
    }
}

// adjoint of the average (X^P + X^C)/2 at a node, the plate values folded in
// (L_z plates: Y = (rho, 0, 0, rho e_w)); zero on plate rows of L_x
template <int AL>
__device__ __forceinline__ Q4 y1bar_of(const Coef<double>& C, const double* Ybar, long long fs, int k, long long n)
{
    const Q4 y = ld4(Ybar, fs, n);
    if (interior_row(C, k)) return y;
    Q4 z = {{0.0, 0.0, 0.0, 0.0}};
    if (AL == 2) z.v[0] = y.v[0] + y.v[3] * (k == 0 ? C.ebot : C.etop);
    return z;
}

// stage 2: corrector and average.  X^C = X - lam (F^P_{n+1} - F^P_n) + Delta S(X^P)
// on interior nodes; plate densities of L_z: (X^P + X - 2 lam F^P_1)/2 at the
// bottom, (X^P + X)/2 at the top; plate rows of L_x pass X through.
template <int AL>
__global__ void r_corr(const double* __restrict__ Ybar, double* __restrict__ Xbar, Coef<double> C, AdjWork w,
                       double Delta)
{
    const double lam = Delta / (AL == 2 ? C.dz : C.dx);
    FOR_NODES(C)
    {
        NODE(C);
        const Q4 y1 = y1bar_of<AL>(C, Ybar, w.fs, k, n);
        Q4 xb = ld4(Xbar, w.fs, n);
        Q4 xpb = {{0.0, 0.0, 0.0, 0.0}};
        if (interior_row(C, k)) {
            for (int c = 0; c < 4; ++c) {
                xb.v[c] += 0.5 * y1.v[c];
                xpb.v[c] = 0.5 * y1.v[c];
            }
            if (AL == 2) xpb.v[0] += Delta * (-C.g) * (0.5 * y1.v[2]);
        } else if (AL == 2) {
            xb.v[0] += 0.5 * y1.v[0];
            xpb.v[0] = 0.5 * y1.v[0];
        } else {
            const Q4 y = ld4(Ybar, w.fs, n);
            for (int c = 0; c < 4; ++c) xb.v[c] += y.v[c];
        }
        st4(Xbar, w.fs, n, xb);
        st4(w.XPB, w.fs, n, xpb);
        if (has_flux<AL, false>(C, k)) {
            const int km = AL == 2 ? k - 1 : k;
            // Delta / w of planes k and k-1, half of the bottom plate's (stretched L_z)
            double lk = lam, lkm = lam, lhb = lam;
            if (AL == 2 && C.zp) {
                lk = Delta / C.zp[k].w;
                lkm = Delta / C.zp[km].w;
                lhb = 0.5 * (Delta / C.zp[0].w);
            }
            Q4 fpb = {{0.0, 0.0, 0.0, 0.0}};
            if (interior_row(C, k))
                for (int c = 0; c < 4; ++c) fpb.v[c] += lk * (0.5 * y1.v[c]);
            const long long nm = nb_al<AL>(C, i, k, -1);
            if (interior_row(C, km)) {
                const Q4 y1m = y1bar_of<AL>(C, Ybar, w.fs, km, nm);
                for (int c = 0; c < 4; ++c) fpb.v[c] -= lkm * (0.5 * y1m.v[c]);
            }
            if (AL == 2 && k == 1) fpb.v[0] += -lhb * y1bar_of<AL>(C, Ybar, w.fs, 0, nm).v[0];
            st4(w.FPB, w.fs, n, fpb);
        }
    }
}

// deterministic block sum of two values into part[2 * blockIdx.x + {0, 1}]
__device__ __forceinline__ void block_sum2(double a, double b, double* part)
{
    __shared__ double sh[2][kAdjThreads / 32];
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int wi = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sh[0][wi] = a;
        sh[1][wi] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0.0, y = 0.0;
        for (int q = 0; q < kAdjThreads / 32; ++q) {
            x += sh[0][q];
            y += sh[1][q];
        }
        part[2 * blockIdx.x] = x;
        part[2 * blockIdx.x + 1] = y;
    }
}

// stages 3 and 6: reverse of the flux at each node that carries one (F^P on
// X^P, or F^n on X), given its adjoint Fbar.  Adds the terms in q to Qbar and
// writes the node's direct adjoints of (u_x, u_z, T) to UB, those of the
// derivatives it used to DA (along) and DC (across), and the block sums of
// <Fbar, dF/dmu> and <Fbar, dF/dK>.
template <int AL, bool FWD>
__global__ void __launch_bounds__(kAdjThreads) r_flux(const double* __restrict__ Q, const double* Ux,
                                                      const double* Uz, const double* Tt, const double* Pp,
                                                      const double* __restrict__ Fbar, double* Qbar, Coef<double> C,
                                                      AdjWork w, double* part)
{
    constexpr int fa = AL == 2 ? 2 : 1, fc = AL == 2 ? 1 : 2;
    const long long fs = w.fs;
    double smu = 0.0, skt = 0.0;
    FOR_NODES(C)
    {
        NODE(C);
        double ub[3] = {0.0, 0.0, 0.0}, da[3] = {0.0, 0.0, 0.0}, dc[2] = {0.0, 0.0};
        if (has_flux<AL, FWD>(C, k)) {
            double d[5];
            flux_derivs<AL, FWD>(C, Ux, Uz, Tt, i, k, n, d);
            const Q4 q = ld4(Q, fs, n), fb = ld4(Fbar, fs, n);
            const double ux = Ux[n], uz = Uz[n], p = Pp[n], T = Tt[n];
            const double ua = AL == 2 ? uz : ux, uc = AL == 2 ? ux : uz;
            const double div = d[0] + d[4];
            const double xa = (d[0] + d[0]) + C.stokes * div, xc = d[1] + d[3];
            const double ta = C.mu * xa, tc = C.mu * xc;
            const double Fr = fb.v[0], Fa = fb.v[fa], Fc = fb.v[fc], FE = fb.v[3];
            Q4 qb = ld4(Qbar, fs, n);
            qb.v[fa] += Fr + Fa * ua;
            qb.v[fc] += Fc * ua;
            qb.v[3] += FE * ua;
            const double pb = Fa + FE * ua;
            const double uab = Fa * q.v[fa] + Fc * q.v[fc] + FE * (q.v[3] + p) - FE * ta;
            const double ucb = -FE * tc;
            const double tab = -Fa - FE * ua, tcb = -Fc - FE * uc;
            da[2] = -FE * C.kth;
            skt += -FE * d[2];
            smu += tab * xa + tcb * xc;
            da[0] = C.mu * tab * (2.0 + C.stokes);
            dc[1] = C.mu * tab * C.stokes;
            da[1] = C.mu * tcb;
            dc[0] = C.mu * tcb;
            qb.v[0] += pb * C.a * T;  // p = a rho T
            ub[0] = AL == 2 ? ucb : uab;
            ub[1] = AL == 2 ? uab : ucb;
            ub[2] = pb * C.a * q.v[0];
            st4(Qbar, fs, n, qb);
        }
        w.UB[n] = ub[0];
        w.UB[fs + n] = ub[1];
        w.UB[2 * fs + n] = ub[2];
        w.DA[n] = da[0];
        w.DA[fs + n] = da[1];
        w.DA[2 * fs + n] = da[2];
        w.DC[n] = dc[0];
        w.DC[fs + n] = dc[1];
    }
    block_sum2(smu, skt, part);
}

// stages 4 and 7: each node gathers the derivative adjoints of the fluxes
// that read its u and T (one-sided along the sweep: forward for F^n, backward
// for F^P; central across), adds the wave-speed adjoint (F^n stage only), and
// takes the reverse of its primitives into Qbar.  With fold (X^P of L_z), the
// plate nodes' X^P = (rho, 0, 0, rho e_w) is folded into rho.
template <int AL, bool FWD>
__global__ void __launch_bounds__(kAdjThreads) r_gather(const double* __restrict__ Q, double* Qbar,
                                                        const double* Ux, const double* Uz, const double* Tt,
                                                        Coef<double> C, AdjWork w, int with_A, int fold)
{
    const long long fs = w.fs;
    const double ia = 1.0 / (AL == 2 ? C.hz : C.hx), ic = 1.0 / (AL == 2 ? C.h2x : C.h2z);
    const int K = C.nz - 1;
    FOR_NODES(C)
    {
        NODE(C);
        double uab = AL == 2 ? w.UB[fs + n] : w.UB[n];
        double ucb = AL == 2 ? w.UB[n] : w.UB[fs + n];
        double Tb = w.UB[2 * fs + n];
        // along: the flux at j uses (f[j+1] - f[j]) / h (FWD) or (f[j] - f[j-1]) / h (BWD)
        const double sgn = FWD ? -1.0 : 1.0;
        // 1 / span of the along-sweep difference of the flux at plane j (stretched L_z:
        // h_j for F^n, h_{j-1} for F^P); of the across difference (stretched L_x: sc_j)
        auto ia_of = [&](int j) { return (AL == 2 && C.zp) ? C.zp[FWD ? j : j - 1].ihp : ia; };
        auto ic_of = [&](int j) { return (AL == 0 && C.zp) ? C.zp[j].isc : ic; };
        if (has_flux<AL, FWD>(C, k)) {
            const double a = ia_of(k);
            uab += sgn * w.DA[n] * a;
            ucb += sgn * w.DA[fs + n] * a;
            Tb += sgn * w.DA[2 * fs + n] * a;
        }
        const int kj = AL == 2 ? (FWD ? k - 1 : k + 1) : k;
        if (kj >= 0 && kj <= K && has_flux<AL, FWD>(C, kj)) {
            const long long nj = nb_al<AL>(C, i, k, FWD ? -1 : 1);
            const double a = ia_of(kj);
            uab -= sgn * w.DA[nj] * a;
            ucb -= sgn * w.DA[fs + nj] * a;
            Tb -= sgn * w.DA[2 * fs + nj] * a;
        }
        // across: the flux at j uses (f[j+c] - f[j-c]) / 2h (stretched L_x: / sc_j)
        const int kl = AL == 2 ? k : k - 1, ku = AL == 2 ? k : k + 1;
        if (kl >= 0 && has_flux<AL, FWD>(C, kl)) {
            const long long nj = nb_ac<AL>(C, i, k, -1);
            const double a = ic_of(kl);
            uab += w.DC[nj] * a;
            ucb += w.DC[fs + nj] * a;
        }
        if (ku <= K && has_flux<AL, FWD>(C, ku)) {
            const long long nj = nb_ac<AL>(C, i, k, 1);
            const double a = ic_of(ku);
            uab -= w.DC[nj] * a;
            ucb -= w.DC[fs + nj] * a;
        }
        const double ux = Ux[n], uz = Uz[n];
        if (with_A) {
            const double ab = w.AB[n], ua = AL == 2 ? uz : ux;
            uab += ab * (ua > 0.0 ? 1.0 : (ua < 0.0 ? -1.0 : 0.0));
            Tb += ab * C.cs2 / (2.0 * sqrt(C.cs2 * Tt[n]));
        }
        // u = m / rho, T = b (E / rho - |u|^2 / 2 - g z)
        const Q4 q = ld4(Q, fs, n);
        Q4 qb = ld4(Qbar, fs, n);
        double uxb = AL == 2 ? ucb : uab, uzb = AL == 2 ? uab : ucb;
        const double ri = 1.0 / q.v[0];
        qb.v[3] += Tb * C.b * ri;
        qb.v[0] -= Tb * C.b * (q.v[3] * ri) * ri;
        uxb -= Tb * C.b * ux;
        uzb -= Tb * C.b * uz;
        qb.v[1] += uxb * ri;
        qb.v[2] += uzb * ri;
        qb.v[0] -= (uxb * ux + uzb * uz) * ri;
        if (fold && (k == 0 || k == K)) {
            qb.v[0] += qb.v[3] * (k == 0 ? C.ebot : C.etop);
            qb.v[1] = qb.v[2] = qb.v[3] = 0.0;
        }
        st4(Qbar, fs, n, qb);
    }
}

// stage 5: predictor.  X^P = X - lam (F_n - F_{n-1}) + Delta S(X) on interior
// nodes; L_z plate densities X - 2 lam F_0 and X + 2 lam F_{K-1}; L_x plate rows X.
// Adds dX^P/dX to Xbar and writes the adjoint FB of F^n.
template <int AL>
__global__ void r_pred(double* __restrict__ Xbar, Coef<double> C, AdjWork w, double Delta)
{
    const double lam = Delta / (AL == 2 ? C.dz : C.dx);
    const int K = C.nz - 1;
    const long long fs = w.fs;
    FOR_NODES(C)
    {
        NODE(C);
        const Q4 xpb = ld4(w.XPB, fs, n);
        Q4 xb = ld4(Xbar, fs, n);
        for (int c = 0; c < 4; ++c) xb.v[c] += xpb.v[c];
        if (AL == 2 && interior_row(C, k)) xb.v[0] += Delta * (-C.g) * xpb.v[2];
        st4(Xbar, fs, n, xb);
        if (has_flux<AL, true>(C, k)) {
            const int kp = AL == 2 ? k + 1 : k;
            // Delta / w of planes k and k+1 and of the plate half cells (stretched L_z)
            double lk = lam, lkp = lam, lbot = 2.0 * lam, ltop = 2.0 * lam;
            if (AL == 2 && C.zp) {
                lk = Delta / C.zp[k].w;
                lkp = Delta / C.zp[kp].w;
                lbot = Delta / C.zp[0].w;
                ltop = Delta / C.zp[K].w;
            }
            Q4 fb = {{0.0, 0.0, 0.0, 0.0}};
            if (interior_row(C, k))
                for (int c = 0; c < 4; ++c) fb.v[c] -= lk * xpb.v[c];
            const long long np = nb_al<AL>(C, i, k, 1);
            if (interior_row(C, kp)) {
                const Q4 xpbp = ld4(w.XPB, fs, np);
                for (int c = 0; c < 4; ++c) fb.v[c] += lkp * xpbp.v[c];
            }
            if (AL == 2 && k == 0) fb.v[0] += -lbot * xpb.v[0];
            if (AL == 2 && k == K - 1) fb.v[0] += ltop * w.XPB[np];
            st4(w.FB, fs, n, fb);
        }
    }
}

// acc[0..1] += the block partial sums of both flux stages, in a fixed order
__global__ void r_acc(const double* __restrict__ part, int nparts, double* acc)
{
    __shared__ double sh[2][kAdjThreads];
    double a = 0.0, b = 0.0;
    for (int q = threadIdx.x; q < nparts; q += blockDim.x) {
        a += part[2 * q];
        b += part[2 * q + 1];
    }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + st];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + st];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        acc[0] += sh[0][0];
        acc[1] += sh[1][0];
    }
}

// ---- objective: plane sums of T and their adjoint --------------------------

struct PlaneSet {
    int k[8];
    double w[8];
    int n;
};

__global__ void __launch_bounds__(kAdjThreads) k_plane_T(const double* __restrict__ X, const double* __restrict__ zt,
                                                         Coef<double> C, long long fs, PlaneSet P, double* out)
{
    __shared__ double sh[kAdjThreads];
    const int k = P.k[blockIdx.x];
    double acc = 0.0;
    for (int i = threadIdx.x; i < C.nx; i += blockDim.x) {
        double ux, uz, T, p;
        prims_of(ld4(X, fs, (long long)k * C.pitch + i), zt[k], C, ux, uz, T, p);
        acc += T;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

__global__ void k_seed_T(double* Xbar, const double* __restrict__ X, const double* __restrict__ zt, Coef<double> C,
                         long long fs, PlaneSet P)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)P.n * C.nx;
         t += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(t / C.nx), i = (int)(t % C.nx), k = P.k[q];
        const long long n = (long long)k * C.pitch + i;
        const Q4 x = ld4(X, fs, n);
        Q4 xb = ld4(Xbar, fs, n);
        const double Tb = P.w[q], ri = 1.0 / x.v[0];
        const double ux = x.v[1] * ri, uz = x.v[2] * ri;
        xb.v[3] += Tb * C.b * ri;
        xb.v[0] -= Tb * C.b * (x.v[3] * ri) * ri;
        const double uxb = -Tb * C.b * ux, uzb = -Tb * C.b * uz;
        xb.v[1] += uxb * ri;
        xb.v[2] += uzb * ri;
        xb.v[0] -= (uxb * ux + uzb * uz) * ri;
        st4(Xbar, fs, n, xb);
        (void)zt;
    }
}

__global__ void k_record_dt(const DevCtl* ctl, int slot, double cfl, double dt_fixed, double* out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) out[0] = step_dt(ctl, slot, cfl, dt_fixed);
}

// dJ/dT at fixed p and u: rho = p/(a T), m = rho u, E = rho (|u|^2/2 + T/b + g z)
// give d(rho, m, E)/dT = (-rho, -m, -E + rho T / b) / T
__global__ void k_grad_T(const double* __restrict__ X, const double* __restrict__ Xbar,
                         const double* __restrict__ zt, Coef<double> C, long long fs, double* gT)
{
    FOR_NODES(C)
    {
        NODE(C);
        double g = 0.0;
        if (interior_row(C, k)) {
            const Q4 x = ld4(X, fs, n), xb = ld4(Xbar, fs, n);
            double ux, uz, T, p;
            prims_of(x, zt[k], C, ux, uz, T, p);
            g = (-(xb.v[0] * x.v[0] + xb.v[1] * x.v[1] + xb.v[2] * x.v[2] + xb.v[3] * x.v[3]) +
                 xb.v[3] * x.v[0] * T / C.b) / T;
        }
        gT[(long long)k * C.nx + i] = g;
    }
}

}  // namespace

// ---- host side ---------------------------------------------------------------

// grid-stride launches of the reverse stages: at most 8 blocks per SM
static int adj_blocks(const Coef<double>& C)
{
    static int nsm = 0;
    if (!nsm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (nsm <= 0) nsm = 1;
    }
    const long long nodes = (long long)C.nx * C.nz;
    long long b = (nodes + kAdjThreads - 1) / kAdjThreads;
    if (b > 8LL * nsm) b = 8LL * nsm;
    return (int)(b < 1 ? 1 : b);
}

cudaError_t adj_work_create(AdjWork* w, const Coef<double>& C)
{
    std::memset(w, 0, sizeof *w);
    w->fs = C.fstride;
    w->nblocks = adj_blocks(C);
    // the arrays, in order, with their field counts
    double** arrays[] = {&w->U0, &w->U1, &w->T, &w->P, &w->A, &w->F, &w->XP, &w->UP0, &w->UP1, &w->TP,
                         &w->PP, &w->XPB, &w->FPB, &w->FB, &w->UB, &w->DA, &w->DC, &w->AB,
                         &w->DVm, &w->DV0, &w->DVp, &w->DVA};
    const int fields[] = {1, 1, 1, 1, 1, 4, 4, 1, 1, 1, 1, 4, 4, 4, 3, 3, 2, 1, 4, 4, 4, 2};
    static_assert(sizeof arrays / sizeof arrays[0] == sizeof fields / sizeof fields[0], "one count per array");
    size_t nfields = 0;
    for (int f : fields) nfields += (size_t)f;
    const size_t bytes = nfields * (size_t)w->fs * sizeof(double) + (size_t)4 * w->nblocks * sizeof(double);
    cudaError_t e = cudaMalloc(&w->base, bytes);
    if (e != cudaSuccess) return e;
    double* p = w->base;
    for (size_t q = 0; q < sizeof fields / sizeof fields[0]; ++q) {
        *arrays[q] = p;
        p += (size_t)fields[q] * w->fs;
    }
    w->part = p;  // 2 flux stages x nblocks x 2 sums
    return cudaMemset(w->base, 0, bytes);
}

void adj_work_free(AdjWork* w)
{
    if (w->base) cudaFree(w->base);
    w->base = nullptr;
}

template <int AL>
static cudaError_t vjp_dir(AdjWork* w, double Delta, const double* X, const double* Ybar, double* Xbar,
                           const double* zt, const Coef<double>& C, double* acc, cudaStream_t s)
{
    const int B = w->nblocks, T = kAdjThreads;
    const AdjWork W = *w;
    k_prims<AL><<<B, T, 0, s>>>(X, zt, C, W);
    k_flux<AL, true><<<B, T, 0, s>>>(X, W.U0, W.U1, W.T, W.P, W.F, C, W.fs);
    k_pred<AL><<<B, T, 0, s>>>(X, zt, C, W, Delta);
    r_tvd_iface<AL><<<B, T, 0, s>>>(X, Ybar, C, W, Delta);
    r_tvd_gather<AL><<<B, T, 0, s>>>(Xbar, C, W);
    r_corr<AL><<<B, T, 0, s>>>(Ybar, Xbar, C, W, Delta);
    r_flux<AL, false><<<B, T, 0, s>>>(W.XP, W.UP0, W.UP1, W.TP, W.PP, W.FPB, W.XPB, C, W, W.part);
    r_gather<AL, false><<<B, T, 0, s>>>(W.XP, W.XPB, W.UP0, W.UP1, W.TP, C, W, 0, AL == 2);
    r_pred<AL><<<B, T, 0, s>>>(Xbar, C, W, Delta);
    r_flux<AL, true><<<B, T, 0, s>>>(X, W.U0, W.U1, W.T, W.P, W.FB, Xbar, C, W, W.part + 2 * B);
    r_gather<AL, true><<<B, T, 0, s>>>(X, Xbar, W.U0, W.U1, W.T, C, W, 1, 0);
    r_acc<<<1, kAdjThreads, 0, s>>>(W.part, 2 * B, acc);
    return cudaGetLastError();
}

cudaError_t adj_sweep_vjp(AdjWork* w, int dir, double Delta, const double* X, const double* Ybar, double* Xbar,
                          const double* zt, const Coef<double>& C, double* acc, cudaStream_t s)
{
    if (dir == 2) return vjp_dir<2>(w, Delta, X, Ybar, Xbar, zt, C, acc, s);
    if (dir == 0) return vjp_dir<0>(w, Delta, X, Ybar, Xbar, zt, C, acc, s);
    return cudaErrorInvalidValue;
}

static PlaneSet plane_set(const int* kq, const double* wq, int nq)
{
    PlaneSet P;
    std::memset(&P, 0, sizeof P);
    P.n = nq < 8 ? nq : 8;
    for (int q = 0; q < P.n; ++q) {
        P.k[q] = kq[q];
        P.w[q] = wq ? wq[q] : 0.0;
    }
    return P;
}

cudaError_t adj_plane_T(const double* X, const double* zt, const Coef<double>& C, const int* kq, int nq, double* out,
                        cudaStream_t s)
{
    const PlaneSet P = plane_set(kq, nullptr, nq);
    k_plane_T<<<P.n, kAdjThreads, 0, s>>>(X, zt, C, C.fstride, P, out);
    return cudaGetLastError();
}

cudaError_t adj_seed_T(double* Xbar, const double* X, const double* zt, const Coef<double>& C, const int* kq,
                       const double* wq, int nq, cudaStream_t s)
{
    const PlaneSet P = plane_set(kq, wq, nq);
    const long long work = (long long)P.n * C.nx;
    const int blocks = (int)((work + kAdjThreads - 1) / kAdjThreads);
    k_seed_T<<<blocks, kAdjThreads, 0, s>>>(Xbar, X, zt, C, C.fstride, P);
    return cudaGetLastError();
}

cudaError_t adj_record_dt(const DevCtl* ctl, int slot, double cfl, double dt_fixed, double* out, cudaStream_t s)
{
    k_record_dt<<<1, 32, 0, s>>>(ctl, slot, cfl, dt_fixed, out);
    return cudaGetLastError();
}

cudaError_t adj_grad_T(const double* X, const double* Xbar, const double* zt, const Coef<double>& C, double* gT,
                       cudaStream_t s)
{
    k_grad_T<<<adj_blocks(C), kAdjThreads, 0, s>>>(X, Xbar, zt, C, C.fstride, gT);
    return cudaGetLastError();
}

}  // namespace cm
