// aux_kernels.cuh -- initial state, standalone dt reduction and the FP64
// diagnostics reduction (Sec. 2: Eqs. volume_Nu, mean_Nu, Re).
#pragma once
#include "cm_device.cuh"
#include "../../include/cm.h"

namespace cm {

// SplitMix64 (Steele, Lea & Flood 2014): output idx+1 of the generator seeded
// with `seed`, i.e. the finaliser applied to seed + (idx+1) * golden gamma.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed, unsigned long long idx)
{
    unsigned long long z = seed + (idx + 1ULL) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}


// Initial state: T = T_c(z) + A xi at interior nodes (plates unperturbed),
// rho = p_c(z)/(a T) (isobaric), u = 0, E = rho (T/b + g z).  FP64, then
// rounded to the state precision.  Grid: x-threads over (i, j), y-blocks over k.
template <class R>
__global__ void init_state(R* X, Coef<R> C, InitArgs A)
{
    const int k = blockIdx.y;
    const long long row = (long long)C.nx * C.ny;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < row; n += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(n % C.nx);
        const int j = (int)(n / C.nx);
        const unsigned long long dense = ((unsigned long long)k * C.ny + j) * C.nx + i;
        double T = A.Tc[k];
        if (k > 0 && k < C.nz - 1) {
            if (A.Tfield) {
                T = A.Tfield[dense];
            } else {
                const double u = (double)(splitmix64(A.seed, dense) >> 11) * 0x1.0p-53;
                T = A.Tc[k] + A.amp * (2.0 * u - 1.0);
            }
        }
        const double rho = A.pc[k] / (A.a * T);
        const double E = rho * (T / A.b + A.g * A.zt[k]);
        R* p = X + ((size_t)k * C.ny + j) * C.pitch + i;
        const long long fs = C.fstride;
        p[0] = (R)rho;
        p[fs] = R(0);
        p[2 * fs] = R(0);
        if (C.ndim == 3) {
            p[3 * fs] = R(0);
            p[4 * fs] = (R)E;
        } else {
            p[3 * fs] = (R)E;
        }
    }
}

// min over nodes and directions of h/(|u|+c) into a dt slot (used at init and
// after cm_set_state; during stepping the last sweep does this reduction).
// FP64 states: the sweeps' exact FP64 operation order.  FP32 states: the FP32
// rates (|u|+c)/h of the FP32 sweeps, one FP64 reciprocal of the block max.
// CFL bound of the nodes one thread visits (Sec. 3.1): FP32 keeps the largest
// rate max((|u_x| + c)/h_x, (|u_z| + c)/h_z), FP64 the smallest
// min(h/(|u| + c)) with the divisions of the sweeps' FP64 path; h_z of plane
// k is its smaller adjacent spacing on a stretched grid.
template <class R>
struct DtAcc {
    double vmin = 1e308;
    float rmax = 0.f;
    int bad = 0;
    // node values rho, m_x, (m_y,) m_z, E of plane k (3D: five values)
    __device__ __forceinline__ void add(const R* v, int k, const R* zt, const Coef<R>& C)
    {
        if constexpr (!kExact<R>) {
            const float rho = v[0], ri = 1.f / rho;
            const float ux = v[1] * ri;
            float uy = 0.f, uz, E;
            if (C.ndim == 3) { uy = v[2] * ri; uz = v[3] * ri; E = v[4]; }
            else { uz = v[2] * ri; E = v[3]; }
            const float T = C.b * (E * ri - 0.5f * ((ux * ux + uy * uy) + uz * uz) - C.g * zt[k]);
            const float c = sqrtf(C.cs2 * T);
            float r = fmaxf((fabsf(ux) + c) * C.inv_dx, (fabsf(uz) + c) * (C.zp ? C.zp[k].ihmin : C.inv_dz));
            if (C.ndim == 3) r = fmaxf(r, (fabsf(uy) + c) * C.inv_dy);
            if (!(r > 0.f) || !(r < 1e30f)) bad = 1;
            rmax = fmaxf(rmax, r);
        } else {
            // same operation order as the sweeps' FP64 path (divisions by rho)
            const double rho = (double)v[0];
            double ux = (double)v[1] / rho, uy = 0.0, uz, E;
            if (C.ndim == 3) { uy = (double)v[2] / rho; uz = (double)v[3] / rho; E = (double)v[4]; }
            else { uz = (double)v[2] / rho; E = (double)v[3]; }
            const double T = (double)C.b * (E / rho - 0.5 * ((ux * ux + uy * uy) + uz * uz) - (double)C.g * (double)zt[k]);
            const double c = sqrt((double)C.cs2 * T);
            double h = fmin(C.dx / (fabs(ux) + c), (C.zp ? (double)C.zp[k].hmin : C.dz) / (fabs(uz) + c));
            if (C.ndim == 3) h = fmin(h, C.dy / (fabs(uy) + c));
            if (!(h > 0.0) || !(h < 1e300)) bad = 1;
            vmin = fmin(vmin, h);
        }
    }
    // the block's contribution to the dt slot (smallest h/(|u| + c))
    __device__ __forceinline__ double result() const
    {
        if constexpr (!kExact<R>) return rmax > 0.f ? 1.0 / (double)rmax : 1e308;
        else return vmin;
    }
};

template <class R>
__global__ void dt_reduce(const R* X, const R* zt, Coef<R> C, DevCtl* ctl, int slot)
{
    DtAcc<R> acc;
    const long long plane = (long long)C.nx * C.ny;
    const long long total = plane * C.nz;
    const long long fs = C.fstride;
    const int nf = C.ndim == 3 ? 5 : 4;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < total; n += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(n % C.nx);
        const long long jk = n / C.nx;
        const int j = (int)(jk % C.ny);
        const int k = (int)(jk / C.ny);
        const R* p = X + ((size_t)k * C.ny + j) * C.pitch + i;
        R v[5];
        for (int f = 0; f < nf; ++f) v[f] = p[f * fs];
        acc.add(v, k, zt, C);
    }
    block_dt_reduce(acc.result(), acc.bad, ctl, slot);
}

// Packs planes [k0, k1) of a dense state (field-major, then k, j, i; any
// element type S, converted to R) into the pitched layout X and reduces the
// CFL bound of those nodes into dt slot `slot`, the operations of dt_reduce
// on the packed values.  One launch per plane chunk of an upload.
template <class R, class S>
__global__ void pack_dt(const S* __restrict__ dense, R* __restrict__ X, const R* __restrict__ zt, Coef<R> C,
                        DevCtl* ctl, int slot, int k0, int k1)
{
    DtAcc<R> acc;
    const long long plane = (long long)C.nx * C.ny;
    const long long field = plane * C.nz;
    const int nf = C.ndim == 3 ? 5 : 4;
    for (long long n = plane * k0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; n < plane * k1;
         n += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(n % C.nx);
        const long long row = n / C.nx;  // k*ny + j
        const int k = (int)(row / C.ny);
        R v[5];
        for (int f = 0; f < nf; ++f) {
            v[f] = (R)dense[f * field + n];
            X[f * C.fstride + row * C.pitch + i] = v[f];
        }
        acc.add(v, k, zt, C);
    }
    block_dt_reduce(acc.result(), acc.bad, ctl, slot);
}

// ---- diagnostics ---------------------------------------------------------

// deterministic block sum of kDiagQ doubles (fixed tree); result in thread 0
__device__ __forceinline__ void block_sum_q(double (&v)[kDiagQ], double* out)
{
    __shared__ double sh[kDiagThreads / 32][kDiagQ];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int q = 0; q < kDiagQ; ++q) {
        double x = v[q];
        for (int o = 16; o > 0; o >>= 1) {
            const double y = __shfl_xor_sync(0xffffffffu, x, o);
            x = (q == kDiagQ - 1) ? fmax(x, y) : x + y;
        }
        if (l == 0) sh[w][q] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 0; q < kDiagQ; ++q) {
            double x = sh[0][q];
            for (int ww = 1; ww < kDiagThreads / 32; ++ww) x = (q == kDiagQ - 1) ? fmax(x, sh[ww][q]) : x + sh[ww][q];
            out[q] = x;
        }
    }
}

// per-plane FP64 sums of the diagnostics integrands; one block per plane k,
// results in scratch[k*kDiagQ + q]
template <class R>
__global__ void __launch_bounds__(kDiagThreads) diag_planes(const R* X, Coef<R> C, DiagArgs A, double* scratch, DevCtl* ctl)
{
    const int k = blockIdx.x;
    const double z = A.zt[k];
    const long long fs = C.fstride;
    double v[kDiagQ] = {0, 0, 0, 0, 0, 0, 0, 0};
    // FP32 states: per-thread compensated (Kahan) FP32 sums of the FP32
    // integrands over the thread's nodes of the plane, widened once to FP64;
    // the max in FP32 (exact).  Every sum across threads, blocks and planes is
    // FP64.  (The compensated partial is accurate to FP32 rounding of the
    // partial itself, the precision of each integrand; on GB300 this keeps the
    // FP64 pipe out of the per-node work.)
    float ks[kDiagQ - 1] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float kc[kDiagQ - 1] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float mach32 = 0.f;
    int bad = 0;
    // node (j, i) of the plane: rows j, columns i strided by the block (no
    // division per node)
    for (int j = 0; j < C.ny; ++j)
    for (int i = threadIdx.x; i < C.nx; i += kDiagThreads) {
        const R* p = X + ((size_t)k * C.ny + j) * C.pitch + i;
        if constexpr (!kExact<R>) {
            const float rho = p[0], ri = 1.f / rho;
            const float u = p[fs] * ri;
            float vy = 0.f, w, E;
            if (C.ndim == 3) { vy = p[2 * fs] * ri; w = p[3 * fs] * ri; E = p[4 * fs]; }
            else { w = p[2 * fs] * ri; E = p[3 * fs]; }
            const float zf = (float)z;
            const float u2 = (u * u + vy * vy) + w * w;
            const float T = (float)A.b * (E * ri - 0.5f * u2 - (float)A.g * zf);
            const float Tsa = T - (1.f - (float)A.D * zf);
            const float x[kDiagQ - 1] = {rho, E, rho * w * Tsa, rho * w * u2, u2, 0.5f * rho * u2, T};
#pragma unroll
            for (int q = 0; q < kDiagQ - 1; ++q) {
                const float y = __fsub_rn(x[q], kc[q]);
                const float t = __fadd_rn(ks[q], y);
                kc[q] = __fsub_rn(__fsub_rn(t, ks[q]), y);
                ks[q] = t;
            }
            mach32 = fmaxf(mach32, sqrtf(u2) / sqrtf((float)A.cs2 * T));
            if (!isfinite(E + rho + T + u2)) bad = 1;
        } else {
            const double rho = (double)p[0];
            const double u = (double)p[fs] / rho;
            double vy = 0.0, w, E;
            if (C.ndim == 3) { vy = (double)p[2 * fs] / rho; w = (double)p[3 * fs] / rho; E = (double)p[4 * fs]; }
            else { w = (double)p[2 * fs] / rho; E = (double)p[3 * fs]; }
            const double u2 = u * u + vy * vy + w * w;
            const double T = A.b * (E / rho - 0.5 * u2 - A.g * z);
            const double Tsa = T - (1.0 - A.D * z);
            v[0] += rho;
            v[1] += E;
            v[2] += rho * w * Tsa;
            v[3] += rho * w * u2;
            v[4] += u2;
            v[5] += 0.5 * rho * u2;
            v[6] += T;
            const double M = sqrt(u2) / sqrt(A.cs2 * T);
            v[7] = fmax(v[7], M);
            if (!isfinite(E + rho + T + u2)) bad = 1;
        }
    }
    if constexpr (!kExact<R>) {
#pragma unroll
        for (int q = 0; q < kDiagQ - 1; ++q) v[q] = (double)ks[q] - (double)kc[q];
        v[7] = (double)mach32;
    }
    block_sum_q(v, scratch + (size_t)k * kDiagQ);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&ctl->status, 1);
}


// ---- extended diagnostics -------------------------------------------------

// FP64 primitives of the node at `off` (the oracle's order of operations)
template <class R>
__device__ __forceinline__ void ext_prims(const R* X, long long fs, int ndim, long long off, double z, const ExtArgs& A,
                                          double& rho, double& ux, double& uy, double& uz, double& T)
{
    rho = (double)X[off];
    ux = (double)X[off + fs] / rho;
    double E;
    if (ndim == 3) {
        uy = (double)X[off + 2 * fs] / rho;
        uz = (double)X[off + 3 * fs] / rho;
        E = (double)X[off + 4 * fs];
    } else {
        uy = 0.0;
        uz = (double)X[off + 2 * fs] / rho;
        E = (double)X[off + 3 * fs];
    }
    T = A.b * (E / rho - 0.5 * ((ux * ux + uy * uy) + uz * uz) - A.g * z);
}

// FP64 primitives of every node, once: P[q * n + node], q = 0..4 rho, u_x,
// u_y, u_z, T; node = (k ny + j) nx + i (dense)
template <class R>
__global__ void ext_prims_all(const R* X, Coef<R> C, ExtArgs A, double* P)
{
    const long long n = (long long)C.nx * C.ny * C.nz;
    for (long long d = blockIdx.x * (long long)blockDim.x + threadIdx.x; d < n; d += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(d % C.nx);
        const long long jk = d / C.nx;
        const int j = (int)(jk % C.ny), k = (int)(jk / C.ny);
        double rho, ux, uy, uz, T;
        ext_prims(X, C.fstride, C.ndim, ((long long)k * C.ny + j) * C.pitch + i, A.zt[k], A, rho, ux, uy, uz, T);
        P[d] = rho;
        P[n + d] = ux;
        P[2 * n + d] = uy;
        P[3 * n + d] = uz;
        P[4 * n + d] = T;
    }
}

// One block per plane k: FP64 sums over the plane of the z-momentum terms
// (z derivatives: derivative and second derivative at plane k of the
// quadratic through planes k-1, k, k+1; central on uniform planes)
//   F_n = rho (u . grad) u_z, F_p = -dp/dz, F_b = rho g,
//   F_v = mu (d_xx u_z + d_yy u_z + (2 + s) d_zz u_z + (1 + s)(d_x d_z u_x + d_y d_z u_y))
// (interior planes; 0 on the plates), of (rho u_z)^2, T_sa^2, rho u_z T_sa
// and T, the max of r = K_e/I_e = b u^2/(2T), and the histogram of log10 r,
// from the primitives P of ext_prims_all.  scratch[k*16 + q]: q = 0..5 F_n,
// F_p, F_b, F_v, (rho u_z)^2, T_sa^2; 6 rho u_z T_sa; 7 max r; 8 T; 9 rho;
// 10 u^2.
static __global__ void __launch_bounds__(kDiagThreads) ext_planes(int nx, int ny, int nz, int ndim, ExtArgs A, const double* P,
                                                           double* scratch)
{
    __shared__ unsigned int bins[kExtMaxBins];
    const int k = blockIdx.x, K = nz - 1;
    for (int q = threadIdx.x; q < A.nbins; q += kDiagThreads) bins[q] = 0u;
    __syncthreads();
    const long long N = (long long)nx * ny * nz;
    const double *Pr = P, *Pux = P + N, *Puy = P + 2 * N, *Puz = P + 3 * N, *PT = P + 4 * N;
    const double z = A.zt[k];
    const bool inner = k > 0 && k < K;
    double v[kDiagQ] = {0, 0, 0, 0, 0, 0, 0, 0};
    double tsum[kDiagQ] = {0, 0, 0, 0, 0, 0, 0, 0};
    auto at = [&](int kk, int j, int i) { return ((long long)kk * ny + j) * nx + i; };
    // the plane's spacings and the reciprocals of the three-plane derivatives'
    // denominators (one division each per block instead of per node)
    double hm = 1.0, hp = 1.0, iden = 0.0, ihm = 0.0, ihp = 0.0, ihs = 0.0;
    if (inner) {
        hm = A.zt[k] - A.zt[k - 1];
        hp = A.zt[k + 1] - A.zt[k];
        iden = 1.0 / (hm * hp * (hm + hp));
        ihm = 1.0 / hm;
        ihp = 1.0 / hp;
        ihs = 1.0 / (hm + hp);
    }
    auto dz = [&](double fm, double f0, double fp) { return (hm * hm * fp - hp * hp * fm + (hp * hp - hm * hm) * f0) * iden; };
    auto dzz = [&](double fm, double f0, double fp) { return 2.0 * ((fp - f0) * ihp - (f0 - fm) * ihm) * ihs; };
    const double i2dx = 1.0 / (2.0 * A.dx), idx2 = 1.0 / (A.dx * A.dx);
    const double i2dy = 1.0 / (2.0 * A.dy), idy2 = 1.0 / (A.dy * A.dy);
    for (long long n = threadIdx.x; n < (long long)nx * ny; n += kDiagThreads) {
        const int i = (int)(n % nx), j = (int)(n / nx);
        const long long c0 = at(k, j, i);
        const double rho = Pr[c0], ux = Pux[c0], uy = Puy[c0], uz = Puz[c0], T = PT[c0];
        const double Tsa = T - (1.0 - A.D * z);
        v[4] += (rho * uz) * (rho * uz);
        v[5] += Tsa * Tsa;
        v[6] += rho * uz * Tsa;
        tsum[0] += T;
        const double u2 = (ux * ux + uy * uy) + uz * uz;
        tsum[1] += rho;
        tsum[2] += u2;
        const double r = A.b * u2 / (2.0 * T);
        v[7] = fmax(v[7], r);
        int q = 0;
        if (r > 0.0) {
            const double t = (log10(r) - A.lo) / A.bw;
            q = t < 0.0 ? 0 : (t >= A.nbins ? A.nbins - 1 : (int)t);
        }
        atomicAdd(&bins[q], 1u);
        if (!inner) continue;
        const int ip = (i + 1) % nx, im = (i - 1 + nx) % nx;
        const long long zm = at(k - 1, j, i), zp = at(k + 1, j, i);
        const double uzp = Puz[at(k, j, ip)], uzm = Puz[at(k, j, im)];
        const double dxuz = (uzp - uzm) * i2dx;
        const double dxx = (uzp - 2.0 * uz + uzm) * idx2;
        const double dzuz = dz(Puz[zm], uz, Puz[zp]);
        const double dzzu = dzz(Puz[zm], uz, Puz[zp]);
        // d_x d_z u_x: x-central of the z derivatives at columns i +- 1
        const double dxdzux = (dz(Pux[at(k - 1, j, ip)], Pux[at(k, j, ip)], Pux[at(k + 1, j, ip)]) -
                               dz(Pux[at(k - 1, j, im)], Pux[at(k, j, im)], Pux[at(k + 1, j, im)])) * i2dx;
        double dyuz = 0.0, dyy = 0.0, dydzuy = 0.0;
        if (ndim == 3) {
            const int jp = (j + 1) % ny, jm = (j - 1 + ny) % ny;
            const double uyp_ = Puz[at(k, jp, i)], uym_ = Puz[at(k, jm, i)];
            dyuz = (uyp_ - uym_) * i2dy;
            dyy = (uyp_ - 2.0 * uz + uym_) * idy2;
            dydzuy = (dz(Puy[at(k - 1, jp, i)], Puy[at(k, jp, i)], Puy[at(k + 1, jp, i)]) -
                      dz(Puy[at(k - 1, jm, i)], Puy[at(k, jm, i)], Puy[at(k + 1, jm, i)])) * i2dy;
        }
        v[0] += rho * ((ux * dxuz + uy * dyuz) + uz * dzuz);
        v[1] += -dz(A.a * Pr[zm] * PT[zm], A.a * rho * T, A.a * Pr[zp] * PT[zp]);
        v[2] += rho * A.g;
        v[3] += A.mu * ((dxx + dyy) + (2.0 + A.stokes) * dzzu + (1.0 + A.stokes) * (dxdzux + dydzuy));
    }
    block_sum_q(v, scratch + (size_t)k * 16);
    __syncthreads();  // block_sum_q's shared staging is reused
    block_sum_q(tsum, scratch + (size_t)k * 16 + 8);
    __syncthreads();
    for (int q = threadIdx.x; q < A.nbins; q += kDiagThreads)
        if (bins[q]) atomicAdd(A.hist + q, (unsigned long long)bins[q]);
}

#ifdef CM_DEFINE_DIAG_FINAL  // one definition, in kernels_f64.cu
// combine the plane sums (trapezoid weights, fixed order) into one cm_diag
// record: Eq. volume_Nu, Eq. mean_Nu (second-order one-sided differences of
// <T_sa>_A at the plates), Eq. Re (instantaneous), KE, mass, energy.  On a
// stretched z-grid (F.zp) the weight of plane k is its cell width w_k and the
// plate derivative that of the quadratic through three planes.
__global__ void __launch_bounds__(kDiagThreads) diag_final(const double* scratch, const double* zt, DiagFinal F, DevCtl* ctl, cm_diag* rec)
{
    double v[kDiagQ] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = threadIdx.x; k < F.nz; k += kDiagThreads) {
        const double w = F.zp ? F.zp[k].w : ((k == 0 || k == F.nz - 1) ? 0.5 : 1.0);
        for (int q = 0; q < 6; ++q) v[q] += w * scratch[(size_t)k * kDiagQ + q];
        v[7] = fmax(v[7], scratch[(size_t)k * kDiagQ + 7]);
    }
    __shared__ double tot[kDiagQ];
    block_sum_q(v, tot);
    if (threadIdx.x == 0) {
        const double vol = F.zp ? F.cells : F.cells * (double)(F.nz - 1);
        const double sRP = sqrt(F.Ra * F.Pr);
        cm_diag d;
        d.Nu_conv = sRP / F.eps * (tot[2] / vol);
        d.Nu_K = F.D * sRP / 2.0 * (tot[3] / vol);
        d.Nu = 1.0 + d.Nu_conv + d.Nu_K;
        const int K = F.nz - 1;
        const double dz = 1.0 / (double)K;
        double f[3], g[3];
        for (int q = 0; q < 3; ++q) {
            f[q] = scratch[(size_t)q * kDiagQ + 6] / F.cells - (1.0 - F.D * zt[q]);
            g[q] = scratch[(size_t)(K - q) * kDiagQ + 6] / F.cells - (1.0 - F.D * zt[K - q]);
        }
        if (!F.zp) {
            d.Nu_bot = -(1.0 / F.eps) * (-3.0 * f[0] + 4.0 * f[1] - f[2]) / (2.0 * dz);
            d.Nu_top = -(1.0 / F.eps) * (3.0 * g[0] - 4.0 * g[1] + g[2]) / (2.0 * dz);
        } else {
            // spacings h1 (plate to the next plane) and h2 (the one after)
            double h1 = zt[1] - zt[0], h2 = zt[2] - zt[1];
            const double db = -(2.0 * h1 + h2) / (h1 * (h1 + h2)) * f[0] + (h1 + h2) / (h1 * h2) * f[1]
                              - h1 / (h2 * (h1 + h2)) * f[2];
            h1 = zt[K] - zt[K - 1];
            h2 = zt[K - 1] - zt[K - 2];
            const double dtp = (2.0 * h1 + h2) / (h1 * (h1 + h2)) * g[0] - (h1 + h2) / (h1 * h2) * g[1]
                               + h1 / (h2 * (h1 + h2)) * g[2];
            d.Nu_bot = -(1.0 / F.eps) * db;
            d.Nu_top = -(1.0 / F.eps) * dtp;
        }
        d.Nu_bar = (d.Nu_bot + d.Nu_top) / 2.0;
        d.Re = sqrt(F.Ra / F.Pr) * sqrt(tot[4] / vol);
        d.KE = tot[5] / vol;
        d.mass = tot[0] / vol;
        d.energy = tot[1] / vol;
        d.mach_max = tot[7];
        d.step = (long long)ctl->steps;
        d.t = ctl->t;
        d.dt = F.dt_fixed > 0.0 ? F.dt_fixed : F.cfl * __longlong_as_double((long long)ctl->dt_slot[F.slot]);
        d.status = (ctl->status & 1) || !isfinite(d.Nu + d.Nu_bar + d.Re + d.energy) ? CM_ENAN : CM_OK;
        d.pad_ = 0;
        *rec = d;
    }
}
#endif

}  // namespace cm
