// sweep3d_common.cuh -- 3D state, primitives and flux of the MacCormack-TVD
// sweeps (Sec. 2 closures, Sec. 3.1 flux F_alpha, any direction alpha).
//
// 3D state X = (rho, m_x, m_y, m_z, E).  The FP64 instantiation evaluates
// every formula in a fixed written order with true divisions (see
// cm_device.cuh), the FP32 one with reciprocals.
#pragma once
#include "cm_device.cuh"

namespace cm {

template <class R>
struct S3 {
    R r, m[3], E;
};

template <class R>
__device__ __forceinline__ S3<R> s3_sub(const S3<R>& a, const S3<R>& b)
{
    return {a.r - b.r, {a.m[0] - b.m[0], a.m[1] - b.m[1], a.m[2] - b.m[2]}, a.E - b.E};
}

// dot product over the five components, summed in component order
template <class R>
__device__ __forceinline__ R s3_dot(const S3<R>& a, const S3<R>& b)
{
    return (((a.r * b.r + a.m[0] * b.m[0]) + a.m[1] * b.m[1]) + a.m[2] * b.m[2]) + a.E * b.E;
}

template <class R>
__device__ __forceinline__ void prims3(const S3<R>& q, R z, const Coef<R>& C, R (&u)[3], R& T, R& p)
{
    if constexpr (kExact<R>) {
        u[0] = q.m[0] / q.r;
        u[1] = q.m[1] / q.r;
        u[2] = q.m[2] / q.r;
        T = C.b * (q.E / q.r - R(0.5) * ((u[0] * u[0] + u[1] * u[1]) + u[2] * u[2]) - C.g * z);
    } else {
        const R ri = R(1) / q.r;
        u[0] = q.m[0] * ri;
        u[1] = q.m[1] * ri;
        u[2] = q.m[2] * ri;
        T = C.b * (q.E * ri - R(0.5) * ((u[0] * u[0] + u[1] * u[1]) + u[2] * u[2]) - C.g * z);
    }
    p = C.a * q.r * T;
}

// F_al at one node from the velocity gradient du[c][d] = d u_c / d x_d and
// dT_al = dT/dx_al:
//   [ m_al ;  m_i u_al - tau_{i al} + p delta_{i al} ;  u_al (E + p) - K dT_al - u_b tau_{b al} ]
//   tau_ij = mu (d_j u_i + d_i u_j + s (div u) delta_ij)
template <int AL, class R>
__device__ __forceinline__ S3<R> flux3(const S3<R>& q, const R (&u)[3], R p, const R (&du)[3][3], R dT_al,
                                       const Coef<R>& C)
{
    const R div = (du[0][0] + du[1][1]) + du[2][2];
    R tau[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
        tau[i] = (i == AL) ? C.mu * ((du[i][AL] + du[AL][i]) + C.stokes * div) : C.mu * (du[i][AL] + du[AL][i]);
    S3<R> F;
    F.r = q.m[AL];
#pragma unroll
    for (int i = 0; i < 3; ++i) F.m[i] = (i == AL) ? (q.m[i] * u[AL] - tau[i]) + p : q.m[i] * u[AL] - tau[i];
    const R work = (u[0] * tau[0] + u[1] * tau[1]) + u[2] * tau[2];
    F.E = (u[AL] * (q.E + p) - C.kth * dT_al) - work;
    return F;
}

template <class R>
__device__ __forceinline__ R span_of(const Coef<R>& C, int d, bool central)
{
    if (d == 0) return central ? C.h2x : C.hx;
    if (d == 1) return central ? C.h2y : C.hy;
    return central ? C.h2z : C.hz;
}

template <class R>
__device__ __forceinline__ R inv_span_of(const Coef<R>& C, int d, bool central)
{
    if (d == 0) return central ? C.inv_2dx : C.inv_dx;
    if (d == 1) return central ? C.inv_2dy : C.inv_dy;
    return central ? C.inv_2dz : C.inv_dz;
}

// (a - b) / span for direction d
template <class R>
__device__ __forceinline__ R d3(R a, R b, const Coef<R>& C, int d, bool central)
{
    return diff(a, b, span_of(C, d, central), inv_span_of(C, d, central));
}

template <class R>
__device__ __forceinline__ S3<R> s3_load(const R* __restrict__ base, long long fs, long long off)
{
    const R* s = base + off;
    return {__ldg(s), {__ldg(s + fs), __ldg(s + 2 * fs), __ldg(s + 3 * fs)}, __ldg(s + 4 * fs)};
}

template <class R>
__device__ __forceinline__ void s3_store(R* __restrict__ base, long long fs, long long off, const S3<R>& q)
{
    R* d = base + off;
    d[0] = q.r;
    d[fs] = q.m[0];
    d[2 * fs] = q.m[1];
    d[3 * fs] = q.m[2];
    d[4 * fs] = q.E;
}

}  // namespace cm
