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
//
// The sweep bodies (sweep2d_x2_body.inc) are compiled twice.  Namespace pkf
// uses the compiler intrinsics and specialised first steps: the fastest
// form, reproducible bit for bit for a given segment length, but a node's
// FP32 rounding may differ by an ulp with the segment length, because the
// compiler may round separately inlined copies of a step differently.
// Namespace pkx (cm_params.layout_exact) issues every packed operation as an
// opaque PTX instruction and runs interior segments through the same two
// copies of the step from their first step on, so results are bit for bit
// independent of the segment lengths the tuner picks (~6% slower at 4096 x
// 1024).
#pragma once
#include "cm_device.cuh"
#include "sweep2d_x2_types.h"

namespace cm {


typedef float2 f2;

__device__ __forceinline__ f2 bc(float s) { return make_float2(s, s); }
// Packed FP32x2 arithmetic as compiler intrinsics, rounded once per
// operation: the 3D kernels use these directly; the 2D sweeps below take one
// of two sets of their own (namespaces pkf and pkx).
__device__ __forceinline__ f2 add2f(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul2f(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2f(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
// a - b, rounded once
__device__ __forceinline__ f2 sub2f(f2 a, f2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
// a - s*b
__device__ __forceinline__ f2 fnma2f(f2 s, f2 b, f2 a) { return __ffma2_rn(make_float2(-s.x, -s.y), b, a); }

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
// max(a, b) that returns NaN if either is NaN (fmaxf would drop it)
__device__ __forceinline__ float fmax_nan(float a, float b)
{
    float r;
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}

// Delta of a sweep (dt/2 from the step's dt slot, or the single-sweep
// Delta) in FP32, with two FP64 multiplies and one conversion: equal to
// (float)Delta of the FP64 rule.  FP64 issues at a small fraction of the
// FP32 rate on this GPU and every thread of a sweep needs this value at its
// start, where an FP64 division per thread held the warps back at each
// launch.
__device__ __forceinline__ float sweep_delta_f32(const SweepCtl& sc, const Coef<float>& C)
{
    if (sc.Delta > 0.0) return (float)sc.Delta;
    if (C.dt_fixed > 0.0) return (float)(0.5 * C.dt_fixed);
    return (float)(0.5 * (C.cfl * __longlong_as_double((long long)sc.ctl->dt_slot[sc.slot_in])));
}

// the step's advance of t and the step counter, and the reset of the other
// dt slot, by one thread in the first sweep of a step (FP64)
__device__ __forceinline__ void step_bookkeeping(const SweepCtl& sc, const Coef<float>& C)
{
    sc.ctl->dt_slot[sc.slot_in ^ 1] = 0x7FF0000000000000ULL;
    sc.ctl->t += step_dt(sc.ctl, sc.slot_in, C.cfl, C.dt_fixed);
    sc.ctl->steps += 1.0;
}

__device__ __forceinline__ f2 abs2(f2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ f2 max2(f2 a, f2 b) { return make_float2(fmaxf(a.x, b.x), fmaxf(a.y, b.y)); }
__device__ __forceinline__ f2 sqrt2(f2 a) { return make_float2(sqrt_fast(a.x), sqrt_fast(a.y)); }
// next dt from the FP32 sweeps: the block's maximum of r = max (|u|+c)/h
// over its nodes (NaN-propagating), then one thread stores 1/r in FP64 into
// the dt slot; 1/r is monotone, so this is the minimum of h/(|u|+c) over the
// nodes.  A non-finite maximum sets the sticky status instead.  Every thread
// of the block calls it.
__device__ __forceinline__ void block_rmax_dt(float r, DevCtl* ctl, int slot)
{
    __shared__ float sm[32];
    for (int o = 16; o > 0; o >>= 1) r = fmax_nan(r, __shfl_xor_sync(0xffffffffu, r, o));
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = r;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = sm[0];
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) m = fmax_nan(m, sm[i]);
        if (!(m < 1e30f)) atomicOr(&ctl->status, 1);
        else if (m > 0.f) atomicMin(&ctl->dt_slot[slot], (unsigned long long)__double_as_longlong(1.0 / (double)m));
    }
}

// TVD coefficient G of the flux G dX, both columns at once:
//   C = c(1 - c), c = min(Co, 1/2);  phi(s) = clamp(2 s / dd, 0, 1)
//   Davis form: G = C (2 - phi(sp) - phi(sm)) / 2;  printed form: C (1 - phi(sp + sm)) / 2
// One reciprocal of dd serves both ratios.  dd = 0 (dX = 0) gives 0 * inf =
// NaN, which the clamp maps to 0; the flux G dX is 0 there anyway.
__device__ __forceinline__ float clamp01(float x) { return fminf(fmaxf(x, 0.f), 1.f); }

__device__ __forceinline__ f2 tvd_G2f(f2 sp, f2 sm, f2 dd, f2 Co, int form)
{
    const f2 c = make_float2(fminf(Co.x, 0.5f), fminf(Co.y, 0.5f));
    const f2 hC = mul2f(make_float2(0.5f, 0.5f), fma2f(make_float2(-c.x, -c.y), c, c));  // C/2
    const f2 r2 = mul2f(make_float2(2.f, 2.f), rcp2(dd));
    if (form == 0) {
        const f2 a = mul2f(sp, r2), b = mul2f(sm, r2);
        const f2 phis = make_float2(clamp01(a.x) + clamp01(b.x), clamp01(a.y) + clamp01(b.y));
        return mul2f(hC, sub2f(make_float2(2.f, 2.f), phis));
    }
    if (form == 1) {
        const f2 a = mul2f(add2f(sp, sm), r2);
        return mul2f(hC, sub2f(make_float2(1.f, 1.f), make_float2(clamp01(a.x), clamp01(a.y))));
    }
    return make_float2(0.f, 0.f);
}

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
// touches (ks - 3 .. ke + 1, clamped; ke + 2 for the extra step of an odd
// interior segment in pkx) into its own slice of shared memory,
// after the row ring, so that every row reads it by broadcast.  NV values
// per plane; entry e holds plane clamp(ks - 3 + e).
constexpr int kPlaneBack2 = 3;
__host__ __device__ constexpr int plane_cap2(int seg_rows) { return seg_rows + kPlaneBack2 + 3; }
template <int NV>
__device__ __forceinline__ float* plane_cache2(f2* ring_mem, int seg_rows)
{
    return reinterpret_cast<float*>(ring_mem + kRing * 4 * kThreads2) + (threadIdx.x >> 5) * plane_cap2(seg_rows) * NV;
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

constexpr size_t kRingBytes = (size_t)kRing * 4 * kThreads2 * sizeof(f2);


// ---- the two compiled forms of the 2D sweeps -----------------------------
namespace pkf {
constexpr bool kXL = false;
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return add2f(a, b); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return mul2f(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return fma2f(a, b, c); }
__device__ __forceinline__ f2 sub2(f2 a, f2 b) { return sub2f(a, b); }
__device__ __forceinline__ f2 fnma2(f2 s, f2 b, f2 a) { return fnma2f(s, b, a); }
#include "sweep2d_x2_body.inc"
}  // namespace pkf

namespace pkx {
constexpr bool kXL = true;
// each packed operation one PTX instruction, rounded once, that the compiler
// cannot merge, split or re-associate
__device__ __forceinline__ unsigned long long pk(f2 a) { return *reinterpret_cast<unsigned long long*>(&a); }
__device__ __forceinline__ f2 upk(unsigned long long d) { return *reinterpret_cast<f2*>(&d); }
__device__ __forceinline__ f2 add2(f2 a, f2 b)
{
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
    return upk(d);
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b)
{
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
    return upk(d);
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)), "l"(pk(c)));
    return upk(d);
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
    return upk(d);
}
__device__ __forceinline__ f2 fnma2(f2 s, f2 b, f2 a) { return fma2(make_float2(-s.x, -s.y), b, a); }
#include "sweep2d_x2_body.inc"
}  // namespace pkx

}  // namespace cm
