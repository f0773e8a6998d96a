// kernels_impl.cuh -- launcher definitions; included once per precision.
#pragma once
#include <cstdlib>
#include "kernels.h"
#include "sweep2d.cuh"
#include "sweep3d.cuh"
#include "aux_kernels.cuh"

namespace cm {

template <class R, class S>
__global__ void pack_state(const S* __restrict__ dense, R* __restrict__ X, Coef<R> C, int nf)
{
    const long long plane = (long long)C.nx * C.ny * C.nz;
    const long long total = plane * nf;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < total; n += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(n / plane);
        const long long r = n % plane;
        const int i = (int)(r % C.nx);
        const long long row = r / C.nx;  // k*ny + j
        X[f * C.fstride + row * C.pitch + i] = (R)dense[n];
    }
}

template <class R, class S>
__global__ void unpack_state(const R* __restrict__ X, S* __restrict__ dense, Coef<R> C, int nf)
{
    const long long plane = (long long)C.nx * C.ny * C.nz;
    const long long total = plane * nf;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < total; n += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(n / plane);
        const long long r = n % plane;
        const int i = (int)(r % C.nx);
        const long long row = r / C.nx;
        dense[n] = (S)X[f * C.fstride + row * C.pitch + i];
    }
}

static inline int sm_count()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

// grid-stride launches: at most 16 blocks per SM
static inline int grid_for(long long work, int threads)
{
    long long b = (work + threads - 1) / threads;
    if (b > 16LL * sm_count()) b = 16LL * sm_count();
    if (b < 1) b = 1;
    return (int)b;
}

// rows per warp segment: each segment pays a 4-row pipeline ramp, and the
// grid should fill the GPU in whole waves; pick the segment length that
// minimises waves * (rows + ramp) for the kernel's occupancy
static inline int pick_segment(int nstrips, int nz, int blocks_per_sm, int nsm)
{
    // CM_SEG_ROWS=n forces the segment length (tuning experiments)
    if (const char* e = getenv("CM_SEG_ROWS")) {
        const int v = atoi(e);
        if (v >= 4 && v <= 4096) return v;
    }
    const long long cap = (long long)blocks_per_sm * kWarpsPerBlock * nsm;
    int best = 64;
    double best_cost = 1e300;
    for (int seg = 256; seg >= 8; seg /= 2) {
        const long long warps = (long long)nstrips * ((nz + seg - 1) / seg);
        const long long waves = (warps + cap - 1) / cap;
        const double cost = (double)waves * (double)(seg + 4);
        if (cost < best_cost - 1e-9) { best_cost = cost; best = seg; }
    }
    return best;
}

template <class K>
static inline int blocks_per_sm(K kernel, size_t smem = 0)
{
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, kWarpsPerBlock * 32, smem) != cudaSuccess || b < 1) {
        cudaGetLastError();
        b = 1;
    }
    return b;
}

// 3D sweeps: warps per block of the 2.5D kernels (the outer two on each side
// are halo), and the march segment minimising waves * (rows + ramp)
constexpr int kNW3 = 16;

static inline int pick_segment3(long long blocks_per_seg, int nmarch, int blocks_per_sm, int nsm)
{
    if (const char* e = getenv("CM_SEG_ROWS")) {
        const int v = atoi(e);
        if (v >= 4 && v <= 4096) return v;
    }
    const long long cap = (long long)blocks_per_sm * nsm;
    int top = 8;
    while (top < nmarch && top < 4096) top *= 2;
    int best = top;
    double best_cost = 1e300;
    for (int seg = top; seg >= 8; seg /= 2) {
        const long long blocks = blocks_per_seg * ((nmarch + seg - 1) / seg);
        const long long waves = (blocks + cap - 1) / cap;
        const double cost = (double)waves * (double)(seg + 4);
        if (cost < best_cost - 1e-9) { best_cost = cost; best = seg; }
    }
    return best;
}

template <class K>
static inline int blocks_per_sm3(K kernel)
{
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, kNW3 * 32, 0) != cudaSuccess || b < 1) {
        cudaGetLastError();
        b = 1;
    }
    return b;
}

// one 3D sweep: dir 2 = L_z (march z, warps over y), 1 = L_y (march y, warps
// over z), 0 = L_x (march z, warps over y); grid (x strips, W groups, segments)
template <class R>
static cudaError_t sweep3(int dir, const R* in, R* out, const R* zt, const Coef<R>& C, const SweepCtl& sc,
                          int seg_rows, cudaStream_t s)
{
    Sweep3IO<R> io;
    io.in = in;
    io.out = out;
    io.zt = zt;
    io.nstrips = (C.nx + kOutW - 1) / kOutW;
    io.nmarch = (dir == 1) ? C.ny : C.nz;
    io.nw = (dir == 1) ? C.nz : C.ny;
    const int groups = (io.nw + kNW3 - 5) / (kNW3 - 4);
    static int bps[3] = {0, 0, 0};
    if (!bps[0]) {
        bps[0] = blocks_per_sm3(sweep3d_x<R, kNW3>);
        bps[1] = blocks_per_sm3(sweep3d_march<R, 1, kNW3>);
        bps[2] = blocks_per_sm3(sweep3d_march<R, 2, kNW3>);
    }
    if (dir < 0 || dir > 2) return cudaErrorInvalidValue;
    io.seg = (seg_rows > 0 && !getenv("CM_SEG_ROWS"))
                 ? seg_rows
                 : pick_segment3((long long)io.nstrips * groups, io.nmarch, bps[dir], sm_count());
    const int nsegs = (io.nmarch + io.seg - 1) / io.seg;
    const dim3 grid(io.nstrips, groups, nsegs), b(kNW3 * 32);
    if (C.zp) {  // stretched z-grid: the z and x kernels cache the segment's plane metric in shared memory
        static bool attr = false;
        if (!attr) {
            const int lim = 96 * 1024;
            cudaFuncSetAttribute(sweep3d_march<R, 2, kNW3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
            cudaFuncSetAttribute(sweep3d_x<R, kNW3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
            attr = true;
        }
        if (dir == 2)
            return launch_pdl(false, sweep3d_march<R, 2, kNW3, true>, grid, b, plane_cache_bytes<R>(io.seg, 4), s, io, C, sc);
        if (dir == 1) return launch_pdl(false, sweep3d_march<R, 1, kNW3, true>, grid, b, 0, s, io, C, sc);
        return launch_pdl(false, sweep3d_x<R, kNW3, true>, grid, b, plane_cache_bytes<R>(io.seg, 2), s, io, C, sc);
    }
    if (dir == 2) return launch_pdl(false, sweep3d_march<R, 2, kNW3>, grid, b, 0, s, io, C, sc);
    if (dir == 1) return launch_pdl(false, sweep3d_march<R, 1, kNW3>, grid, b, 0, s, io, C, sc);
    return launch_pdl(false, sweep3d_x<R, kNW3>, grid, b, 0, s, io, C, sc);
}

template <class R>
cudaError_t Launch<R>::sweep(int dir, const R* in, R* out, const R* zt, const Coef<R>& C, const SweepCtl& sc,
                             int seg_rows, cudaStream_t s)
{
    if (C.ndim == 3) {
        if constexpr (std::is_same<R, float>::value) {
            if (C.nx % 2 == 0 && !getenv("CM_3D_SCALAR") && (long long)C.fstride * 5 < (1LL << 31))
                return launch_sweep3_x2(dir, in, out, zt, C, sc, seg_rows, s);
        }
        return sweep3(dir, in, out, zt, C, sc, seg_rows, s);
    }
    if constexpr (std::is_same<R, float>::value) {
        if (C.nx % 2 == 0 && (long long)C.fstride * 5 < (1LL << 31))
            return launch_sweep_x2(dir, in, out, zt, C, sc, seg_rows, s);
    }
    (void)seg_rows;
    SweepIO<R> io;
    io.in = in;
    io.out = out;
    io.zt = zt;
    io.nstrips = (C.nx + kOutW - 1) / kOutW;
    static int bz = 0, bx = 0;
    if (!bz) { bz = blocks_per_sm(sweep_z2d<R, false>); bx = blocks_per_sm(sweep_x2d<R, false>); }
    io.seg_rows = pick_segment(io.nstrips, C.nz, dir == 2 ? bz : bx, sm_count());
    const int nsegs = (C.nz + io.seg_rows - 1) / io.seg_rows;
    const long long warps = (long long)io.nstrips * nsegs;
    const int blocks = (int)((warps + kWarpsPerBlock - 1) / kWarpsPerBlock);
    const dim3 g(blocks), b(kWarpsPerBlock * 32);
    if (dir == 2)
        return C.zp ? launch_pdl(false, sweep_z2d<R, true>, g, b, 0, s, io, C, sc)
                    : launch_pdl(false, sweep_z2d<R, false>, g, b, 0, s, io, C, sc);
    if (dir == 0)
        return C.zp ? launch_pdl(false, sweep_x2d<R, true>, g, b, 0, s, io, C, sc)
                    : launch_pdl(false, sweep_x2d<R, false>, g, b, 0, s, io, C, sc);
    return cudaErrorInvalidValue;
}

template <class R>
cudaError_t Launch<R>::init(R* X, const Coef<R>& C, const InitArgs& A, cudaStream_t s)
{
    dim3 g(grid_for((long long)C.nx * C.ny, 256) > 64 ? 64 : grid_for((long long)C.nx * C.ny, 256), C.nz);
    init_state<R><<<g, 256, 0, s>>>(X, C, A);
    return cudaGetLastError();
}

template <class R>
cudaError_t Launch<R>::dt(const R* X, const R* zt, const Coef<R>& C, DevCtl* ctl, int slot, cudaStream_t s)
{
    dt_reduce<R><<<grid_for((long long)C.nx * C.ny * C.nz, 256), 256, 0, s>>>(X, zt, C, ctl, slot);
    return cudaGetLastError();
}

template <class R>
cudaError_t Launch<R>::ext_planes(const R* X, const Coef<R>& C, const ExtArgs& A, double* prims, double* scratch,
                                  cudaStream_t s)
{
    ext_prims_all<R><<<grid_for((long long)C.nx * C.ny * C.nz, 256), 256, 0, s>>>(X, C, A, prims);
    cm::ext_planes<<<C.nz, kDiagThreads, 0, s>>>(C.nx, C.ny, C.nz, C.ndim, A, prims, scratch);
    return cudaGetLastError();
}

template <class R>
cudaError_t Launch<R>::diag_planes(const R* X, const Coef<R>& C, const DiagArgs& A, double* scratch, DevCtl* ctl,
                                   cudaStream_t s)
{
    cm::diag_planes<R><<<C.nz, kDiagThreads, 0, s>>>(X, C, A, scratch, ctl);
    return cudaGetLastError();
}

template <class R>
cudaError_t Launch<R>::pack(const double* dense, R* X, const Coef<R>& C, int nf, cudaStream_t s)
{
    pack_state<R, double><<<grid_for((long long)C.nx * C.ny * C.nz * nf, 256), 256, 0, s>>>(dense, X, C, nf);
    return cudaGetLastError();
}

template <class R>
cudaError_t Launch<R>::unpack(const R* X, double* dense, const Coef<R>& C, int nf, cudaStream_t s)
{
    unpack_state<R, double><<<grid_for((long long)C.nx * C.ny * C.nz * nf, 256), 256, 0, s>>>(X, dense, C, nf);
    return cudaGetLastError();
}

template <class R>
cudaError_t Launch<R>::pack32(const float* dense, R* X, const Coef<R>& C, int nf, cudaStream_t s)
{
    pack_state<R, float><<<grid_for((long long)C.nx * C.ny * C.nz * nf, 256), 256, 0, s>>>(dense, X, C, nf);
    return cudaGetLastError();
}

template <class R>
cudaError_t Launch<R>::unpack32(const R* X, float* dense, const Coef<R>& C, int nf, cudaStream_t s)
{
    unpack_state<R, float><<<grid_for((long long)C.nx * C.ny * C.nz * nf, 256), 256, 0, s>>>(X, dense, C, nf);
    return cudaGetLastError();
}

template <class R>
cudaError_t Launch<R>::pack_dt(const double* dense, R* X, const R* zt, const Coef<R>& C, DevCtl* ctl, int slot,
                               int k0, int k1, cudaStream_t s)
{
    cm::pack_dt<R, double><<<grid_for((long long)C.nx * C.ny * (k1 - k0), 256), 256, 0, s>>>(dense, X, zt, C, ctl,
                                                                                             slot, k0, k1);
    return cudaGetLastError();
}

template <class R>
cudaError_t Launch<R>::pack_dt32(const float* dense, R* X, const R* zt, const Coef<R>& C, DevCtl* ctl, int slot,
                                 int k0, int k1, cudaStream_t s)
{
    cm::pack_dt<R, float><<<grid_for((long long)C.nx * C.ny * (k1 - k0), 256), 256, 0, s>>>(dense, X, zt, C, ctl,
                                                                                            slot, k0, k1);
    return cudaGetLastError();
}

}  // namespace cm
