// kernels_impl.cuh -- launcher definitions; included once per precision.
#pragma once
#include "kernels.h"
#include "sweep2d.cuh"
#include "aux_kernels.cuh"

namespace cm {

template <class R>
__global__ void pack_state(const double* __restrict__ dense, R* __restrict__ X, Coef<R> C, int nf)
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

template <class R>
__global__ void unpack_state(const R* __restrict__ X, double* __restrict__ dense, Coef<R> C, int nf)
{
    const long long plane = (long long)C.nx * C.ny * C.nz;
    const long long total = plane * nf;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < total; n += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(n / plane);
        const long long r = n % plane;
        const int i = (int)(r % C.nx);
        const long long row = r / C.nx;
        dense[n] = (double)X[f * C.fstride + row * C.pitch + i];
    }
}

static inline int grid_for(long long work, int threads)
{
    long long b = (work + threads - 1) / threads;
    if (b > 152LL * 16) b = 152LL * 16;
    if (b < 1) b = 1;
    return (int)b;
}

template <class R>
cudaError_t Launch<R>::sweep(int dir, const R* in, R* out, const R* zt, const Coef<R>& C, const SweepCtl& sc,
                             int seg_rows, cudaStream_t s)
{
    SweepIO<R> io;
    io.in = in;
    io.out = out;
    io.zt = zt;
    io.seg_rows = seg_rows;
    io.nstrips = (C.nx + kOutW - 1) / kOutW;
    const int nsegs = (C.nz + seg_rows - 1) / seg_rows;
    const long long warps = (long long)io.nstrips * nsegs;
    const int blocks = (int)((warps + kWarpsPerBlock - 1) / kWarpsPerBlock);
    if (dir == 2) sweep_z2d<R><<<blocks, kWarpsPerBlock * 32, 0, s>>>(io, C, sc);
    else if (dir == 0) sweep_x2d<R><<<blocks, kWarpsPerBlock * 32, 0, s>>>(io, C, sc);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
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
cudaError_t Launch<R>::diag_planes(const R* X, const Coef<R>& C, const DiagArgs& A, double* scratch, DevCtl* ctl,
                                   cudaStream_t s)
{
    cm::diag_planes<R><<<C.nz, kDiagThreads, 0, s>>>(X, C, A, scratch, ctl);
    return cudaGetLastError();
}

template <class R>
cudaError_t Launch<R>::pack(const double* dense, R* X, const Coef<R>& C, int nf, cudaStream_t s)
{
    pack_state<R><<<grid_for((long long)C.nx * C.ny * C.nz * nf, 256), 256, 0, s>>>(dense, X, C, nf);
    return cudaGetLastError();
}

template <class R>
cudaError_t Launch<R>::unpack(const R* X, double* dense, const Coef<R>& C, int nf, cudaStream_t s)
{
    unpack_state<R><<<grid_for((long long)C.nx * C.ny * C.nz * nf, 256), 256, 0, s>>>(X, dense, C, nf);
    return cudaGetLastError();
}

}  // namespace cm
