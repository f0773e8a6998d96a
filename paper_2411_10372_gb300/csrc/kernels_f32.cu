// FP32 instantiation of the kernels (state and stencil arithmetic in FP32,
// FMA contraction allowed; the dt rule and all reductions stay FP64).
#include "kernels_impl.cuh"
#include "sweep2d_x2.cuh"

namespace cm {

template struct Launch<float>;

cudaError_t launch_sweep_x2(int dir, const float* in, float* out, const float* zt, const Coef<float>& C,
                            const SweepCtl& sc, int seg_rows, cudaStream_t s)
{
    SweepIO2 io;
    io.in = in;
    io.out = out;
    io.zt = zt;
    io.nstrips = (C.nx + kOutW2 - 1) / kOutW2;
    static int bz = 0, bx = 0;
    if (!bz) {
        cudaFuncSetAttribute(sweep_z2d_x2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingBytes);
        cudaFuncSetAttribute(sweep_x2d_x2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingBytes);
        cudaFuncSetAttribute(sweep_x2d_x2_dt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingBytes);
        // stretched kernels: the ring plus the warps' plane caches
        cudaFuncSetAttribute(sweep_z2d_x2s, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingBytes + 96 * 1024);
        cudaFuncSetAttribute(sweep_x2d_x2s, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingBytes + 96 * 1024);
        cudaFuncSetAttribute(sweep_x2d_x2s_dt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingBytes + 96 * 1024);
        bz = blocks_per_sm(sweep_z2d_x2, kRingBytes);
        bx = blocks_per_sm(sweep_x2d_x2, kRingBytes);
    }
    io.seg_rows = (seg_rows > 0 && !getenv("CM_SEG_ROWS")) ? seg_rows
                                                           : pick_segment(io.nstrips, C.nz, dir == 2 ? bz : bx, sm_count());
    const int nsegs = (C.nz + io.seg_rows - 1) / io.seg_rows;
    const long long warps = (long long)io.nstrips * nsegs;
    const int blocks = (int)((warps + kWarpsPerBlock - 1) / kWarpsPerBlock);
    const dim3 g(blocks), b(kWarpsPerBlock * 32);
    const size_t cache = (size_t)kWarpsPerBlock * plane_cap2(io.seg_rows) * sizeof(float);
    if (dir == 2)
        return C.zp ? launch_pdl(true, sweep_z2d_x2s, g, b, kRingBytes + 5 * cache, s, io, C, sc)
                    : launch_pdl(true, sweep_z2d_x2, g, b, kRingBytes, s, io, C, sc);
    if (dir == 0) {
        // the last sweep of a step also reduces the next dt (separate kernels, so
        // that the other x sweeps carry none of that code)
        if (C.zp)
            return sc.last ? launch_pdl(true, sweep_x2d_x2s_dt, g, b, kRingBytes + 2 * cache, s, io, C, sc)
                           : launch_pdl(true, sweep_x2d_x2s, g, b, kRingBytes + 2 * cache, s, io, C, sc);
        return sc.last ? launch_pdl(true, sweep_x2d_x2_dt, g, b, kRingBytes, s, io, C, sc)
                       : launch_pdl(true, sweep_x2d_x2, g, b, kRingBytes, s, io, C, sc);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_sweep_batch(int dir, const BatchLaunch& L, int nblocks, bool const_coefs, bool stretched,
                               cudaStream_t s)
{
    // stretched: per-warp plane caches of 5 (z) or 2 (x) values per plane after the ring
    constexpr size_t kCacheZ = kRingBytes + (size_t)kWarpsPerBlock * plane_cap2(kBatchSegMax) * 5 * sizeof(float);
    constexpr size_t kCacheX = kRingBytes + (size_t)kWarpsPerBlock * plane_cap2(kBatchSegMax) * 2 * sizeof(float);
    static bool init = false;
    if (!init) {
        cudaFuncSetAttribute(sweep_z2d_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingBytes);
        cudaFuncSetAttribute(sweep_x2d_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingBytes);
        cudaFuncSetAttribute(sweep_z2d_batch_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingBytes);
        cudaFuncSetAttribute(sweep_x2d_batch_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingBytes);
        cudaFuncSetAttribute(sweep_z2d_batch_s, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCacheZ);
        cudaFuncSetAttribute(sweep_x2d_batch_s, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCacheX);
        cudaFuncSetAttribute(sweep_z2d_batch_smem_s, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCacheZ);
        cudaFuncSetAttribute(sweep_x2d_batch_smem_s, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCacheX);
        init = true;
    }
    if (dir == 2) {
        if (stretched) {
            if (const_coefs) sweep_z2d_batch_s<<<nblocks, kThreads2, kCacheZ, s>>>(L);
            else sweep_z2d_batch_smem_s<<<nblocks, kThreads2, kCacheZ, s>>>(L);
        } else {
            if (const_coefs) sweep_z2d_batch<<<nblocks, kThreads2, kRingBytes, s>>>(L);
            else sweep_z2d_batch_smem<<<nblocks, kThreads2, kRingBytes, s>>>(L);
        }
    } else if (dir == 0) {
        if (stretched) {
            if (const_coefs) sweep_x2d_batch_s<<<nblocks, kThreads2, kCacheX, s>>>(L);
            else sweep_x2d_batch_smem_s<<<nblocks, kThreads2, kCacheX, s>>>(L);
        } else {
            if (const_coefs) sweep_x2d_batch<<<nblocks, kThreads2, kRingBytes, s>>>(L);
            else sweep_x2d_batch_smem<<<nblocks, kThreads2, kRingBytes, s>>>(L);
        }
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t set_batch_coefs(const Coef<float>* C, int n, cudaStream_t s)
{
    if (n < 1 || n > kConstBoxes) return cudaErrorInvalidValue;
    return cudaMemcpyToSymbolAsync(c_box, C, n * sizeof(Coef<float>), 0, cudaMemcpyHostToDevice, s);
}

}  // namespace cm
