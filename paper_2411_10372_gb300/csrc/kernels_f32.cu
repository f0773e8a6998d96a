// FP32 instantiation of the kernels (state and stencil arithmetic in FP32,
// FMA contraction allowed; the dt rule and all reductions stay FP64).
#include "kernels_impl.cuh"
#include "sweep2d_x2.cuh"
#include "sweep3d_x2.cuh"

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
    using K = void (*)(SweepIO2, Coef<float>, SweepCtl);
    // [layout_exact][kernel]: z, x, x with dt, and the stretched-grid forms
    static const K kern[2][6] = {
        {pkf::sweep_z2d_x2, pkf::sweep_x2d_x2, pkf::sweep_x2d_x2_dt, pkf::sweep_z2d_x2s, pkf::sweep_x2d_x2s,
         pkf::sweep_x2d_x2s_dt},
        {pkx::sweep_z2d_x2, pkx::sweep_x2d_x2, pkx::sweep_x2d_x2_dt, pkx::sweep_z2d_x2s, pkx::sweep_x2d_x2s,
         pkx::sweep_x2d_x2s_dt}};
    static int bz = 0, bx = 0;
    if (!bz) {
        for (int v = 0; v < 2; ++v)
            for (int q = 0; q < 6; ++q)  // stretched kernels: the ring plus the warps' plane caches
                cudaFuncSetAttribute(kern[v][q], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kRingBytes + (q >= 3 ? 96 * 1024 : 0));
        bz = blocks_per_sm(pkf::sweep_z2d_x2, kRingBytes);
        bx = blocks_per_sm(pkf::sweep_x2d_x2, kRingBytes);
    }
    const K* k = kern[C.layout_exact ? 1 : 0];
    io.seg_rows = (seg_rows > 0 && !getenv("CM_SEG_ROWS")) ? seg_rows
                                                           : pick_segment(io.nstrips, C.nz, dir == 2 ? bz : bx, sm_count());
    const int nsegs = (C.nz + io.seg_rows - 1) / io.seg_rows;
    const long long warps = (long long)io.nstrips * nsegs;
    const int blocks = (int)((warps + kWarpsPerBlock - 1) / kWarpsPerBlock);
    const dim3 g(blocks), b(kWarpsPerBlock * 32);
    const size_t cache = (size_t)kWarpsPerBlock * plane_cap2(io.seg_rows) * sizeof(float);
    if (dir == 2)
        return C.zp ? launch_pdl(true, k[3], g, b, kRingBytes + 5 * cache, s, io, C, sc)
                    : launch_pdl(true, k[0], g, b, kRingBytes, s, io, C, sc);
    if (dir == 0) {
        // the last sweep of a step also reduces the next dt (separate kernels, so
        // that the other x sweeps carry none of that code)
        if (C.zp)
            return sc.last ? launch_pdl(true, k[5], g, b, kRingBytes + 2 * cache, s, io, C, sc)
                           : launch_pdl(true, k[4], g, b, kRingBytes + 2 * cache, s, io, C, sc);
        return sc.last ? launch_pdl(true, k[2], g, b, kRingBytes, s, io, C, sc)
                       : launch_pdl(true, k[1], g, b, kRingBytes, s, io, C, sc);
    }
    return cudaErrorInvalidValue;
}

template <int NW>
static cudaError_t sweep3_x2_nw(int dir, const float* in, float* out, const float* zt, const Coef<float>& C,
                                const SweepCtl& sc, int seg_rows, cudaStream_t s)
{
    Sweep3IO<float> io;
    io.in = in;
    io.out = out;
    io.zt = zt;
    io.nstrips = (C.nx + kOutW2 - 1) / kOutW2;
    io.nmarch = (dir == 1) ? C.ny : C.nz;
    io.nw = (dir == 1) ? C.nz : C.ny;
    const int groups = (io.nw + NW - 5) / (NW - 4);
    constexpr size_t ring = ring3_bytes(NW);
    // stretched grids: the block's plane cache after the ring (4 values per
    // plane for L_z, 2 for L_x, none for L_y), sized for the longest segment
    constexpr int kSegMax = 256;
    static bool attr = false;
    if (!attr) {
        const int ring_z = (int)(ring + plane_cache_bytes<float>(kSegMax, 4));
        const int ring_x = (int)(ring + plane_cache_bytes<float>(kSegMax, 2));
        cudaFuncSetAttribute(sweep3d_march_x2<2, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ring);
        cudaFuncSetAttribute(sweep3d_march_x2<1, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ring);
        cudaFuncSetAttribute(sweep3d_x_x2<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ring);
        cudaFuncSetAttribute(sweep3d_march_x2<2, NW, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, ring_z);
        cudaFuncSetAttribute(sweep3d_march_x2<1, NW, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ring);
        cudaFuncSetAttribute(sweep3d_x_x2<NW, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, ring_x);
        attr = true;
    }
    if (dir < 0 || dir > 2) return cudaErrorInvalidValue;
    io.seg = (seg_rows > 0 && !getenv("CM_SEG_ROWS"))
                 ? seg_rows
                 : pick_segment3((long long)io.nstrips * groups, io.nmarch, 1, sm_count());
    if (C.zp && io.seg > kSegMax) io.seg = kSegMax;
    const int nsegs = (io.nmarch + io.seg - 1) / io.seg;
    const dim3 grid(io.nstrips, groups, nsegs), b(NW * 32);
    if (C.zp) {
        const size_t ring_z = ring + plane_cache_bytes<float>(io.seg, 4), ring_x = ring + plane_cache_bytes<float>(io.seg, 2);
        if (dir == 2) return launch_pdl(false, sweep3d_march_x2<2, NW, true>, grid, b, ring_z, s, io, C, sc);
        if (dir == 1) return launch_pdl(false, sweep3d_march_x2<1, NW, true>, grid, b, ring, s, io, C, sc);
        return launch_pdl(false, sweep3d_x_x2<NW, true>, grid, b, ring_x, s, io, C, sc);
    }
    if (dir == 2) return launch_pdl(false, sweep3d_march_x2<2, NW>, grid, b, ring, s, io, C, sc);
    if (dir == 1) return launch_pdl(false, sweep3d_march_x2<1, NW>, grid, b, ring, s, io, C, sc);
    return launch_pdl(false, sweep3d_x_x2<NW>, grid, b, ring, s, io, C, sc);
}

cudaError_t launch_sweep3_x2(int dir, const float* in, float* out, const float* zt, const Coef<float>& C,
                             const SweepCtl& sc, int seg_rows, cudaStream_t s)
{
    static int nw = 0;
    if (!nw) {
        const char* e = getenv("CM_3D_NW");
        nw = e ? atoi(e) : kNW3pDefault;  // CM_3D_NW: block height (measurement)
        if (nw != 12 && nw != 14 && nw != 16) nw = kNW3pDefault;
    }
    if (nw == 12) return sweep3_x2_nw<12>(dir, in, out, zt, C, sc, seg_rows, s);
    if (nw == 14) return sweep3_x2_nw<14>(dir, in, out, zt, C, sc, seg_rows, s);
    return sweep3_x2_nw<16>(dir, in, out, zt, C, sc, seg_rows, s);
}

cudaError_t launch_sweep_batch(int dir, const BatchLaunch& L, int nblocks, bool const_coefs, bool stretched,
                               bool layout_exact, cudaStream_t s)
{
    // stretched: per-warp plane caches of 5 (z) or 2 (x) values per plane after the ring
    constexpr size_t kCacheZ = kRingBytes + (size_t)kWarpsPerBlock * plane_cap2(kBatchSegMax) * 5 * sizeof(float);
    constexpr size_t kCacheX = kRingBytes + (size_t)kWarpsPerBlock * plane_cap2(kBatchSegMax) * 2 * sizeof(float);
    using K = void (*)(BatchLaunch);
    // [layout_exact][kernel][stretched][const coefficients]; kernel: z, x, x with dt
    static const K kern[2][3][2][2] = {
        {{{pkf::sweep_z2d_batch_smem<false>, pkf::sweep_z2d_batch<false>},
          {pkf::sweep_z2d_batch_smem<true>, pkf::sweep_z2d_batch<true>}},
         {{pkf::sweep_x2d_batch_smem<false, 0>, pkf::sweep_x2d_batch<false, 0>},
          {pkf::sweep_x2d_batch_smem<true, 0>, pkf::sweep_x2d_batch<true, 0>}},
         {{pkf::sweep_x2d_batch_smem<false, 1>, pkf::sweep_x2d_batch<false, 1>},
          {pkf::sweep_x2d_batch_smem<true, 1>, pkf::sweep_x2d_batch<true, 1>}}},
        {{{pkx::sweep_z2d_batch_smem<false>, pkx::sweep_z2d_batch<false>},
          {pkx::sweep_z2d_batch_smem<true>, pkx::sweep_z2d_batch<true>}},
         {{pkx::sweep_x2d_batch_smem<false, 0>, pkx::sweep_x2d_batch<false, 0>},
          {pkx::sweep_x2d_batch_smem<true, 0>, pkx::sweep_x2d_batch<true, 0>}},
         {{pkx::sweep_x2d_batch_smem<false, 1>, pkx::sweep_x2d_batch<false, 1>},
          {pkx::sweep_x2d_batch_smem<true, 1>, pkx::sweep_x2d_batch<true, 1>}}}};
    static bool init = false;
    if (!init) {
        for (int v = 0; v < 2; ++v)
            for (int d = 0; d < 3; ++d)
                for (int st = 0; st < 2; ++st)
                    for (int cc = 0; cc < 2; ++cc)
                        cudaFuncSetAttribute(kern[v][d][st][cc], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(st ? (d == 0 ? kCacheZ : kCacheX) : kRingBytes));
        init = true;
    }
    if (dir != 2 && dir != 0) return cudaErrorInvalidValue;
    const int d = dir == 2 ? 0 : (L.last ? 2 : 1);
    const size_t smem = stretched ? (d == 0 ? kCacheZ : kCacheX) : kRingBytes;
    kern[layout_exact ? 1 : 0][d][stretched ? 1 : 0][const_coefs ? 1 : 0]<<<nblocks, kThreads2, smem, s>>>(L);
    return cudaGetLastError();
}

cudaError_t set_batch_coefs(const Coef<float>* C, int n, cudaStream_t s)
{
    if (n < 1 || n > kConstBoxes) return cudaErrorInvalidValue;
    return cudaMemcpyToSymbolAsync(c_box, C, n * sizeof(Coef<float>), 0, cudaMemcpyHostToDevice, s);
}

}  // namespace cm
