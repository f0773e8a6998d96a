// kernels.h -- host-side launchers of the device kernels, one instantiation
// per state precision (kernels_f64.cu, kernels_f32.cu).
#pragma once
#include <cuda_runtime.h>
#include "cm_device.cuh"
#include "../../include/cm.h"

namespace cm {

// launch, with programmatic stream serialization when pdl is set (the sweeps
// call pdl_enter first), so a sweep is scheduled while the previous one
// drains.  Used for the packed FP32 2D sweeps (-5% per step at 4096 x 1024);
// the FP64 sweeps run slower with it (-28% at 1024 x 256) and the 3D ones
// gain nothing, so they launch plainly.  CM_PDL=0 turns it off everywhere.
bool pdl_enabled();

template <class K, class... Args>
cudaError_t launch_pdl(bool pdl, K kernel, dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = (pdl && pdl_enabled()) ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <class R>
struct Launch {
    // one sweep L_dir (dir 0 = x, 1 = y (3D only), 2 = z); seg_rows: rows per
    // warp segment of the packed FP32 2D sweeps (0 = occupancy model)
    static cudaError_t sweep(int dir, const R* in, R* out, const R* zt, const Coef<R>& C, const SweepCtl& sc,
                             int seg_rows, cudaStream_t s);
    static cudaError_t init(R* X, const Coef<R>& C, const InitArgs& A, cudaStream_t s);
    static cudaError_t dt(const R* X, const R* zt, const Coef<R>& C, DevCtl* ctl, int slot, cudaStream_t s);
    static cudaError_t diag_planes(const R* X, const Coef<R>& C, const DiagArgs& A, double* scratch, DevCtl* ctl,
                                   cudaStream_t s);
    // extended diagnostics: FP64 primitives of every node into prims (5 x nodes),
    // then per-plane sums into scratch[k*16 + q] (see ext_planes)
    static cudaError_t ext_planes(const R* X, const Coef<R>& C, const ExtArgs& A, double* prims, double* scratch,
                                  cudaStream_t s);
    // dense float64 [nf][nz][ny][nx] <-> pitched state in R
    static cudaError_t pack(const double* dense, R* X, const Coef<R>& C, int nf, cudaStream_t s);
    static cudaError_t unpack(const R* X, double* dense, const Coef<R>& C, int nf, cudaStream_t s);
    // the same with a dense float32 array
    static cudaError_t pack32(const float* dense, R* X, const Coef<R>& C, int nf, cudaStream_t s);
    static cudaError_t unpack32(const R* X, float* dense, const Coef<R>& C, int nf, cudaStream_t s);
    // planes [k0, k1) of a dense float64 / float32 [nf][nz][ny][nx] array into
    // the pitched state, their CFL bound reduced into dt slot `slot` (as dt)
    static cudaError_t pack_dt(const double* dense, R* X, const R* zt, const Coef<R>& C, DevCtl* ctl, int slot,
                               int k0, int k1, cudaStream_t s);
    static cudaError_t pack_dt32(const float* dense, R* X, const R* zt, const Coef<R>& C, DevCtl* ctl, int slot,
                                 int k0, int k1, cudaStream_t s);
};

// FP32 sweeps with two columns per lane (nx even); defined in kernels_f32.cu.
// seg_rows > 0 sets the rows per warp segment, 0 leaves it to the occupancy
// model (CM_SEG_ROWS in the environment overrides both)
cudaError_t launch_sweep_x2(int dir, const float* in, float* out, const float* zt, const Coef<float>& C,
                            const SweepCtl& sc, int seg_rows, cudaStream_t s);

// FP32 3D sweeps with two columns per lane (nx even, uniform z-grid);
// defined in kernels_f32.cu.  seg_rows as for launch_sweep_x2 (march rows)
cudaError_t launch_sweep3_x2(int dir, const float* in, float* out, const float* zt, const Coef<float>& C,
                             const SweepCtl& sc, int seg_rows, cudaStream_t s);

// one batched sweep over every box of a batch (kernels_f32.cu); nblocks from
// the work list; const_coefs: the boxes' coefficients were uploaded with
// set_batch_coefs (batches of at most kConstBoxes boxes); stretched: every
// box has a plane table (C.zp) and no work item spans more than kBatchSegMax
// rows; layout_exact: the layout-independent form of the sweeps
struct BatchLaunch;
constexpr int kConstBoxes = 256;
constexpr int kBatchSegMax = 128;
constexpr int kBatchSegMin = 6;  // shortest segment the batch autotuner tries (sizes the work lists)
cudaError_t launch_sweep_batch(int dir, const BatchLaunch& L, int nblocks, bool const_coefs, bool stretched,
                               bool layout_exact, cudaStream_t s);
// copy the coefficients of n <= kConstBoxes boxes to constant memory (kernels_f32.cu)
cudaError_t set_batch_coefs(const Coef<float>* C, int n, cudaStream_t s);

cudaError_t launch_diag_final(const double* scratch, const double* zt, const DiagFinal& F, DevCtl* ctl, cm_diag* rec,
                              cudaStream_t s);

extern template struct Launch<double>;
extern template struct Launch<float>;

}  // namespace cm
