// adjoint.h -- reverse mode of the 2D FP64 sweeps (Sec. 3.1) and of the plate
// Nusselt number (Eq. mean_Nu), for gradients of a time average of Nu_bar.
#pragma once
#include <cuda_runtime.h>
#include "cm_device.cuh"

namespace cm {

// device work arrays of the vector-Jacobian products of one sweep, sized for
// one pitched 2D FP64 state (fstride elements per field)
struct AdjWork {
    double* base;
    long long fs;
    int nblocks;
    double *U0, *U1, *T, *P, *A;   // primitives of X and |u_al| + c
    double *F;                     // F^n, 4 fields
    double *XP;                    // X^P, 4 fields
    double *UP0, *UP1, *TP, *PP;   // primitives of X^P
    double *XPB, *FPB, *FB;        // adjoints of X^P, F^P, F^n (4 fields each)
    double *UB;                    // direct adjoints of u_x, u_z, T at a node (3 fields)
    double *DA;                    // adjoints of the derivatives along the sweep: u_al, u_across, T
    double *DC;                    // adjoints of the derivatives across: u_al, u_across
    double *AB;                    // adjoint of |u_al| + c
    double *DVm, *DV0, *DVp, *DVA; // per TVD interface: adjoints of its three differences and two wave speeds
    double *part;                  // per-block partial sums of dJ/dmu and dJ/dK, 2 x nblocks x 2
    int frozen_phi;                // 1: no derivative through the limiter's ratios (phi' = 0)
};

// allocate / free the work arrays for grid C (nz planes of pitch C.pitch)
cudaError_t adj_work_create(AdjWork* w, const Coef<double>& C);
void adj_work_free(AdjWork* w);

// Xbar = (dY/dX)^T Ybar for Y = L_dir(Delta) X (dir 0 = x, 2 = z), all
// pitched 4-field FP64 states; acc[0] += <Ybar, dY/dmu>, acc[1] += <Ybar, dY/dK>
// (device).  Xbar must not alias X or Ybar.
cudaError_t adj_sweep_vjp(AdjWork* w, int dir, double Delta, const double* X, const double* Ybar, double* Xbar,
                          const double* zt, const Coef<double>& C, double* acc, cudaStream_t s);

// sums over x of T on planes kq[0..nq-1] of state X into out[0..nq-1]
cudaError_t adj_plane_T(const double* X, const double* zt, const Coef<double>& C, const int* kq, int nq, double* out,
                        cudaStream_t s);

// Xbar += dJ/dX for J = sum_q wq[q] * (sum over x of T on plane kq[q])
cudaError_t adj_seed_T(double* Xbar, const double* X, const double* zt, const Coef<double>& C, const int* kq,
                       const double* wq, int nq, cudaStream_t s);

// out[0] = the dt the next step will use (CFL from the slot, or dt_fixed)
cudaError_t adj_record_dt(const DevCtl* ctl, int slot, double cfl, double dt_fixed, double* out, cudaStream_t s);

// gT[node] = dJ/dT at fixed pressure and velocity on interior planes (0 on
// the plates), from Xbar = dJ/dX and the state X; dense [nz][nx] output
cudaError_t adj_grad_T(const double* X, const double* Xbar, const double* zt, const Coef<double>& C, double* gT,
                       cudaStream_t s);

}  // namespace cm
