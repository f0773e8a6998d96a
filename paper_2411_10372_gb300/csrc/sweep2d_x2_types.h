// sweep2d_x2_types.h -- launch geometry and argument blocks of the packed
// FP32 2D sweeps, shared by the kernels and the host code of the batch.
#pragma once
#include "cm_device.cuh"

namespace cm {

constexpr int kOutW2 = 60;  // output columns per warp strip (two columns per lane, one halo lane each side)

// ---- batched ensemble: many independent boxes in one launch per sweep -----
// Each warp takes one work item (box, strip, first row of its segment); the
// four warps of a block always belong to the same box, whose coefficients
// the block stages in shared memory.  Boxes step in lockstep (same sweep,
// same dt slot parity) but each has its own dt, time and state buffers.
struct BoxDesc {
    Coef<float> C;
    float* buf[2];  // ping-pong state buffers of the box
    DevCtl* ctl;    // dt slots, time, steps, status of the box
    int pad[2];
};

struct BatchWork {
    int box;
    int strip;
    int ks;        // first output row; >= nz for padding warps
    int seg_rows;
    int lead;      // the box's first block: does the per-step bookkeeping
    int pad[3];
};

struct BatchLaunch {
    const BoxDesc* boxes;
    const BatchWork* work;
    int cur;       // buffer holding each box's current state
    int slot;      // dt slot of this step
    int first, last;
    double Delta;  // > 0: fixed Delta for every box (autotuner runs); else each box's dt/2
};


}  // namespace cm
