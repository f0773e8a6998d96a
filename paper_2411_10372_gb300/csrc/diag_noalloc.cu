// diag_noalloc.cu -- cm_diag_noalloc: the diagnostics reduction without any
// allocation, for callers that must not allocate device memory.
//
// Who needs it: an in-situ analysis hook or a coupler that is handed a state
// by another application's time loop.  Such a host usually owns device
// memory through its own pool (often nearly all of HBM), and a cudaMalloc
// from inside its loop either fails once the pool has claimed the memory or
// stalls the host's other streams, because cudaMalloc/cudaFree can
// synchronise the device.  This entry point therefore uses only a
// fixed-size scratch region that lives in the library image itself.
//
// The scratch region is a file-scope __device__ array (kNoAllocWords
// doubles, ~2.8 MB): every GPU that loads libcm.so holds it until the
// process exits.  It contains the control block the reduction reports into,
// the z coordinate of each plane, the per-plane partial sums, the output
// record and, for a stretched z-grid, the FP64 per-plane metric table.
// Host code cannot use the array's name as a device address, so the address
// is looked up once per device with cudaGetSymbolAddress, with that device
// current, on the first call on that device.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>

#include <vector>

#include "../../include/cm.h"
#include "host_setup.h"
#include "kernels.h"

namespace cm {

int set_error(int code, const char* msg);

namespace {

constexpr int kNoAllocMaxNz = 16384;  // largest plane count the scratch holds
constexpr int kCtlWords = 8;          // DevCtl (40 bytes) rounded up
constexpr int kRecWords = 16;         // cm_diag (128 bytes)
constexpr int kZOff = kCtlWords + kRecWords;
constexpr int kPlanesOff = kZOff + kNoAllocMaxNz;
constexpr int kTableOff = kPlanesOff + kNoAllocMaxNz * kDiagQ;
constexpr int kTableWords = kNoAllocMaxNz * (int)(sizeof(Plane<double>) / sizeof(double));
constexpr int kNoAllocWords = kTableOff + kTableWords;
static_assert(sizeof(Plane<double>) % sizeof(double) == 0, "plane table entries must be whole words");
static_assert((kTableOff * sizeof(double)) % alignof(Plane<double>) == 0, "plane table misaligned");
static_assert(sizeof(DevCtl) <= kCtlWords * sizeof(double), "control block does not fit");
static_assert(sizeof(cm_diag) <= kRecWords * sizeof(double), "record does not fit");

// The scratch region: shared by every call on a device, it keeps what the
// last call left.  Each call rewrites the control block and the z table and
// every plane sum it reads, so nothing stale is used; two calls that overlap
// on the GPU (different streams, or host threads) race on it.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocWords];

constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {nullptr};

// z of plane k: nodes on both plates, z = k/(nz-1)
__global__ void fill_plane_z(double* z, int nz)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nz; k += gridDim.x * blockDim.x)
        z[k] = (double)k / (double)(nz - 1);
}

int scratch_on_current_device(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(CM_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return set_error(CM_EINVAL, "device index beyond the no-alloc table");
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            char msg[256];
            snprintf(msg, sizeof msg, "cudaGetSymbolAddress of the no-alloc scratch failed: %s", cudaGetErrorString(e));
            return set_error(CM_ECUDA, msg);
        }
        g_scratch_addr[dev] = (double*)p;
    }
    *out = g_scratch_addr[dev];
    return CM_OK;
}

template <class R>
Coef<R> layout_coef(const cm_grid& G, int pitch, int ny)
{
    Coef<R> C;
    std::memset(&C, 0, sizeof C);
    C.nx = G.nx;
    C.ny = ny;
    C.nz = G.nz;
    C.pitch = pitch;
    C.fstride = (long long)G.nz * ny * pitch;
    C.ndim = G.ndim;
    return C;
}

}  // namespace
}  // namespace cm

using namespace cm;

extern "C" int cm_diag_noalloc(const void* state, int precision, const cm_grid* grid, int pitch, double Ra,
                               double Pr, double gamma, const cm_params* params, double t, double dt,
                               long long step, void* stream, cm_diag* out)
{
    if (!state || !grid || !params || !out) return set_error(CM_EINVAL, "cm_diag_noalloc: NULL argument");
    if (grid->ndim != 2 && grid->ndim != 3) return set_error(CM_EINVAL, "cm_diag_noalloc: ndim must be 2 or 3");
    const int ny = grid->ndim == 3 ? grid->ny : 1;
    if (grid->nx < 1 || ny < 1 || grid->nz < 5) return set_error(CM_EINVAL, "cm_diag_noalloc: bad grid");
    if (grid->nz > kNoAllocMaxNz) {
        char msg[160];
        snprintf(msg, sizeof msg, "cm_diag_noalloc: nz = %d exceeds the no-alloc maximum of %d planes", grid->nz,
                 kNoAllocMaxNz);
        return set_error(CM_EINVAL, msg);
    }
    if (pitch < grid->nx) return set_error(CM_EINVAL, "cm_diag_noalloc: pitch < nx");
    if (precision != CM_FP64 && precision != CM_FP32)
        return set_error(CM_EINVAL, "cm_diag_noalloc: precision must be CM_FP64 or CM_FP32");
    if (!(Ra > 0) || !(Pr > 0) || !(gamma > 1) || !(params->eps > 0) || !(params->D > 0))
        return set_error(CM_EINVAL, "cm_diag_noalloc: need Ra, Pr, eps, D > 0 and gamma > 1");
    // stretched z-grid: the planes and their FP64 metric, built on the host
    // (host memory only) and copied into the scratch array below
    const bool st = stretched(*grid);
    std::vector<double> zplanes;
    std::vector<Plane<double>> table;
    if (st) {
        const char* why = "";
        if (!make_planes(*grid, zplanes, &why)) {
            char msg[160];
            snprintf(msg, sizeof msg, "cm_diag_noalloc: %s", why);
            return set_error(CM_EINVAL, msg);
        }
        plane_table(zplanes, table);
    }

    double* base = nullptr;
    int rc = scratch_on_current_device(&base);
    if (rc) return rc;
    DevCtl* ctl = reinterpret_cast<DevCtl*>(base);
    cm_diag* rec = reinterpret_cast<cm_diag*>(base + kCtlWords);
    double* zt = base + kZOff;
    double* planes = base + kPlanesOff;
    Plane<double>* ztab = reinterpret_cast<Plane<double>*>(base + kTableOff);
    cudaStream_t s = (cudaStream_t)stream;

    // control block of this call: status cleared, time, steps, dt in slot 0
    DevCtl h;
    std::memset(&h, 0, sizeof h);
    h.t = t;
    h.steps = (double)step;
    std::memcpy(&h.dt_slot[0], &dt, sizeof dt);
    cudaError_t e = cudaMemcpyAsync(ctl, &h, sizeof h, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && st) {
        e = cudaMemcpyAsync(zt, zplanes.data(), grid->nz * sizeof(double), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ztab, table.data(), grid->nz * sizeof(Plane<double>), cudaMemcpyHostToDevice, s);
    } else if (e == cudaSuccess) {
        fill_plane_z<<<(grid->nz + 255) / 256, 256, 0, s>>>(zt, grid->nz);
        e = cudaGetLastError();
    }
    const double a = (gamma - 1.0) / (gamma * params->eps * params->D);
    DiagArgs A;
    A.zt = zt;
    A.a = a;
    A.b = gamma * params->eps * params->D;
    A.g = params->gravity / params->eps;
    A.D = params->D;
    A.cs2 = gamma * a;
    if (e == cudaSuccess)
        e = precision == CM_FP64
                ? Launch<double>::diag_planes((const double*)state, layout_coef<double>(*grid, pitch, ny), A, planes, ctl, s)
                : Launch<float>::diag_planes((const float*)state, layout_coef<float>(*grid, pitch, ny), A, planes, ctl, s);
    DiagFinal F{};
    F.Ra = Ra;
    F.Pr = Pr;
    F.eps = params->eps;
    F.D = params->D;
    F.cfl = 1.0;       // the record's dt is the caller's dt, read from slot 0
    F.dt_fixed = 0.0;
    F.cells = (double)grid->nx * ny;
    F.nz = grid->nz;
    F.slot = 0;
    F.zp = st ? ztab : nullptr;
    if (e == cudaSuccess) e = launch_diag_final(planes, zt, F, ctl, rec, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, rec, sizeof(cm_diag), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_error(CM_ECUDA, cudaGetErrorString(e));
    if (out->status != CM_OK) return set_error(CM_ENAN, "cm_diag_noalloc: non-finite value in the state");
    return CM_OK;
}
