// cm_api.cu -- the C ABI of include/cm.h: context, stepping driver,
// diagnostics ring, host transfers, checkpoints.
//
// A step (Sec. 3.1, Eq. time_step) is 4 sweep launches in 2D (z, x, z, x).
// The dt of a step is produced on the device by the previous step's last
// sweep (an FP64 atomic min of h/(|u|+c) over the new state into one of two
// slots) and read by the next step's sweeps, so the host never waits on it.
#include <cuda.h>  // driver API types only: the one driver call is fetched through the runtime
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <type_traits>
#include <vector>

#include "../../include/cm.h"
#include "adjoint.h"
#include "host_setup.h"
#include "kernels.h"

using namespace cm;

namespace {

constexpr int kUpChunks = 4;  // most plane chunks of a copied host upload

// state of the adjoint (cm_adj_forward / cm_adj_backward)
struct AdjCtx {
    int nsteps = 0, K = 0, win = 0;
    std::vector<double> dts;        // dt of each forward step (host)
    std::vector<double> replay;     // dts the next forward of replay.size() steps takes (cm_adj_set_dts)
    std::vector<double> plane_sums; // sum over x of T on planes 0, 1, 2, K, K-1, K-2 per window step
    char* ckpt = nullptr;           // device: state at steps 0, K, 2K, ... (K = 0: every sweep input)
    double* dts_d = nullptr;
    double* planes_d = nullptr;
    double J = 0.0;
};

struct Ctx {
    cm_grid grid;
    cm_params prm;
    double Ra, Pr, gamma;
    int nf, ny, pitch, prec;
    long long fstride;          // elements between fields
    size_t elem;                // bytes per element
    size_t buf_bytes;           // bytes of one state buffer
    void* buf[2];
    bool own_buf;
    int cur;                    // buffer holding the current state
    void* zt_r;                 // z table in the state precision
    double* zt_d;               // z table, FP64
    void* zp_r;                 // stretched z-grid: per-plane metric in the state precision (else NULL)
    Plane<double>* zp_d;        // the same in FP64 (diagnostics), else NULL
    double* zplanes;            // host copy of the nz plane heights
    unsigned long long zhash;   // FNV-1a of the plane heights of a stretched grid, 0 if uniform
    double* Tc_d;
    double* pc_d;
    DevCtl* ctl;
    double* scratch;            // per-plane diagnostics sums (nz * kDiagQ)
    double* ext_scratch;        // extended diagnostics: per-plane sums (nz * 16), allocated on first use
    double* ext_prims;          // extended diagnostics: FP64 rho, u, T of every node (5 x nodes), first use
    unsigned long long* ext_hist; // histogram counts (kExtMaxBins), allocated on first use
    double* dense;              // dense FP64 staging for host transfers (lazy)
    cudaStream_t copy_stream;   // host uploads: chunk copies (lazy, with dense)
    cudaEvent_t up_ev[kUpChunks + 1];  // chunk q arrived (q < kUpChunks); compute stream ready (last)
    cm_diag* ring;
    int ring_cap, ring_head, ring_count;
    cudaStream_t stream;
    long long step;
    long long launches;
    int seg[3];                 // rows per segment of the FP32 sweeps by direction x, y, z (0 = model)
    Coef<double> cd;
    Coef<float> cf;
    double a, b, g, cs2;
    AdjCtx* adj;
};

Ctx* g_ctx = nullptr;
char g_err[512] = "no error";

int fail(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(CM_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

#define NEED_CTX() \
    do { if (!g_ctx) return fail(CM_ENOTINIT, "no context: call cm_init first"); } while (0)

template <class R>
void fill_coef(Coef<R>& C, const Ctx& c)
{
    Closure K(c.gamma, c.prm);
    cm::fill_coef(C, c.grid, c.ny, c.pitch, c.fstride, c.Ra, c.Pr, K, c.prm);
}

void free_ctx(Ctx* c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    if (c->own_buf && c->buf[0]) cudaFree(c->buf[0]);
    cudaFree(c->zt_r);
    cudaFree(c->zt_d);
    if (c->zp_r != (void*)c->zp_d) cudaFree(c->zp_r);
    cudaFree(c->zp_d);
    std::free(c->zplanes);
    cudaFree(c->Tc_d);
    cudaFree(c->pc_d);
    cudaFree(c->ctl);
    cudaFree(c->scratch);
    cudaFree(c->ext_scratch);
    cudaFree(c->ext_prims);
    cudaFree(c->ext_hist);
    cudaFree(c->dense);
    for (cudaEvent_t& e : c->up_ev)
        if (e) cudaEventDestroy(e);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    cudaFree(c->ring);
    if (c->adj) {
        cudaFree(c->adj->ckpt);
        cudaFree(c->adj->dts_d);
        cudaFree(c->adj->planes_d);
        delete c->adj;
    }
    delete c;
}

int check_grid(const cm_grid* G)
{
    if (!G) return fail(CM_EINVAL, "grid is NULL");
    if (G->ndim != 2 && G->ndim != 3) return fail(CM_EINVAL, "ndim = %d: must be 2 or 3", G->ndim);
    if (G->nx < 4 || G->nz < 5) return fail(CM_EINVAL, "grid too small: nx >= 4 and nz >= 5 needed (got %d, %d)", G->nx, G->nz);
    if (G->ndim == 3 && G->ny < 4) return fail(CM_EINVAL, "grid too small: ny >= 4 needed in 3D (got %d)", G->ny);
    const long long ny = G->ndim == 3 ? G->ny : 1;
    if ((long long)G->nx * ny * G->nz > (1LL << 31)) return fail(CM_EINVAL, "grid too large");
    if (!(G->aspect > 0)) return fail(CM_EINVAL, "aspect must be > 0");
    return CM_OK;
}


// queue one sweep on the current buffer and swap buffers
int sweep(Ctx* c, int dir, const SweepCtl& sc)
{
    cudaError_t e;
    if (c->prec == CM_FP64)
        e = Launch<double>::sweep(dir, (const double*)c->buf[c->cur], (double*)c->buf[c->cur ^ 1],
                                  (const double*)c->zt_r, c->cd, sc, 0, c->stream);
    else
        e = Launch<float>::sweep(dir, (const float*)c->buf[c->cur], (float*)c->buf[c->cur ^ 1],
                                 (const float*)c->zt_r, c->cf, sc, c->seg[dir], c->stream);
    if (e != cudaSuccess) return fail(CM_ECUDA, "sweep launch: %s", cudaGetErrorString(e));
    c->launches++;
    c->cur ^= 1;
    return CM_OK;
}

int recompute_dt(Ctx* c, int slot)
{
    unsigned long long inf = 0x7FF0000000000000ULL;
    CK(cudaMemcpyAsync(&c->ctl->dt_slot[slot], &inf, sizeof inf, cudaMemcpyHostToDevice, c->stream));
    cudaError_t e = c->prec == CM_FP64
        ? Launch<double>::dt((const double*)c->buf[c->cur], (const double*)c->zt_r, c->cd, c->ctl, slot, c->stream)
        : Launch<float>::dt((const float*)c->buf[c->cur], (const float*)c->zt_r, c->cf, c->ctl, slot, c->stream);
    if (e != cudaSuccess) return fail(CM_ECUDA, "dt launch: %s", cudaGetErrorString(e));
    c->launches++;
    return CM_OK;
}

// queue one diagnostics record of the current state into dst (device)
int sample_into(Ctx* c, cm_diag* dst)
{
    DiagArgs A;
    A.zt = c->zt_d;
    A.a = c->a;
    A.b = c->b;
    A.g = c->g;
    A.D = c->prm.D;
    A.cs2 = c->cs2;
    cudaError_t e = c->prec == CM_FP64
        ? Launch<double>::diag_planes((const double*)c->buf[c->cur], c->cd, A, c->scratch, c->ctl, c->stream)
        : Launch<float>::diag_planes((const float*)c->buf[c->cur], c->cf, A, c->scratch, c->ctl, c->stream);
    if (e != cudaSuccess) return fail(CM_ECUDA, "diagnostics launch: %s", cudaGetErrorString(e));
    DiagFinal F{};
    F.Ra = c->Ra;
    F.Pr = c->Pr;
    F.eps = c->prm.eps;
    F.D = c->prm.D;
    F.cfl = c->prm.cfl;
    F.dt_fixed = c->prm.dt_fixed;
    F.cells = (double)c->grid.nx * c->ny;
    F.nz = c->grid.nz;
    F.slot = (int)(c->step & 1);
    F.zp = c->zp_d;
    e = launch_diag_final(c->scratch, c->zt_d, F, c->ctl, dst, c->stream);
    if (e != cudaSuccess) return fail(CM_ECUDA, "diagnostics launch: %s", cudaGetErrorString(e));
    c->launches += 2;
    return CM_OK;
}

// queue a sample into the ring (a full ring drops its oldest sample)
int sample(Ctx* c)
{
    if (c->ring_count == c->ring_cap) {
        c->ring_head = (c->ring_head + 1) % c->ring_cap;
        c->ring_count--;
    }
    const int rc = sample_into(c, c->ring + (c->ring_head + c->ring_count) % c->ring_cap);
    if (!rc) c->ring_count++;
    return rc;
}

// the record of the final state of cm_run_host / cm_run_host_f32: its own
// device slot after the ring, so queued samples stay untouched
int sample_final(Ctx* c, cm_diag* host_out)
{
    cm_diag* dst = c->ring + c->ring_cap;
    int rc = sample_into(c, dst);
    if (rc) return rc;
    CK(cudaMemcpyAsync(host_out, dst, sizeof(cm_diag), cudaMemcpyDeviceToHost, c->stream));
    return CM_OK;
}

// the staging array of host transfers and the copy stream and events of
// chunked uploads, each created on first use (a failed call leaves the
// others in place and the next call retries the missing ones)
int ensure_dense(Ctx* c)
{
    if (!c->dense) {
        size_t n = (size_t)c->nf * c->grid.nz * c->ny * c->grid.nx;
        if (cudaMalloc(&c->dense, n * sizeof(double)) != cudaSuccess) {
            c->dense = nullptr;
            cudaGetLastError();
            return fail(CM_ENOMEM, "cudaMalloc of %zu bytes (host transfer staging) failed", n * sizeof(double));
        }
    }
    bool ok = true;
    if (!c->copy_stream && cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
        c->copy_stream = nullptr;
        ok = false;
    }
    for (cudaEvent_t& e : c->up_ev)
        if (ok && !e && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            e = nullptr;
            ok = false;
        }
    if (!ok) {
        cudaGetLastError();
        return fail(CM_ECUDA, "creation of the upload stream and events failed");
    }
    return CM_OK;
}

size_t dense_count(const Ctx* c) { return (size_t)c->nf * c->grid.nz * c->ny * c->grid.nx; }

// Device address of a pinned host array of `count` elements that the GPU can
// read in place: both ends pinned and inside ONE pinned allocation (the same
// CUDA buffer ID, so every page between them is pinned and mapped), their
// device addresses as far apart as their host addresses; else NULL, and the
// caller copies.  Two separately pinned ranges (adjacent or with pageable
// pages between them) have different buffer IDs and take the copy.
using PtrAttrFn = CUresult (*)(void*, CUpointer_attribute, CUdeviceptr);

PtrAttrFn ptr_attr_fn()
{
    static PtrAttrFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PtrAttrFn)f;
        else
            cudaGetLastError();
    }
    return fn;
}

bool one_pinned_buffer(const void* a, const void* b)
{
    PtrAttrFn fn = ptr_attr_fn();
    unsigned long long ia = 0, ib = 0;
    if (!fn || fn(&ia, CU_POINTER_ATTRIBUTE_BUFFER_ID, (CUdeviceptr)a) != CUDA_SUCCESS ||
        fn(&ib, CU_POINTER_ATTRIBUTE_BUFFER_ID, (CUdeviceptr)b) != CUDA_SUCCESS)
        return false;
    return ia != 0 && ia == ib;
}

// Kind of a host array of count elements: 1 = inside one pinned allocation
// (*view = its device-mapped address), 0 = pageable at both ends (copied
// through the staging array), -1 = pinned at an end but not one allocation
// (several registrations, or pinned and pageable pages): CUDA's copies
// reject such a range, so the entry points refuse it up front.
template <class S>
int host_kind(const S* host, size_t count, const S** view)
{
    cudaPointerAttributes a0, a1;
    if (cudaPointerGetAttributes(&a0, host) != cudaSuccess ||
        cudaPointerGetAttributes(&a1, host + (count - 1)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const bool p0 = a0.type == cudaMemoryTypeHost, p1 = a1.type == cudaMemoryTypeHost;
    if (!p0 && !p1) return 0;
    if (!p0 || !p1 || !a0.devicePointer || !a1.devicePointer) return -1;
    if ((const char*)a1.devicePointer - (const char*)a0.devicePointer != (ptrdiff_t)((count - 1) * sizeof(S)))
        return -1;
    if (!one_pinned_buffer(host, host + (count - 1))) return -1;
    if (view) *view = (const S*)a0.devicePointer;
    return 1;
}

int refuse_split_pinned(const char* what)
{
    return fail(CM_EINVAL, "%s spans several pinned allocations (or pinned and pageable memory): pass one pinned "
                "allocation or pageable memory", what);
}

// packs planes [k0, k1) of the dense array src (device-readable) into the
// current buffer, their CFL bound reduced into dt slot `slot`
template <class S>
int pack_planes(Ctx* c, const S* src, int slot, int k0, int k1)
{
    cudaError_t e;
    if constexpr (std::is_same<S, double>::value)
        e = c->prec == CM_FP64
            ? Launch<double>::pack_dt(src, (double*)c->buf[c->cur], (const double*)c->zt_r, c->cd, c->ctl, slot, k0, k1, c->stream)
            : Launch<float>::pack_dt(src, (float*)c->buf[c->cur], (const float*)c->zt_r, c->cf, c->ctl, slot, k0, k1, c->stream);
    else
        e = Launch<float>::pack_dt32(src, (float*)c->buf[c->cur], (const float*)c->zt_r, c->cf, c->ctl, slot, k0, k1, c->stream);
    if (e != cudaSuccess) return fail(CM_ECUDA, "pack launch: %s", cudaGetErrorString(e));
    c->launches++;
    return CM_OK;
}

// Upload of a dense host state (S = double or float) into the current
// buffer, with the step's dt recomputed by the same kernel (pack_dt).  A
// pinned host array is read in place over the host link by that one kernel.
// Other host memory is copied in up to kUpChunks plane chunks (one 2D copy
// of all fields per chunk) on the copy stream into the staging array, and
// each chunk is packed on the compute stream as soon as it has arrived, so
// the packing of one chunk runs under the copy of the next.
template <class S>
int upload_host(Ctx* c, const S* host)
{
    const int slot = (int)(c->step & 1), nz = c->grid.nz;
    const size_t plane = (size_t)c->ny * c->grid.nx, field = plane * nz;
    const S* view = nullptr;
    const int kind = host_kind(host, field * c->nf, &view);
    if (kind < 0) return refuse_split_pinned("the host state");
    const unsigned long long inf = 0x7FF0000000000000ULL;
    CK(cudaMemcpyAsync(&c->ctl->dt_slot[slot], &inf, sizeof inf, cudaMemcpyHostToDevice, c->stream));
    if (kind > 0) return pack_planes(c, view, slot, 0, nz);
    int rc = ensure_dense(c);
    if (rc) return rc;
    S* staging = (S*)c->dense;  // sized for float64, so it holds either type
    const size_t bytes = field * c->nf * sizeof(S), fbytes = field * sizeof(S);
    const int nch = (int)std::min<size_t>({(size_t)kUpChunks, (size_t)nz, std::max<size_t>(1, bytes >> 23)});
    // the staging array may still be read by earlier work on the compute stream
    CK(cudaEventRecord(c->up_ev[kUpChunks], c->stream));
    CK(cudaStreamWaitEvent(c->copy_stream, c->up_ev[kUpChunks], 0));
    for (int q = 0; q < nch; ++q) {
        const int k0 = (int)((long long)nz * q / nch), k1 = (int)((long long)nz * (q + 1) / nch);
        const size_t off = k0 * plane, w = (k1 - k0) * plane * sizeof(S);
        if (fbytes <= ((size_t)1 << 30)) {
            CK(cudaMemcpy2DAsync(staging + off, fbytes, host + off, fbytes, w, c->nf, cudaMemcpyHostToDevice,
                                 c->copy_stream));
        } else {
            for (int f = 0; f < c->nf; ++f)
                CK(cudaMemcpyAsync(staging + f * field + off, host + f * field + off, w, cudaMemcpyHostToDevice,
                                   c->copy_stream));
        }
        CK(cudaEventRecord(c->up_ev[q], c->copy_stream));
        CK(cudaStreamWaitEvent(c->stream, c->up_ev[q], 0));
        if ((rc = pack_planes(c, (const S*)staging, slot, k0, k1))) return rc;
    }
    return CM_OK;
}

int upload(Ctx* c, const double* host) { return upload_host(c, host); }

// An entry point that failed after queuing work on the caller's host memory
// (an in-place read of a pinned state, copies into or out of it) waits for
// that work before it returns, so that no kernel or copy still touches the
// caller's buffers afterwards.  Returns rc.
int drain_on_error(Ctx* c, int rc)
{
    if (rc != CM_OK) {
        cudaStreamSynchronize(c->stream);
        if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
    }
    return rc;
}

int download(Ctx* c, double* host)
{
    if (host_kind<double>(host, dense_count(c), nullptr) < 0) return refuse_split_pinned("the host output");
    int rc = ensure_dense(c);
    if (rc) return rc;
    cudaError_t e = c->prec == CM_FP64
        ? Launch<double>::unpack((const double*)c->buf[c->cur], c->dense, c->cd, c->nf, c->stream)
        : Launch<float>::unpack((const float*)c->buf[c->cur], c->dense, c->cf, c->nf, c->stream);
    if (e != cudaSuccess) return fail(CM_ECUDA, "unpack launch: %s", cudaGetErrorString(e));
    c->launches++;
    CK(cudaMemcpyAsync(host, c->dense, dense_count(c) * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return CM_OK;
}

// sweeps per step: L_x L_z L_x L_z in 2D, L_x L_y L_z L_x L_y L_z in 3D
// (applied right to left)
int sweeps_per_step(const Ctx* c) { return c->grid.ndim == 3 ? 6 : 4; }

// queue n steps; with ev != NULL and per_sweep (S+1 events per step, S sweeps
// per step), record ev[(S+1)s+q] before sweep q of step s and ev[(S+1)s+S]
// after its last sweep; with ev != NULL and !per_sweep, ev[2s] before the
// step and ev[2s+1] after it; with flush, overwrite flush_bytes of it before
// each step, outside the brackets
int queue_steps(Ctx* c, int n, cudaEvent_t* ev = nullptr, void* flush = nullptr, size_t flush_bytes = 0,
                bool per_sweep = true)
{
    // sweep directions in the order applied (Eq. time_step, rightmost first;
    // CM_SPLIT_SYMMETRIC: the palindrome); the last is always L_x, which
    // reduces the next dt
    static const int printed2[4] = {2, 0, 2, 0}, symmetric2[4] = {0, 2, 2, 0};
    static const int printed3[6] = {2, 1, 0, 2, 1, 0}, symmetric3[6] = {0, 1, 2, 2, 1, 0};
    const int S = sweeps_per_step(c);
    const bool sym = c->prm.split == CM_SPLIT_SYMMETRIC;
    const int* order = S == 6 ? (sym ? symmetric3 : printed3) : (sym ? symmetric2 : printed2);
    for (int s = 0; s < n; ++s) {
        const int slot = (int)(c->step & 1);
        SweepCtl sc;
        sc.ctl = c->ctl;
        sc.slot_in = slot;
        sc.Delta = 0.0;
        if (flush) CK(cudaMemsetAsync(flush, s & 0xff, flush_bytes, c->stream));
        for (int q = 0; q < S; ++q) {
            sc.first = (q == 0);
            sc.last = (q == S - 1);
            if (ev && (per_sweep || q == 0)) CK(cudaEventRecord(ev[per_sweep ? (S + 1) * s + q : 2 * s], c->stream));
            int rc = sweep(c, order[q], sc);
            if (rc) return rc;
        }
        if (ev) CK(cudaEventRecord(ev[per_sweep ? (S + 1) * s + S : 2 * s + 1], c->stream));
        c->step++;
        if (c->prm.diag_every > 0 && c->step % c->prm.diag_every == 0) {
            int rc = sample(c);
            if (rc) return rc;
        }
    }
    return CM_OK;
}

unsigned long long fnv1a(const void* p, size_t n, unsigned long long h = 1469598103934665603ULL)
{
    const unsigned char* b = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) { h ^= b[i]; h *= 1099511628211ULL; }
    return h;
}

unsigned long long param_hash(const Ctx* c)
{
    double v[12] = {c->Ra, c->Pr, c->gamma, c->prm.eps, c->prm.D, c->prm.cfl, c->prm.dt_fixed,
                    c->prm.gravity, c->prm.t_bot, c->prm.t_top, c->prm.stokes, (double)c->prm.tvd_form};
    const unsigned long long h = fnv1a(v, sizeof v);
    if (!c->zhash) return h;  // uniform planes: the hash of earlier checkpoints
    const unsigned long long both[2] = {h, c->zhash};
    return fnv1a(both, sizeof both);
}

struct CkptHeader {
    char magic[8];
    int version, ndim, nx, ny, nz, precision;
    long long step;
    double t;
    unsigned long long hash;
};

}  // namespace

extern "C" {

int cm_default_params(cm_params* p)
{
    if (!p) return fail(CM_EINVAL, "params is NULL");
    std::memset(p, 0, sizeof *p);
    p->eps = 0.1;
    p->D = 0.5;
    p->cfl = 0.5;
    p->dt_fixed = 0.0;
    p->gravity = 1.0;
    p->t_bot = 1.0;
    p->t_top = 1.0 - p->eps - p->D;
    p->pert_amp = 1e-3;
    p->stokes = -2.0 / 3.0;
    p->seed = 12345ULL;
    p->precision = CM_FP64;
    p->tvd_form = CM_TVD_DAVIS;
    p->diag_every = 0;
    p->diag_capacity = 1024;
    p->stream = nullptr;
    p->state_buf = nullptr;
    p->adj_limiter = CM_ADJ_PHI_EXACT;
    return CM_OK;
}

int cm_state_bytes(const cm_grid* grid, int precision, unsigned long long* bytes)
{
    int rc = check_grid(grid);
    if (rc) return rc;
    if (precision != CM_FP64 && precision != CM_FP32) return fail(CM_EINVAL, "precision must be CM_FP64 or CM_FP32");
    if (!bytes) return fail(CM_EINVAL, "bytes is NULL");
    const int nf = grid->ndim == 3 ? 5 : 4;
    const int ny = grid->ndim == 3 ? grid->ny : 1;
    const size_t elem = precision == CM_FP64 ? 8 : 4;
    *bytes = 2ULL * nf * (unsigned long long)grid->nz * ny * pitch_of(grid->nx, precision) * elem;
    return CM_OK;
}

// Segment length of the FP32 sweeps (rows per warp segment of the march).
// Their time at a grid size depends on it in ways no simple occupancy model
// captures (measured at 4096 x 1024: 29 rows 0.140 ms per step, 32 rows 0.160,
// 28 rows 0.161, 24 rows 0.150; at 512 x 512 x 128: 64 rows 4.97 ms, the model's
// 128 rows 5.16 ms), so each direction is timed at a fixed list of lengths and
// the fastest kept.  The sweeps read the current state and write the spare
// buffer, so the state, dt and time are untouched; the choice only changes
// how the work is split (the result only at FP32 rounding level).
int tune_segments(Ctx* c)
{
    const bool d2 = c->grid.ndim == 2;
    if (c->prec != CM_FP32 || (d2 && (c->grid.nx & 1)) || getenv("CM_SEG_ROWS")) return CM_OK;
    static const int cand2[] = {12, 16, 18, 20, 21, 22, 24, 26, 28, 29, 30, 31, 32, 36, 40, 48, 64, 96, 128};
    static const int cand3[] = {32, 48, 64, 96, 128, 192, 256};
    const int* cand = d2 ? cand2 : cand3;
    const int ncand = d2 ? (int)(sizeof cand2 / sizeof cand2[0]) : (int)(sizeof cand3 / sizeof cand3[0]);
    const int reps = d2 ? 3 : 1;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    SweepCtl sc;
    std::memset(&sc, 0, sizeof sc);
    sc.ctl = c->ctl;
    sc.slot_in = (int)(c->step & 1);
    sc.Delta = 1e-9;
    const float* in = (const float*)c->buf[c->cur];
    float* spare = (float*)c->buf[c->cur ^ 1];
    int best_seg[3] = {0, 0, 0};
    cudaError_t e = cudaSuccess;
    for (int dir = 0; dir <= 2 && e == cudaSuccess; ++dir) {
        if (d2 && dir == 1) continue;
        const int nmarch = dir == 1 ? c->ny : c->grid.nz;
        float best = 1e30f;
        for (int q = 0; q < ncand && e == cudaSuccess; ++q) {
            const int seg = cand[q];
            if (seg > nmarch) break;
            float t_min = 1e30f;
            for (int rep = 0; rep < reps && e == cudaSuccess; ++rep) {
                e = Launch<float>::sweep(dir, in, spare, (const float*)c->zt_r, c->cf, sc, seg, c->stream);
                if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
                for (int k = 0; k < 4 && e == cudaSuccess; ++k)
                    e = Launch<float>::sweep(dir, in, spare, (const float*)c->zt_r, c->cf, sc, seg, c->stream);
                if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float t = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
                t_min = std::min(t_min, t);
                c->launches += 5;
            }
            if (t_min < best) {
                best = t_min;
                best_seg[dir] = seg;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return fail(CM_ECUDA, "segment tuning: %s", cudaGetErrorString(e));
    for (int d = 0; d < 3; ++d) c->seg[d] = best_seg[d];
    return CM_OK;
}

int cm_init(const cm_grid* grid, double Ra, double Pr, double gamma, const cm_params* params)
{
    int rc = check_grid(grid);
    if (rc) return rc;
    cm_params P;
    if (params) P = *params;
    else cm_default_params(&P);
    if (!(Ra > 0) || !(Pr > 0) || !(gamma > 1)) return fail(CM_EINVAL, "need Ra > 0, Pr > 0, gamma > 1");
    if (!(P.eps > 0) || !(P.D > 0)) return fail(CM_EINVAL, "need eps > 0 and D > 0");
    if (!(P.cfl > 0) || P.cfl > 1.0) return fail(CM_EINVAL, "cfl must be in (0, 1]");
    if (!(P.t_bot > 0) || !(P.t_top > 0)) return fail(CM_EINVAL, "plate temperatures must be > 0");
    if (P.precision != CM_FP64 && P.precision != CM_FP32) return fail(CM_EINVAL, "precision must be CM_FP64 or CM_FP32");
    if (P.tvd_form < 0 || P.tvd_form > 2) return fail(CM_EINVAL, "tvd_form must be 0, 1 or 2");
    if (P.adj_limiter != CM_ADJ_PHI_EXACT && P.adj_limiter != CM_ADJ_PHI_FROZEN)
        return fail(CM_EINVAL, "adj_limiter must be CM_ADJ_PHI_EXACT or CM_ADJ_PHI_FROZEN");
    if (P.layout_exact != 0 && P.layout_exact != 1) return fail(CM_EINVAL, "layout_exact must be 0 or 1");
    if (P.split != CM_SPLIT_PRINTED && P.split != CM_SPLIT_SYMMETRIC)
        return fail(CM_EINVAL, "split must be CM_SPLIT_PRINTED or CM_SPLIT_SYMMETRIC");
    if (P.diag_capacity < 1) P.diag_capacity = 1024;
    if (P.state_buf && ((uintptr_t)P.state_buf & 255)) return fail(CM_EINVAL, "state_buf must be 256-byte aligned");
    std::vector<double> planes;
    const char* why = "";
    if (!make_planes(*grid, planes, &why)) return fail(CM_EINVAL, "%s", why);
    const bool st = stretched(*grid);

    if (g_ctx) { free_ctx(g_ctx); g_ctx = nullptr; }
    Ctx* c = new Ctx();
    std::memset((void*)c, 0, sizeof *c);
    c->grid = *grid;
    c->grid.znodes = nullptr;  // caller memory: the planes are copied below
    c->prm = P;
    c->Ra = Ra;
    c->Pr = Pr;
    c->gamma = gamma;
    c->prec = P.precision;
    c->nf = grid->ndim == 3 ? 5 : 4;
    c->ny = grid->ndim == 3 ? grid->ny : 1;
    c->pitch = pitch_of(grid->nx, c->prec);
    c->elem = c->prec == CM_FP64 ? 8 : 4;
    c->fstride = (long long)grid->nz * c->ny * c->pitch;
    c->buf_bytes = (size_t)c->nf * c->fstride * c->elem;
    c->stream = (cudaStream_t)P.stream;
    c->ring_cap = P.diag_capacity;
    c->a = (gamma - 1.0) / (gamma * P.eps * P.D);
    c->b = gamma * P.eps * P.D;
    c->g = P.gravity / P.eps;
    c->cs2 = gamma * c->a;
    c->seg[0] = c->seg[1] = c->seg[2] = 0;  // occupancy model until tune_segments
    fill_coef(c->cd, *c);
    fill_coef(c->cf, *c);

    auto bail = [&](int code) { free_ctx(c); return code; };
    const int nz = grid->nz;
    if (P.state_buf) {
        c->buf[0] = P.state_buf;
        c->own_buf = false;
    } else {
        if (cudaMalloc(&c->buf[0], 2 * c->buf_bytes) != cudaSuccess) {
            cudaGetLastError();
            return bail(fail(CM_ENOMEM, "cudaMalloc of %zu bytes (state) failed", 2 * c->buf_bytes));
        }
        c->own_buf = true;
    }
    c->buf[1] = (char*)c->buf[0] + c->buf_bytes;
    if (cudaMalloc(&c->zt_r, nz * c->elem) != cudaSuccess || cudaMalloc(&c->zt_d, nz * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->Tc_d, nz * sizeof(double)) != cudaSuccess || cudaMalloc(&c->pc_d, nz * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->ctl, sizeof(DevCtl)) != cudaSuccess ||
        cudaMalloc(&c->scratch, (size_t)nz * kDiagQ * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->ring, (size_t)(c->ring_cap + 1) * sizeof(cm_diag)) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(CM_ENOMEM, "cudaMalloc of the work arrays failed"));
    }

    c->zplanes = (double*)std::malloc(nz * sizeof(double));
    if (!c->zplanes) return bail(fail(CM_ENOMEM, "host allocation of the plane table failed"));
    std::memcpy(c->zplanes, planes.data(), nz * sizeof(double));
    if (st) {
        // per-plane metric tables of the stretched grid (FP64 for the
        // diagnostics, the state precision for the sweeps)
        c->zhash = fnv1a(planes.data(), nz * sizeof(double)) | 1ULL;
        std::vector<Plane<double>> td;
        plane_table(planes, td);
        std::vector<Plane<float>> tf;
        plane_table(planes, tf);
        if (cudaMalloc(&c->zp_d, nz * sizeof(Plane<double>)) != cudaSuccess) {
            cudaGetLastError();
            return bail(fail(CM_ENOMEM, "cudaMalloc of the plane table failed"));
        }
        if (c->prec == CM_FP64) c->zp_r = c->zp_d;
        else if (cudaMalloc(&c->zp_r, nz * sizeof(Plane<float>)) != cudaSuccess) {
            cudaGetLastError();
            return bail(fail(CM_ENOMEM, "cudaMalloc of the plane table failed"));
        }
        if (cudaMemcpyAsync(c->zp_d, td.data(), nz * sizeof(Plane<double>), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
            (c->prec == CM_FP32 &&
             cudaMemcpyAsync(c->zp_r, tf.data(), nz * sizeof(Plane<float>), cudaMemcpyHostToDevice, c->stream) != cudaSuccess) ||
            cudaStreamSynchronize(c->stream) != cudaSuccess) {
            cudaGetLastError();
            return bail(fail(CM_ECUDA, "upload of the plane table failed"));
        }
        c->cd.zp = c->zp_d;
        c->cf.zp = (const Plane<float>*)c->zp_r;
    }

    // conduction / hydrostatic profile of constant K, FP64 on the host (nz values)
    const Profile prof(planes, P, Closure(gamma, P));
    const std::vector<double>& z = prof.z;
    const std::vector<double>& Tc = prof.Tc;
    const std::vector<double>& pc = prof.pc;
    const double rho_min = prof.rho_min;
    std::vector<float> zf(nz);
    for (int k = 0; k < nz; ++k) zf[k] = (float)z[k];
    cudaStream_t s = c->stream;
    if (cudaMemcpyAsync(c->zt_d, z.data(), nz * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(c->zt_r, c->prec == CM_FP64 ? (const void*)z.data() : (const void*)zf.data(), nz * c->elem,
                        cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(c->Tc_d, Tc.data(), nz * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(c->pc_d, pc.data(), nz * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(c->buf[0], 0, 2 * c->buf_bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(CM_ECUDA, "upload of the profile tables failed"));
    }
    DevCtl h;
    std::memset(&h, 0, sizeof h);
    h.dt_slot[0] = h.dt_slot[1] = 0x7FF0000000000000ULL;
    if (cudaMemcpyAsync(c->ctl, &h, sizeof h, cudaMemcpyHostToDevice, s) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(CM_ECUDA, "upload of the control block failed"));
    }
    InitArgs A;
    A.Tc = c->Tc_d;
    A.pc = c->pc_d;
    A.zt = c->zt_d;
    A.a = c->a;
    A.b = c->b;
    A.g = c->g;
    A.amp = P.pert_amp;
    A.seed = P.seed;
    cudaError_t e = c->prec == CM_FP64 ? Launch<double>::init((double*)c->buf[0], c->cd, A, s)
                                        : Launch<float>::init((float*)c->buf[0], c->cf, A, s);
    if (e != cudaSuccess) return bail(fail(CM_ECUDA, "init launch: %s", cudaGetErrorString(e)));
    c->launches = 1;
    c->cur = 0;
    c->step = 0;
    rc = recompute_dt(c, 0);
    if (rc) return bail(rc);
    // diffusion number of the explicit viscous / conduction terms at the first dt
    if (cudaMemcpyAsync(&h, c->ctl, sizeof h, cudaMemcpyDeviceToHost, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(CM_ECUDA, "init failed on the device: %s", cudaGetErrorString(cudaGetLastError())));
    }
    double hmin;
    std::memcpy(&hmin, &h.dt_slot[0], sizeof hmin);
    const double dt0 = P.dt_fixed > 0 ? P.dt_fixed : P.cfl * hmin;
    if (!(dt0 > 0) || !std::isfinite(dt0) || (h.status & 1)) return bail(fail(CM_ENAN, "non-finite initial state"));
    const double dnum = diffusion_number(*grid, planes, Ra, Pr, P, Closure(gamma, P), rho_min, dt0);
    if (dnum > 0.5)
        return bail(fail(CM_EUNSTABLE, "explicit diffusion number %.3g > 0.5 at dt = %.3g: refine dt (dt_fixed) or raise Ra", dnum, dt0));
    if ((rc = tune_segments(c))) return bail(rc);
    g_ctx = c;
    return CM_OK;
}

int cm_znodes(double* z)
{
    NEED_CTX();
    if (!z) return fail(CM_EINVAL, "z is NULL");
    std::memcpy(z, g_ctx->zplanes, g_ctx->grid.nz * sizeof(double));
    return CM_OK;
}

int cm_tuning(int* seg_z, int* seg_x)
{
    NEED_CTX();
    if (seg_z) *seg_z = g_ctx->seg[2];
    if (seg_x) *seg_x = g_ctx->seg[0];
    return CM_OK;
}

int cm_step(int n)
{
    NEED_CTX();
    if (n < 0) return fail(CM_EINVAL, "n must be >= 0");
    return queue_steps(g_ctx, n);
}

int cm_sample(void)
{
    NEED_CTX();
    return sample(g_ctx);
}

int cm_profiles(double* out)
{
    NEED_CTX();
    Ctx* c = g_ctx;
    if (!out) return fail(CM_EINVAL, "out is NULL");
    DiagArgs A;
    A.zt = c->zt_d;
    A.a = c->a;
    A.b = c->b;
    A.g = c->g;
    A.D = c->prm.D;
    A.cs2 = c->cs2;
    cudaError_t e = c->prec == CM_FP64
        ? Launch<double>::diag_planes((const double*)c->buf[c->cur], c->cd, A, c->scratch, c->ctl, c->stream)
        : Launch<float>::diag_planes((const float*)c->buf[c->cur], c->cf, A, c->scratch, c->ctl, c->stream);
    if (e != cudaSuccess) return fail(CM_ECUDA, "profiles launch: %s", cudaGetErrorString(e));
    c->launches++;
    const int nz = c->grid.nz;
    std::vector<double> sums((size_t)nz * kDiagQ);
    CK(cudaMemcpyAsync(sums.data(), c->scratch, sums.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const double cells = (double)c->grid.nx * c->ny;
    for (int k = 0; k < nz; ++k)
        for (int q = 0; q < kDiagQ; ++q)
            out[(size_t)k * kDiagQ + q] = q == kDiagQ - 1 ? sums[(size_t)k * kDiagQ + q] : sums[(size_t)k * kDiagQ + q] / cells;
    return CM_OK;
}

// extended diagnostics of the current state: per-plane sums (nz x 16, see
// ext_planes) and, with nbins > 0, the histogram of log10 K_e/I_e
int run_ext(Ctx* c, int nbins, double lo, double hi, std::vector<double>& sums, std::vector<unsigned long long>& hist)
{
    const int nz = c->grid.nz;
    if (!c->ext_scratch) {
        const size_t nodes = (size_t)c->grid.nx * c->ny * nz;
        if (cudaMalloc(&c->ext_scratch, (size_t)nz * 16 * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&c->ext_prims, 5 * nodes * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&c->ext_hist, kExtMaxBins * sizeof(unsigned long long)) != cudaSuccess) {
            cudaGetLastError();
            return fail(CM_ENOMEM, "cudaMalloc of the extended-diagnostics scratch failed");
        }
    }
    ExtArgs A;
    A.zt = c->zt_d;
    A.a = c->a;
    A.b = c->b;
    A.g = c->g;
    A.D = c->prm.D;
    A.mu = std::sqrt(c->Pr / c->Ra);
    A.stokes = c->prm.stokes;
    A.dx = c->grid.aspect / c->grid.nx;
    A.dy = c->grid.aspect / c->ny;
    A.nbins = nbins > 0 ? nbins : 1;
    A.lo = nbins > 0 ? lo : -16.0;
    A.bw = nbins > 0 ? (hi - lo) / nbins : 16.0;
    A.hist = c->ext_hist;
    CK(cudaMemsetAsync(c->ext_hist, 0, kExtMaxBins * sizeof(unsigned long long), c->stream));
    cudaError_t e = c->prec == CM_FP64
        ? Launch<double>::ext_planes((const double*)c->buf[c->cur], c->cd, A, c->ext_prims, c->ext_scratch, c->stream)
        : Launch<float>::ext_planes((const float*)c->buf[c->cur], c->cf, A, c->ext_prims, c->ext_scratch, c->stream);
    if (e != cudaSuccess) return fail(CM_ECUDA, "extended diagnostics launch: %s", cudaGetErrorString(e));
    c->launches++;
    sums.assign((size_t)nz * 16, 0.0);
    hist.assign(A.nbins, 0ULL);
    CK(cudaMemcpyAsync(sums.data(), c->ext_scratch, sums.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(hist.data(), c->ext_hist, hist.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return CM_OK;
}

int cm_ext_profiles(double* out)
{
    NEED_CTX();
    if (!out) return fail(CM_EINVAL, "out is NULL");
    Ctx* c = g_ctx;
    std::vector<double> sums;
    std::vector<unsigned long long> hist;
    int rc = run_ext(c, 0, 0.0, 0.0, sums, hist);
    if (rc) return rc;
    const double cells = (double)c->grid.nx * c->ny, D = c->prm.D;
    for (int k = 0; k < c->grid.nz; ++k) {
        const double* sk = &sums[(size_t)k * 16];
        const double z = c->zplanes[k];
        for (int q = 0; q < 6; ++q) out[(size_t)k * 9 + q] = sk[q] / cells;
        out[(size_t)k * 9 + 6] = sk[8] / cells - (1.0 - D * z);
        out[(size_t)k * 9 + 7] = sk[9] / cells - std::pow(1.0 - D * z, 1.0 / (c->gamma - 1.0));
        out[(size_t)k * 9 + 8] = std::sqrt(sk[10] / cells);
    }
    return CM_OK;
}

int cm_extended(cm_ext* out, long long* hist_out, int nbins, double log10_lo, double log10_hi)
{
    NEED_CTX();
    if (!out) return fail(CM_EINVAL, "out is NULL");
    if (hist_out && (nbins < 1 || nbins > kExtMaxBins || !(log10_hi > log10_lo)))
        return fail(CM_EINVAL, "need 1 <= nbins <= %d and log10_hi > log10_lo", kExtMaxBins);
    Ctx* c = g_ctx;
    std::vector<double> sums;
    std::vector<unsigned long long> hist;
    int rc = run_ext(c, hist_out ? nbins : 0, log10_lo, log10_hi, sums, hist);
    if (rc) return rc;
    const int nz = c->grid.nz, K = nz - 1;
    const double* z = c->zplanes;
    const bool st = c->zp_d != nullptr;
    const double cells = (double)c->grid.nx * c->ny;
    // trapezoid weights of the planes (cell widths on a stretched grid)
    auto wgt = [&](int k) {
        if (!st) return (k == 0 || k == K) ? 0.5 : 1.0;
        if (k == 0) return (z[1] - z[0]) / 2.0;
        if (k == K) return (z[K] - z[K - 1]) / 2.0;
        return ((z[k] - z[k - 1]) + (z[k + 1] - z[k])) / 2.0;
    };
    double s_conv = 0, s_m2 = 0, s_t2 = 0, wsum = 0, f[4] = {0, 0, 0, 0}, rmax = 0;
    std::vector<double> TA(nz);
    for (int k = 0; k < nz; ++k) {
        const double* sk = &sums[(size_t)k * 16];
        const double w = wgt(k);
        s_conv += w * sk[6] / cells;
        s_m2 += w * (sk[4] / cells);
        s_t2 += w * (sk[5] / cells);
        TA[k] = sk[8] / cells;
        rmax = std::fmax(rmax, sk[7]);
        if (k > 0 && k < K) {
            wsum += w;
            for (int q = 0; q < 4; ++q) f[q] += w * (sk[q] / cells);
        }
    }
    const double vol = st ? 1.0 : (double)(nz - 1);
    cm_ext r;
    r.rho_uz_sq = s_m2 / vol;
    r.Tsa_sq = s_t2 / vol;
    r.C = (s_conv / vol) / std::sqrt(r.rho_uz_sq * r.Tsa_sq);
    {
        // boundary layers: the plate tangent of <T_sa>_A against the bulk mean
        // of <T_sa>_A over 1/4 <= z <= 3/4 (trapezoid weights)
        const double D = c->prm.D;
        double sa[3], sb[3], tb = 0.0, tw = 0.0;
        for (int q = 0; q < 3; ++q) {
            sa[q] = TA[q] - (1.0 - D * z[q]);
            sb[q] = TA[K - q] - (1.0 - D * z[K - q]);
        }
        for (int k = 0; k <= K; ++k)
            if (z[k] >= 0.25 && z[k] <= 0.75) {
                const double wk = st ? wgt(k) : 1.0;
                tb += wk * (TA[k] - (1.0 - D * z[k]));
                tw += wk;
            }
        tb /= tw;
        double h1 = z[1] - z[0], h2 = z[2] - z[1];
        const double db = -(2.0 * h1 + h2) / (h1 * (h1 + h2)) * sa[0] + (h1 + h2) / (h1 * h2) * sa[1] -
                          h1 / (h2 * (h1 + h2)) * sa[2];
        h1 = z[K] - z[K - 1];
        h2 = z[K - 1] - z[K - 2];
        const double dtp = (2.0 * h1 + h2) / (h1 * (h1 + h2)) * sb[0] - (h1 + h2) / (h1 * h2) * sb[1] +
                           h1 / (h2 * (h1 + h2)) * sb[2];
        r.lambda_b = (tb - sa[0]) / db;
        r.lambda_top = (sb[0] - tb) / dtp;
        // the slope reading: the first distance from a plate where the slope
        // of <T_sa>_A (three-plane quadratic) has fallen to 0.1 D, interpolated
        std::vector<double> s_sa(nz);
        for (int k = 0; k <= K; ++k) s_sa[k] = TA[k] - (1.0 - D * z[k]);
        auto slope = [&](int k) {
            if (k == 0) {
                const double a = z[1] - z[0], b = z[2] - z[1];
                return -(2.0 * a + b) / (a * (a + b)) * s_sa[0] + (a + b) / (a * b) * s_sa[1] - a / (b * (a + b)) * s_sa[2];
            }
            if (k == K) {
                const double a = z[K] - z[K - 1], b = z[K - 1] - z[K - 2];
                return (2.0 * a + b) / (a * (a + b)) * s_sa[K] - (a + b) / (a * b) * s_sa[K - 1] +
                       a / (b * (a + b)) * s_sa[K - 2];
            }
            const double a = z[k] - z[k - 1], b = z[k + 1] - z[k];
            return -b / (a * (a + b)) * s_sa[k - 1] + (b - a) / (a * b) * s_sa[k] + a / (b * (a + b)) * s_sa[k + 1];
        };
        auto crossing = [&](bool top) {
            const double target = 0.1 * D;
            double dprev = 0.0, sprev = 0.0;
            for (int q = 0; q <= K; ++q) {
                const int k = top ? K - q : q;
                const double sk = std::fabs(slope(k)), dk = top ? 1.0 - z[k] : z[k];
                if (sk <= target) return q == 0 ? 0.0 : dprev + (sprev - target) / (sprev - sk) * (dk - dprev);
                dprev = dk;
                sprev = sk;
            }
            return std::nan("");
        };
        r.lambda_b_slope = crossing(false);
        r.lambda_top_slope = crossing(true);
    }
    r.F_n = f[0] / wsum;
    r.F_p = f[1] / wsum;
    r.F_b = f[2] / wsum;
    r.F_v = f[3] / wsum;
    r.r_max = rmax;
    *out = r;
    if (hist_out)
        for (int q = 0; q < nbins; ++q) hist_out[q] = (long long)hist[q];
    return CM_OK;
}

int cm_diagnostics(cm_diag* out, int max, int* n_out)
{
    NEED_CTX();
    if (n_out) *n_out = 0;
    if (max < 0 || (max > 0 && !out)) return fail(CM_EINVAL, "bad output buffer");
    Ctx* c = g_ctx;
    CK(cudaStreamSynchronize(c->stream));
    const int n = c->ring_count < max ? c->ring_count : max;
    int status = CM_OK;
    for (int q = 0; q < n; ++q) {
        const int slot = (c->ring_head + q) % c->ring_cap;
        CK(cudaMemcpy(out + q, c->ring + slot, sizeof(cm_diag), cudaMemcpyDeviceToHost));
        if (out[q].status != CM_OK) status = CM_ENAN;
    }
    c->ring_head = (c->ring_head + n) % c->ring_cap;
    c->ring_count -= n;
    if (n_out) *n_out = n;
    if (status) return fail(status, "a diagnostics sample met a non-finite value");
    return CM_OK;
}

void* cm_state_ptr(int field)
{
    if (!g_ctx || field < 0 || field >= g_ctx->nf) return nullptr;
    return (char*)g_ctx->buf[g_ctx->cur] + (size_t)field * g_ctx->fstride * g_ctx->elem;
}

int cm_state_layout(int* pitch, int* nfields, int* elem_bytes)
{
    NEED_CTX();
    if (pitch) *pitch = g_ctx->pitch;
    if (nfields) *nfields = g_ctx->nf;
    if (elem_bytes) *elem_bytes = (int)g_ctx->elem;
    return CM_OK;
}

int cm_get_state(double* host)
{
    NEED_CTX();
    if (!host) return fail(CM_EINVAL, "host is NULL");
    int rc = download(g_ctx, host);
    if (rc) return rc;
    CK(cudaStreamSynchronize(g_ctx->stream));
    return CM_OK;
}

int cm_set_state(const double* host)
{
    NEED_CTX();
    if (!host) return fail(CM_EINVAL, "host is NULL");
    int rc = upload(g_ctx, host);
    if (rc) return drain_on_error(g_ctx, rc);
    CK(cudaStreamSynchronize(g_ctx->stream));
    return CM_OK;
}

int cm_set_temperature(const double* T)
{
    NEED_CTX();
    Ctx* c = g_ctx;
    if (!T) return fail(CM_EINVAL, "T is NULL");
    const int nz = c->grid.nz;
    const size_t plane = (size_t)c->ny * c->grid.nx;
    for (size_t n = plane; n < (size_t)(nz - 1) * plane; ++n)
        if (!(T[n] > 0.0) || !std::isfinite(T[n]))
            return fail(CM_EINVAL, "interior temperature %g at dense index %zu is not a positive finite number", T[n], n);
    return drain_on_error(c, [&]() -> int {
        int rc = ensure_dense(c);
        if (rc) return rc;
        CK(cudaMemcpyAsync(c->dense, T, (size_t)nz * plane * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        InitArgs A;
        A.Tc = c->Tc_d;
        A.pc = c->pc_d;
        A.zt = c->zt_d;
        A.a = c->a;
        A.b = c->b;
        A.g = c->g;
        A.amp = 0.0;
        A.seed = 0;
        A.Tfield = c->dense;
        cudaError_t e = c->prec == CM_FP64 ? Launch<double>::init((double*)c->buf[c->cur], c->cd, A, c->stream)
                                            : Launch<float>::init((float*)c->buf[c->cur], c->cf, A, c->stream);
        if (e != cudaSuccess) return fail(CM_ECUDA, "init launch: %s", cudaGetErrorString(e));
        c->launches++;
        if ((rc = recompute_dt(c, (int)(c->step & 1)))) return rc;
        CK(cudaStreamSynchronize(c->stream));
        return CM_OK;
    }());
}

int cm_run_host(const double* state_in, int nsteps, double* state_out, cm_diag* diag_out)
{
    NEED_CTX();
    if (nsteps < 0) return fail(CM_EINVAL, "nsteps must be >= 0");
    Ctx* c = g_ctx;
    return drain_on_error(c, [&]() -> int {
        int rc;
        if (state_in && (rc = upload(c, state_in))) return rc;
        if ((rc = queue_steps(c, nsteps))) return rc;
        if (state_out && (rc = download(c, state_out))) return rc;
        if (diag_out && (rc = sample_final(c, diag_out))) return rc;
        CK(cudaStreamSynchronize(c->stream));
        if (diag_out && diag_out->status != CM_OK) return fail(CM_ENAN, "non-finite value in the final state");
        return CM_OK;
    }());
}

int cm_run_host_f32(const float* state_in, int nsteps, float* state_out, cm_diag* diag_out)
{
    NEED_CTX();
    Ctx* c = g_ctx;
    if (c->prec != CM_FP32) return fail(CM_EINVAL, "cm_run_host_f32 needs an FP32 context");
    if (nsteps < 0) return fail(CM_EINVAL, "nsteps must be >= 0");
    return drain_on_error(c, [&]() -> int {
        int rc;
        float* dense32 = nullptr;
        if (state_out && host_kind<float>(state_out, dense_count(c), nullptr) < 0)
            return refuse_split_pinned("the host output");
        if ((state_in || state_out) && (rc = ensure_dense(c))) return rc;
        dense32 = (float*)c->dense;  // the FP64 staging area holds twice as many floats
        const size_t bytes = dense_count(c) * sizeof(float);
        if (state_in && (rc = upload_host(c, state_in))) return rc;
        if ((rc = queue_steps(c, nsteps))) return rc;
        if (state_out) {
            cudaError_t e = Launch<float>::unpack32((const float*)c->buf[c->cur], dense32, c->cf, c->nf, c->stream);
            if (e != cudaSuccess) return fail(CM_ECUDA, "unpack launch: %s", cudaGetErrorString(e));
            c->launches++;
            CK(cudaMemcpyAsync(state_out, dense32, bytes, cudaMemcpyDeviceToHost, c->stream));
        }
        if (diag_out && (rc = sample_final(c, diag_out))) return rc;
        CK(cudaStreamSynchronize(c->stream));
        if (diag_out && diag_out->status != CM_OK) return fail(CM_ENAN, "non-finite value in the final state");
        return CM_OK;
    }());
}

int cm_sweep(int dir, double Delta)
{
    NEED_CTX();
    if (g_ctx->grid.ndim == 3 ? (dir < 0 || dir > 2) : (dir != 0 && dir != 2))
        return fail(CM_EINVAL, "dir must be 0 (x), 1 (y, 3D only) or 2 (z)");
    if (!(Delta > 0)) return fail(CM_EINVAL, "Delta must be > 0");
    SweepCtl sc;
    sc.ctl = g_ctx->ctl;
    sc.slot_in = (int)(g_ctx->step & 1);
    sc.first = 0;
    sc.last = 0;
    sc.Delta = Delta;
    return sweep(g_ctx, dir, sc);
}

int cm_get_dt(double* dt)
{
    NEED_CTX();
    if (!dt) return fail(CM_EINVAL, "dt is NULL");
    DevCtl h;
    CK(cudaMemcpyAsync(&h, g_ctx->ctl, sizeof h, cudaMemcpyDeviceToHost, g_ctx->stream));
    CK(cudaStreamSynchronize(g_ctx->stream));
    double m;
    std::memcpy(&m, &h.dt_slot[g_ctx->step & 1], sizeof m);
    *dt = g_ctx->prm.dt_fixed > 0 ? g_ctx->prm.dt_fixed : g_ctx->prm.cfl * m;
    return CM_OK;
}

int cm_get_time(double* t, long long* steps)
{
    NEED_CTX();
    DevCtl h;
    CK(cudaMemcpyAsync(&h, g_ctx->ctl, sizeof h, cudaMemcpyDeviceToHost, g_ctx->stream));
    CK(cudaStreamSynchronize(g_ctx->stream));
    if (t) *t = h.t;
    if (steps) *steps = (long long)h.steps;
    return CM_OK;
}

int cm_profile_steps(int n, unsigned long long flush_bytes, double* ms_out, double* step_ms)
{
    NEED_CTX();
    if (n < 1 || (!ms_out && !step_ms)) return fail(CM_EINVAL, "need n >= 1 and ms_out or step_ms");
    Ctx* c = g_ctx;
    void* flush = nullptr;
    if (flush_bytes) {
        if (cudaMalloc(&flush, flush_bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(CM_ENOMEM, "cudaMalloc of the %llu-byte flush buffer failed", flush_bytes);
        }
    }
    const int S = sweeps_per_step(c);
    const bool per_sweep = ms_out != nullptr;
    std::vector<cudaEvent_t> ev((per_sweep ? S + 1 : 2) * (size_t)n, nullptr);
    int rc = CM_OK;
    for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) { rc = fail(CM_ECUDA, "cudaEventCreate failed"); break; }
    if (!rc) rc = queue_steps(c, n, ev.data(), flush, flush_bytes, per_sweep);
    if (!rc && cudaStreamSynchronize(c->stream) != cudaSuccess)
        rc = fail(CM_ECUDA, "profiled steps failed: %s", cudaGetErrorString(cudaGetLastError()));
    double ms[6] = {0, 0, 0, 0, 0, 0};
    for (int s = 0; !rc && !per_sweep && s < n; ++s) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, ev[2 * s], ev[2 * s + 1]) != cudaSuccess)
            rc = fail(CM_ECUDA, "cudaEventElapsedTime failed");
        step_ms[s] = t;
    }
    for (int s = 0; !rc && per_sweep && s < n; ++s) {
        double tot = 0;
        for (int q = 0; q < S; ++q) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, ev[(S + 1) * s + q], ev[(S + 1) * s + q + 1]) != cudaSuccess) {
                rc = fail(CM_ECUDA, "cudaEventElapsedTime failed");
                break;
            }
            ms[q] += t;
            tot += t;
        }
        if (step_ms) step_ms[s] = tot;
    }
    for (auto& e : ev)
        if (e) cudaEventDestroy(e);
    if (flush) cudaFree(flush);
    if (rc) return rc;
    if (per_sweep)
        for (int q = 0; q < S; ++q) ms_out[q] = ms[q] / n;
    return CM_OK;
}

long long cm_launch_count(void) { return g_ctx ? g_ctx->launches : 0; }

int cm_sync(void)
{
    NEED_CTX();
    CK(cudaStreamSynchronize(g_ctx->stream));
    DevCtl h;
    CK(cudaMemcpy(&h, g_ctx->ctl, sizeof h, cudaMemcpyDeviceToHost));
    if (h.status & 1) return fail(CM_ENAN, "a non-finite value was met while stepping");
    return CM_OK;
}

int cm_save(const char* path)
{
    NEED_CTX();
    if (!path) return fail(CM_EINVAL, "path is NULL");
    Ctx* c = g_ctx;
    std::vector<double> host(dense_count(c));
    int rc = download(c, host.data());
    if (rc) return rc;
    DevCtl h;
    CK(cudaMemcpyAsync(&h, c->ctl, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    CkptHeader H;
    std::memset(&H, 0, sizeof H);
    std::memcpy(H.magic, "CMCKPT1", 8);
    H.version = 1;
    H.ndim = c->grid.ndim;
    H.nx = c->grid.nx;
    H.ny = c->ny;
    H.nz = c->grid.nz;
    H.precision = c->prec;
    H.step = c->step;
    H.t = h.t;
    H.hash = param_hash(c);
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(CM_EINVAL, "cannot open %s for writing", path);
    bool ok = std::fwrite(&H, sizeof H, 1, f) == 1 && std::fwrite(host.data(), sizeof(double), host.size(), f) == host.size();
    ok = (std::fclose(f) == 0) && ok;
    return ok ? CM_OK : fail(CM_EINVAL, "write to %s failed", path);
}

int cm_load(const char* path)
{
    NEED_CTX();
    if (!path) return fail(CM_EINVAL, "path is NULL");
    Ctx* c = g_ctx;
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(CM_EBADCKPT, "cannot open %s", path);
    CkptHeader H;
    std::vector<double> host(dense_count(c));
    bool ok = std::fread(&H, sizeof H, 1, f) == 1;
    ok = ok && std::memcmp(H.magic, "CMCKPT1", 8) == 0 && H.version == 1 && H.ndim == c->grid.ndim &&
         H.nx == c->grid.nx && H.ny == c->ny && H.nz == c->grid.nz && H.precision == c->prec && H.hash == param_hash(c);
    ok = ok && std::fread(host.data(), sizeof(double), host.size(), f) == host.size();
    std::fclose(f);
    if (!ok) return fail(CM_EBADCKPT, "%s is not a checkpoint of this grid, precision and parameter set", path);
    for (double v : host)
        if (!std::isfinite(v)) return fail(CM_EBADCKPT, "%s holds non-finite values", path);
    c->step = H.step;
    int rc = upload(c, host.data());
    if (rc) return drain_on_error(c, rc);
    DevCtl h;
    CK(cudaMemcpyAsync(&h, c->ctl, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    h.t = H.t;
    h.steps = (double)H.step;
    CK(cudaMemcpyAsync(c->ctl, &h, sizeof h, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return CM_OK;
}

// Coefficients of the plate derivative of the quadratic through three planes
// h1 and h1 + h2 away from the plate: f'(plate) = c0 f_0 + c1 f_1 + c2 f_2
// (second-order one-sided difference; on uniform planes (-3, 4, -1) / (2 dz)).
static void plate_coefs(double h1, double h2, double c[3])
{
    c[0] = -(2.0 * h1 + h2) / (h1 * (h1 + h2));
    c[1] = (h1 + h2) / (h1 * h2);
    c[2] = -h1 / (h2 * (h1 + h2));
}

// planes of the plate Nusselt differences and the weights of dNu_bar/d(sum_x T)
// (Eq. mean_Nu: Nu_0 = -(1/eps)(-3 f_0 + 4 f_1 - f_2)/(2 dz), Nu_1 = -(1/eps)(3 g_0 -
// 4 g_1 + g_2)/(2 dz), f_q, g_q the x-mean of T minus 1 - D z at planes q and K-q;
// on a stretched grid the three-plane quadratic's derivative at each plate)
static void nu_planes(const Ctx* c, int kq[6], double wq[6])
{
    const int K = c->grid.nz - 1;
    const int k6[6] = {0, 1, 2, K, K - 1, K - 2};
    for (int q = 0; q < 6; ++q) kq[q] = k6[q];
    if (c->zp_d) {
        const double* z = c->zplanes;
        const double s = -(1.0 / c->prm.eps) / (double)c->grid.nx;
        double cb[3], ct[3];
        plate_coefs(z[1] - z[0], z[2] - z[1], cb);
        plate_coefs(z[K] - z[K - 1], z[K - 1] - z[K - 2], ct);
        for (int q = 0; q < 3; ++q) {
            wq[q] = 0.5 * s * cb[q];
            wq[3 + q] = -0.5 * s * ct[q];  // the top derivative points into the fluid: -d/dz
        }
        return;
    }
    const double dz = 1.0 / K, s = -(1.0 / c->prm.eps) / (2.0 * dz) / (double)c->grid.nx;
    const double c6[6] = {-3.0, 4.0, -1.0, 3.0, -4.0, 1.0};
    for (int q = 0; q < 6; ++q) wq[q] = 0.5 * s * c6[q];
}

static double nu_bar_of(const Ctx* c, const double* S)
{
    const int K = c->grid.nz - 1;
    const double nx = (double)c->grid.nx, D = c->prm.D, eps = c->prm.eps, dz = 1.0 / K;
    double f[3], g[3];
    if (c->zp_d) {
        // as the diagnostics on a stretched grid: quadratic through three planes
        const double* z = c->zplanes;
        for (int q = 0; q < 3; ++q) {
            f[q] = S[q] / nx - (1.0 - D * z[q]);
            g[q] = S[3 + q] / nx - (1.0 - D * z[K - q]);
        }
        double h1 = z[1] - z[0], h2 = z[2] - z[1];
        const double db = -(2.0 * h1 + h2) / (h1 * (h1 + h2)) * f[0] + (h1 + h2) / (h1 * h2) * f[1]
                          - h1 / (h2 * (h1 + h2)) * f[2];
        h1 = z[K] - z[K - 1];
        h2 = z[K - 1] - z[K - 2];
        const double dtp = (2.0 * h1 + h2) / (h1 * (h1 + h2)) * g[0] - (h1 + h2) / (h1 * h2) * g[1]
                           + h1 / (h2 * (h1 + h2)) * g[2];
        return (-(1.0 / eps) * db + -(1.0 / eps) * dtp) / 2.0;
    }
    for (int q = 0; q < 3; ++q) {
        f[q] = S[q] / nx - (1.0 - D * ((double)q / (double)K));
        g[q] = S[3 + q] / nx - (1.0 - D * ((double)(K - q) / (double)K));
    }
    const double nb = -(1.0 / eps) * (-3.0 * f[0] + 4.0 * f[1] - f[2]) / (2.0 * dz);
    const double nt = -(1.0 / eps) * (3.0 * g[0] - 4.0 * g[1] + g[2]) / (2.0 * dz);
    return (nb + nt) / 2.0;
}

int cm_adj_set_dts(const double* dts, int n)
{
    NEED_CTX();
    Ctx* c = g_ctx;
    if (n < 0 || (n > 0 && !dts)) return fail(CM_EINVAL, "cm_adj_set_dts: need n >= 0 and dts for n > 0");
    for (int s = 0; s < n; ++s)
        if (!(dts[s] > 0.0) || !std::isfinite(dts[s]))
            return fail(CM_EINVAL, "cm_adj_set_dts: dt of step %d is %g, not a positive finite number", s, dts[s]);
    if (!c->adj) c->adj = new AdjCtx();
    c->adj->replay.assign(dts, dts + n);
    return CM_OK;
}

int cm_adj_get_dts(double* dts, int n)
{
    NEED_CTX();
    const AdjCtx* A = g_ctx->adj;
    if (!A || A->nsteps < 1 || n != A->nsteps || !dts)
        return fail(CM_EINVAL, "cm_adj_get_dts: need the step count of the last cm_adj_forward and a buffer");
    std::memcpy(dts, A->dts.data(), sizeof(double) * (size_t)n);
    return CM_OK;
}

int cm_adj_forward(int nsteps, int K, int win_begin, double* J)
{
    NEED_CTX();
    Ctx* c = g_ctx;
    if (c->prec != CM_FP64 || c->grid.ndim != 2) return fail(CM_EINVAL, "the adjoint needs a 2D FP64 context");
    if (c->prm.split != CM_SPLIT_PRINTED) return fail(CM_EINVAL, "the adjoint needs split = CM_SPLIT_PRINTED");
    if (nsteps < 1 || K < 0 || win_begin < 1 || win_begin > nsteps)
        return fail(CM_EINVAL, "need nsteps >= 1, K >= 0, 1 <= win_begin <= nsteps");
    if (!c->adj) c->adj = new AdjCtx();
    AdjCtx* A = c->adj;
    // replayed dts: each step runs with dt_fixed = its dt (restored below)
    const bool replay = (int)A->replay.size() == nsteps;
    const double dt_fixed0 = c->cd.dt_fixed;
    cudaFree(A->ckpt);
    cudaFree(A->dts_d);
    cudaFree(A->planes_d);
    A->ckpt = nullptr;
    A->dts_d = A->planes_d = nullptr;
    A->nsteps = 0;
    // K = 0: the forward sweeps write into 4 nsteps + 1 stored states, which the
    // reverse pass reads without recomputing anything
    const bool keep_all = K == 0;
    const int nck = keep_all ? 4 * nsteps + 1 : (nsteps + K - 1) / K, nwin = nsteps - win_begin + 1;
    if (cudaMalloc(&A->ckpt, (size_t)nck * c->buf_bytes) != cudaSuccess ||
        cudaMalloc(&A->dts_d, (size_t)nsteps * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&A->planes_d, (size_t)nwin * 6 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return fail(CM_ENOMEM, "adjoint forward: cudaMalloc of %zu checkpoint bytes failed", (size_t)nck * c->buf_bytes);
    }
    int kq[6];
    double wq[6];
    nu_planes(c, kq, wq);
    auto stored = [&](int q) { return (double*)(A->ckpt + (size_t)q * c->buf_bytes); };
    if (keep_all) CK(cudaMemcpyAsync(stored(0), c->buf[c->cur], c->buf_bytes, cudaMemcpyDeviceToDevice, c->stream));
    const int order[4] = {2, 0, 2, 0};
    for (int s = 0; s < nsteps; ++s) {
        if (!keep_all && s % K == 0)
            CK(cudaMemcpyAsync(stored(s / K), c->buf[c->cur], c->buf_bytes, cudaMemcpyDeviceToDevice, c->stream));
        if (replay) c->cd.dt_fixed = A->replay[s];
        cudaError_t e = adj_record_dt(c->ctl, (int)(c->step & 1), c->prm.cfl, c->cd.dt_fixed, A->dts_d + s, c->stream);
        if (e != cudaSuccess) {
            c->cd.dt_fixed = dt_fixed0;
            return fail(CM_ECUDA, "adjoint forward: %s", cudaGetErrorString(e));
        }
        if (keep_all) {  // the step of queue_steps, each sweep into its own stored state
            SweepCtl sc;
            std::memset(&sc, 0, sizeof sc);
            sc.ctl = c->ctl;
            sc.slot_in = (int)(c->step & 1);
            for (int q = 0; q < 4 && e == cudaSuccess; ++q) {
                sc.first = q == 0;
                sc.last = q == 3;
                e = Launch<double>::sweep(order[q], stored(4 * s + q), stored(4 * s + q + 1),
                                          (const double*)c->zt_r, c->cd, sc, 0, c->stream);
                c->launches++;
            }
            c->cd.dt_fixed = dt_fixed0;
            if (e != cudaSuccess) return fail(CM_ECUDA, "adjoint forward: %s", cudaGetErrorString(e));
            c->step++;
        } else {
            int rc = queue_steps(c, 1);
            c->cd.dt_fixed = dt_fixed0;
            if (rc) return rc;
        }
        const double* Xn = keep_all ? stored(4 * s + 4) : (const double*)c->buf[c->cur];
        if (s + 1 >= win_begin) {
            e = adj_plane_T(Xn, c->zt_d, c->cd, kq, 6, A->planes_d + (size_t)(s + 1 - win_begin) * 6, c->stream);
            if (e != cudaSuccess) return fail(CM_ECUDA, "adjoint forward: %s", cudaGetErrorString(e));
        }
        c->launches += 2;
    }
    if (keep_all)
        CK(cudaMemcpyAsync(c->buf[c->cur], stored(4 * nsteps), c->buf_bytes, cudaMemcpyDeviceToDevice, c->stream));
    A->dts.assign(nsteps, 0.0);
    A->plane_sums.assign((size_t)nwin * 6, 0.0);
    CK(cudaMemcpyAsync(A->dts.data(), A->dts_d, nsteps * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(A->plane_sums.data(), A->planes_d, (size_t)nwin * 6 * sizeof(double), cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    double sum = 0.0;
    for (int q = 0; q < nwin; ++q) sum += nu_bar_of(c, A->plane_sums.data() + (size_t)q * 6);
    A->J = sum / nwin;
    A->nsteps = nsteps;
    A->K = K;
    A->win = win_begin;
    if (J) *J = A->J;
    return CM_OK;
}

int cm_adj_backward(double* grad_X0, double* grad_T0, double* grad_Ra)
{
    NEED_CTX();
    Ctx* c = g_ctx;
    AdjCtx* A = c->adj;
    if (!A || A->nsteps < 1) return fail(CM_EINVAL, "cm_adj_backward needs a cm_adj_forward first");
    const bool keep_all = A->K == 0;
    const int K = keep_all ? A->nsteps : A->K, nsteps = A->nsteps, nwin = nsteps - A->win + 1;
    const int nck = keep_all ? 1 : (nsteps + K - 1) / K;
    const size_t bb = c->buf_bytes;
    char* slots = nullptr;   // 4K+1 sweep inputs of one segment
    char* xbar = nullptr;    // two adjoint states
    double* acc = nullptr;   // dJ/dmu, dJ/dK
    double* gT = nullptr;    // dense dJ/dT
    AdjWork W;
    std::memset(&W, 0, sizeof W);
    int rc = CM_OK;
    auto cleanup = [&]() {
        cudaFree(slots);
        cudaFree(xbar);
        cudaFree(acc);
        cudaFree(gT);
        adj_work_free(&W);
    };
    if ((!keep_all && cudaMalloc(&slots, (size_t)(4 * K + 1) * bb) != cudaSuccess) ||
        cudaMalloc(&xbar, 2 * bb) != cudaSuccess ||
        cudaMalloc(&acc, 2 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&gT, (size_t)c->grid.nx * c->grid.nz * sizeof(double)) != cudaSuccess ||
        adj_work_create(&W, c->cd) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return fail(CM_ENOMEM, "adjoint backward: cudaMalloc of %zu bytes of sweep inputs failed",
                    (size_t)(4 * K + 1) * bb);
    }
    W.frozen_phi = c->prm.adj_limiter == CM_ADJ_PHI_FROZEN ? 1 : 0;
    char* base = keep_all ? A->ckpt : slots;
    auto slot = [&](int q) { return (double*)(base + (size_t)q * bb); };
    int xc = 0;
    auto xb = [&](int q) { return (double*)(xbar + (size_t)q * bb); };
    int kq[6];
    double wq[6];
    nu_planes(c, kq, wq);
    for (int q = 0; q < 6; ++q) wq[q] /= (double)nwin;
    const int order[4] = {2, 0, 2, 0};
    cudaError_t e = cudaMemsetAsync(xbar, 0, 2 * bb, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, 2 * sizeof(double), c->stream);
    for (int j = nck - 1; j >= 0 && e == cudaSuccess; --j) {
        const int s0 = j * K, s1 = std::min(nsteps, s0 + K) - 1;
        // recompute the segment, keeping every sweep input (stored already when K = 0)
        if (!keep_all) e = cudaMemcpyAsync(slot(0), A->ckpt + (size_t)j * bb, bb, cudaMemcpyDeviceToDevice, c->stream);
        for (int s = s0; s <= s1 && e == cudaSuccess && !keep_all; ++s) {
            SweepCtl sc;
            std::memset(&sc, 0, sizeof sc);
            sc.ctl = c->ctl;
            sc.Delta = 0.5 * A->dts[s];
            for (int q = 0; q < 4 && e == cudaSuccess; ++q) {
                const int at = 4 * (s - s0) + q;
                e = Launch<double>::sweep(order[q], slot(at), slot(at + 1), (const double*)c->zt_r, c->cd, sc, 0,
                                          c->stream);
                c->launches++;
            }
        }
        // reverse, step by step
        for (int s = s1; s >= s0 && e == cudaSuccess; --s) {
            const double Delta = 0.5 * A->dts[s];
            if (s + 1 >= A->win) {
                e = adj_seed_T(xb(xc), slot(4 * (s - s0) + 4), c->zt_d, c->cd, kq, wq, 6, c->stream);
                c->launches++;
            }
            for (int q = 3; q >= 0 && e == cudaSuccess; --q) {
                e = adj_sweep_vjp(&W, order[q], Delta, slot(4 * (s - s0) + q), xb(xc), xb(xc ^ 1), c->zt_d, c->cd,
                                  acc, c->stream);
                c->launches += 11;
                xc ^= 1;
            }
        }
    }
    if (e != cudaSuccess) {
        cleanup();
        return fail(CM_ECUDA, "adjoint backward: %s", cudaGetErrorString(e));
    }
    if (grad_X0) {
        if ((rc = ensure_dense(c))) { cleanup(); return rc; }
        e = Launch<double>::unpack(xb(xc), c->dense, c->cd, c->nf, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(grad_X0, c->dense, dense_count(c) * sizeof(double), cudaMemcpyDefault, c->stream);
        c->launches++;
    }
    if (grad_T0 && e == cudaSuccess) {
        e = adj_grad_T((const double*)A->ckpt, xb(xc), c->zt_d, c->cd, gT, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(grad_T0, gT, (size_t)c->grid.nx * c->grid.nz * sizeof(double), cudaMemcpyDefault,
                                c->stream);
        c->launches++;
    }
    double hacc[2] = {0.0, 0.0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(hacc, acc, sizeof hacc, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cleanup();
    if (e != cudaSuccess) return fail(CM_ECUDA, "adjoint backward: %s", cudaGetErrorString(e));
    if (grad_Ra) {
        const double mu = std::sqrt(c->Pr / c->Ra), kth = 1.0 / (c->prm.eps * c->prm.D * std::sqrt(c->Ra * c->Pr));
        *grad_Ra = hacc[0] * (-0.5 * mu / c->Ra) + hacc[1] * (-0.5 * kth / c->Ra);
    }
    return CM_OK;
}

int cm_finalize(void)
{
    if (g_ctx) {
        free_ctx(g_ctx);
        g_ctx = nullptr;
    }
    return CM_OK;
}

const char* cm_last_error(void) { return g_err; }

}  // extern "C"

// shared with the other translation units of the library
namespace cm {
int pitch_of(int nx, int prec)
{
    const int align = prec == CM_FP64 ? 32 : 64;  // 256-byte rows
    return (nx + align - 1) / align * align;
}


int set_error(int code, const char* msg) { return fail(code, "%s", msg); }
}  // namespace cm
