// batch.cu -- the batched ensemble: many independent 2D boxes of uneven sizes
// and Rayleigh numbers advanced together, FP32 state, one launch per sweep
// for all boxes, the steps replayed from a captured CUDA graph.
//
// Each box is the single-box problem of include/cm.h (Sec. 2 equations,
// Sec. 3.1 scheme) with its own dt (per-box device control block), seed and
// Ra, on uniform planes or on a stretched z-grid (Sec. 3; then every box of
// the batch carries a plane table).  Work is split into warp items (box,
// column strip, row segment); the segment length of each box size class is
// chosen at init by an autotuner that times the batched sweeps themselves.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/cm.h"
#include "host_setup.h"
#include "kernels.h"
#include "sweep2d_x2_types.h"

namespace cm {
int set_error(int code, const char* msg);
}
using namespace cm;

namespace {

struct Box {
    cm_grid grid;
    double Ra;
    int pitch;
    long long fstride;
    size_t buf_elems;   // floats in one state buffer
    float* buf[2];
    float* zt_f;
    double* zt_d;
    double* Tc;
    double* pc;
    double* scratch;    // per-plane diagnostics sums
    DevCtl* ctl;
    Plane<float>* zp_f;     // stretched batches: per-plane metric (sweeps), else NULL
    Plane<double>* zp_d;    // the same in FP64 (diagnostics), else NULL
    Coef<float> C;
    int cls;            // size class for the autotuner
    int seg_z, seg_x;   // chosen segment lengths
};

struct Batch {
    std::vector<Box> boxes;
    cm_params prm;
    double Pr, gamma;
    void* pool;         // one allocation for every box's arrays
    BoxDesc* d_boxes;
    BatchWork* d_work_z;
    BatchWork* d_work_x;
    int nblk_z, nblk_x;
    size_t work_cap;    // items the work buffers hold
    cm_diag* d_recs;
    cudaStream_t stream;
    bool own_stream;
    long long step;
    long long launches;
    cudaGraphExec_t graph;
    int graph_steps;
    int cur;
    bool const_coefs;   // coefficients in constant memory (at most kConstBoxes boxes)
    bool stretched;     // some box has a stretched z-grid: every box runs the plane-table sweeps
};

Batch* g_batch = nullptr;

int ck(cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return CM_OK;
    char msg[256];
    snprintf(msg, sizeof msg, "%s: %s", what, cudaGetErrorString(e));
    cudaGetLastError();
    return set_error(CM_ECUDA, msg);
}

#define CKB(call) do { int rc_ = ck((call), #call); if (rc_) return rc_; } while (0)

// warp work items of one sweep for the given per-box segment lengths;
// each box's items are padded to whole blocks of kWarpsPerBlock warps.  The
// blocks are then ordered by decreasing cost (rows stepped by their longest
// warp, pipeline ramp included), so that the hardware's in-order block
// dispatch schedules the longest first and short blocks fill the tail.
std::vector<BatchWork> build_work(const Batch& B, bool zdir)
{
    std::vector<BatchWork> w;
    for (int b = 0; b < (int)B.boxes.size(); ++b) {
        const Box& x = B.boxes[b];
        const int seg = zdir ? x.seg_z : x.seg_x;
        const int nstrips = (x.grid.nx + kOutW2 - 1) / kOutW2;
        const int nsegs = (x.grid.nz + seg - 1) / seg;
        const size_t first = w.size();
        for (int sg = 0; sg < nsegs; ++sg)
            for (int st = 0; st < nstrips; ++st) w.push_back({b, st, sg * seg, seg, 0, {0, 0, 0}});
        while ((w.size() - first) % kWarpsPerBlock) w.push_back({b, 0, 1 << 30, seg, 0, {0, 0, 0}});
        for (size_t q = first; q < first + kWarpsPerBlock; ++q) w[q].lead = 1;
    }
    const size_t nblk = w.size() / kWarpsPerBlock;
    std::vector<int> cost(nblk, 0), order(nblk);
    for (size_t k = 0; k < nblk; ++k) {
        for (int q = 0; q < kWarpsPerBlock; ++q) {
            const BatchWork& it = w[k * kWarpsPerBlock + q];
            const int nz = B.boxes[it.box].grid.nz;
            if (it.ks < nz) cost[k] = std::max(cost[k], std::min(it.seg_rows, nz - it.ks) + 3);
        }
        order[k] = (int)k;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<BatchWork> sorted(w.size());
    for (size_t k = 0; k < nblk; ++k)
        for (int q = 0; q < kWarpsPerBlock; ++q) sorted[k * kWarpsPerBlock + q] = w[order[k] * kWarpsPerBlock + q];
    return sorted;
}

int upload_work(Batch& B)
{
    const std::vector<BatchWork> wz = build_work(B, true), wx = build_work(B, false);
    if (wz.size() > B.work_cap || wx.size() > B.work_cap) return set_error(CM_EINVAL, "batch work list overflow");
    CKB(cudaMemcpyAsync(B.d_work_z, wz.data(), wz.size() * sizeof(BatchWork), cudaMemcpyHostToDevice, B.stream));
    CKB(cudaMemcpyAsync(B.d_work_x, wx.data(), wx.size() * sizeof(BatchWork), cudaMemcpyHostToDevice, B.stream));
    CKB(cudaStreamSynchronize(B.stream));
    B.nblk_z = (int)(wz.size() / kWarpsPerBlock);
    B.nblk_x = (int)(wx.size() / kWarpsPerBlock);
    return CM_OK;
}

int launch(Batch& B, int dir, int first, int last, double Delta)
{
    BatchLaunch L;
    L.boxes = B.d_boxes;
    L.work = dir == 2 ? B.d_work_z : B.d_work_x;
    L.cur = B.cur;
    L.slot = (int)(B.step & 1);
    L.first = first;
    L.last = last;
    L.Delta = Delta;
    CKB(launch_sweep_batch(dir, L, dir == 2 ? B.nblk_z : B.nblk_x, B.const_coefs, B.stretched, B.prm.layout_exact != 0,
                           B.stream));
    B.launches++;
    return CM_OK;
}

int queue_steps(Batch& B, int n)
{
    for (int s = 0; s < n; ++s) {
        // z, x, z, x (Eq. time_step, rightmost operator first), or its palindrome x, z, z, x
        static const int printed[4] = {2, 0, 2, 0}, symmetric[4] = {0, 2, 2, 0};
        const int* order = B.prm.split == CM_SPLIT_SYMMETRIC ? symmetric : printed;
        for (int q = 0; q < 4; ++q) {
            int rc = launch(B, order[q], q == 0, q == 3, 0.0);
            if (rc) return rc;
            B.cur ^= 1;
        }
        B.step++;
    }
    return CM_OK;
}

// time one batched sweep (fixed tiny Delta, written to the scratch buffer,
// no bookkeeping): *ms = median of 3 after a warm-up
int time_sweep(Batch& B, int dir, float* ms_out)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CKB(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return set_error(CM_ECUDA, "autotune: cudaEventCreate failed");
    }
    std::vector<float> t;
    int rc = CM_OK;
    for (int r = 0; r < 4 && !rc; ++r) {
        float ms = 0.f;
        rc = ck(cudaEventRecord(e0, B.stream), "autotune: cudaEventRecord");
        if (!rc) rc = launch(B, dir, 0, 0, 1e-9);
        if (!rc) rc = ck(cudaEventRecord(e1, B.stream), "autotune: cudaEventRecord");
        if (!rc) rc = ck(cudaEventSynchronize(e1), "autotune: cudaEventSynchronize");
        if (!rc) rc = ck(cudaEventElapsedTime(&ms, e0, e1), "autotune: cudaEventElapsedTime");
        if (!rc && r) t.push_back(ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    std::sort(t.begin(), t.end());
    *ms_out = t[t.size() / 2];
    return CM_OK;
}

// Autotuner: coordinate descent over the segment length of each box size
// class (nz < 64, < 128, < 256, >= 256), per sweep direction, on the timed
// batched sweep itself; two passes over the classes, since the best length
// of one class depends on how the others fill the GPU.
int autotune(Batch& B)
{
    // CM_SEG_ROWS=n: every box runs n-row segments, untuned (profiling captures)
    if (const char* e = getenv("CM_SEG_ROWS")) {
        const int n = std::min(std::max(atoi(e), kBatchSegMin), kBatchSegMax);
        for (Box& x : B.boxes) x.seg_z = x.seg_x = n;
        return upload_work(B);
    }
    // not only powers of two: the single-box sweeps ran fastest at 29 rows
    const int cand[] = {kBatchSegMin, 8, 10, 12, 14, 16, 20, 24, 29, 32, 40, 48, 64, 96, 128};
    static_assert(kBatchSegMax >= 128, "the stretched batch kernels size their plane caches for kBatchSegMax rows");
    bool present[4] = {false, false, false, false};
    for (const Box& x : B.boxes) present[x.cls] = true;
    for (int dir : {2, 0}) {
        int seg[4] = {32, 32, 32, 32};
        auto apply = [&]() {
            for (Box& x : B.boxes) (dir == 2 ? x.seg_z : x.seg_x) = seg[x.cls];
            return upload_work(B);
        };
        int rc = apply();
        if (rc) return rc;
        float best = 0.f;
        if ((rc = time_sweep(B, dir, &best))) return rc;
        for (int pass = 0; pass < 2; ++pass) {
            for (int c = 0; c < 4; ++c) {
                if (!present[c]) continue;
                for (int v : cand) {
                    if (v == seg[c]) continue;
                    const int keep = seg[c];
                    seg[c] = v;
                    if ((rc = apply())) return rc;
                    float t = 0.f;
                    if ((rc = time_sweep(B, dir, &t))) return rc;
                    if (t < 0.99f * best) best = t;
                    else seg[c] = keep;
                }
            }
        }
        if ((rc = apply())) return rc;
    }
    return ck(cudaGetLastError(), "autotune");
}

void free_batch(Batch* B)
{
    if (!B) return;
    cudaStreamSynchronize(B->stream);
    if (B->graph) cudaGraphExecDestroy(B->graph);
    cudaFree(B->pool);
    cudaFree(B->d_boxes);
    cudaFree(B->d_work_z);
    cudaFree(B->d_work_x);
    cudaFree(B->d_recs);
    if (B->own_stream) cudaStreamDestroy(B->stream);
    delete B;
}

}  // namespace

extern "C" {

int cm_batch_init(int nbox, const cm_grid* grids, const double* Ra, double Pr, double gamma, const cm_params* params)
{
    if (nbox < 1 || !grids || !Ra) return set_error(CM_EINVAL, "cm_batch_init: need nbox >= 1, grids and Ra");
    cm_params P;
    if (params) P = *params;
    else cm_default_params(&P);
    if (P.precision != CM_FP32) return set_error(CM_EINVAL, "cm_batch_init: the batch steps FP32 states");
    if (P.layout_exact != 0 && P.layout_exact != 1) return set_error(CM_EINVAL, "cm_batch_init: layout_exact must be 0 or 1");
    if (P.split != CM_SPLIT_PRINTED && P.split != CM_SPLIT_SYMMETRIC)
        return set_error(CM_EINVAL, "cm_batch_init: split must be CM_SPLIT_PRINTED or CM_SPLIT_SYMMETRIC");
    if (!(Pr > 0) || !(gamma > 1) || !(P.eps > 0) || !(P.D > 0) || !(P.cfl > 0) || P.cfl > 1.0)
        return set_error(CM_EINVAL, "cm_batch_init: bad physical parameters");
    for (int b = 0; b < nbox; ++b) {
        const cm_grid& G = grids[b];
        if (G.ndim != 2 || G.nx < 4 || G.nz < 5 || (G.nx & 1) || !(G.aspect > 0) || !(Ra[b] > 0))
            return set_error(CM_EINVAL, "cm_batch_init: every box must be 2D with even nx >= 4, nz >= 5, Ra > 0");
        if ((long long)G.nz * pitch_of(G.nx, CM_FP32) * 5 >= (1LL << 31))
            return set_error(CM_EINVAL, "cm_batch_init: box too large");
    }
    // z-planes of every box (uniform, tanh or given), validated before any device work
    std::vector<std::vector<double>> planes(nbox);
    bool any_st = false;
    for (int b = 0; b < nbox; ++b) {
        const char* why = "";
        if (!make_planes(grids[b], planes[b], &why)) {
            char msg[160];
            snprintf(msg, sizeof msg, "cm_batch_init: box %d: %s", b, why);
            return set_error(CM_EINVAL, msg);
        }
        any_st = any_st || stretched(grids[b]);
    }
    if (g_batch) { free_batch(g_batch); g_batch = nullptr; }
    Batch* B = new Batch();
    B->prm = P;
    B->Pr = Pr;
    B->gamma = gamma;
    B->pool = nullptr;
    B->d_boxes = nullptr;
    B->d_work_z = B->d_work_x = nullptr;
    B->d_recs = nullptr;
    B->graph = nullptr;
    B->graph_steps = 0;
    B->step = 0;
    B->launches = 0;
    B->cur = 0;
    B->stretched = any_st;
    auto bail = [&](int code) { free_batch(B); return code; };
    if (P.stream) {
        B->stream = (cudaStream_t)P.stream;
        B->own_stream = false;
    } else {
        if (cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(ck(cudaGetLastError(), "cudaStreamCreate"));
        B->own_stream = true;
    }
    // sizes of every box's arrays in one pool (256-byte aligned pieces)
    const Closure K(gamma, P);
    B->boxes.resize(nbox);
    size_t bytes = 0, items = 0;
    auto take = [&](size_t n) { size_t o = bytes; bytes += (n + 255) / 256 * 256; return o; };
    constexpr int kPieces = 9;
    std::vector<size_t> off(kPieces * nbox);
    for (int b = 0; b < nbox; ++b) {
        Box& x = B->boxes[b];
        x.grid = grids[b];
        x.grid.znodes = nullptr;  // caller memory: the planes were copied above
        x.Ra = Ra[b];
        x.pitch = pitch_of(x.grid.nx, CM_FP32);
        x.fstride = (long long)x.grid.nz * x.pitch;
        x.buf_elems = 4 * (size_t)x.fstride;
        const int nz = x.grid.nz;
        x.cls = nz < 64 ? 0 : nz < 128 ? 1 : nz < 256 ? 2 : 3;
        x.seg_z = x.seg_x = kBatchSegMin;  // smallest candidate: sizes the work buffers
        off[kPieces * b + 0] = take(2 * x.buf_elems * sizeof(float));
        off[kPieces * b + 1] = take(nz * sizeof(float));
        off[kPieces * b + 2] = take(nz * sizeof(double));
        off[kPieces * b + 3] = take(nz * sizeof(double));
        off[kPieces * b + 4] = take(nz * sizeof(double));
        off[kPieces * b + 5] = take((size_t)nz * kDiagQ * sizeof(double));
        off[kPieces * b + 6] = take(sizeof(DevCtl));
        off[kPieces * b + 7] = take(any_st ? nz * sizeof(Plane<float>) : 0);
        off[kPieces * b + 8] = take(any_st ? nz * sizeof(Plane<double>) : 0);
        items += ((size_t)((x.grid.nx + kOutW2 - 1) / kOutW2) * ((nz + kBatchSegMin - 1) / kBatchSegMin) + kWarpsPerBlock);
    }
    B->work_cap = items;
    if (cudaMalloc(&B->pool, bytes) != cudaSuccess || cudaMalloc(&B->d_boxes, nbox * sizeof(BoxDesc)) != cudaSuccess ||
        cudaMalloc(&B->d_work_z, items * sizeof(BatchWork)) != cudaSuccess ||
        cudaMalloc(&B->d_work_x, items * sizeof(BatchWork)) != cudaSuccess ||
        cudaMalloc(&B->d_recs, nbox * sizeof(cm_diag)) != cudaSuccess) {
        cudaGetLastError();
        return bail(set_error(CM_ENOMEM, "cm_batch_init: device allocation failed"));
    }
    char* base = (char*)B->pool;
    std::vector<BoxDesc> desc(nbox);
    int rc = CM_OK;
    for (int b = 0; b < nbox && !rc; ++b) {
        Box& x = B->boxes[b];
        const int nz = x.grid.nz;
        x.buf[0] = (float*)(base + off[kPieces * b + 0]);
        x.buf[1] = x.buf[0] + x.buf_elems;
        x.zt_f = (float*)(base + off[kPieces * b + 1]);
        x.zt_d = (double*)(base + off[kPieces * b + 2]);
        x.Tc = (double*)(base + off[kPieces * b + 3]);
        x.pc = (double*)(base + off[kPieces * b + 4]);
        x.scratch = (double*)(base + off[kPieces * b + 5]);
        x.ctl = (DevCtl*)(base + off[kPieces * b + 6]);
        x.zp_f = any_st ? (Plane<float>*)(base + off[kPieces * b + 7]) : nullptr;
        x.zp_d = any_st ? (Plane<double>*)(base + off[kPieces * b + 8]) : nullptr;
        fill_coef(x.C, x.grid, 1, x.pitch, x.fstride, x.Ra, Pr, K, P);
        const Profile prof(planes[b], P, K);
        std::vector<Plane<float>> tf;
        std::vector<Plane<double>> td;
        if (any_st) {
            // uniform boxes of a stretched batch get the table of the planes k/K
            plane_table(planes[b], tf);
            plane_table(planes[b], td);
            x.C.zp = x.zp_f;
        }
        std::vector<float> zf(nz);
        for (int k = 0; k < nz; ++k) zf[k] = (float)prof.z[k];
        DevCtl h;
        std::memset(&h, 0, sizeof h);
        h.dt_slot[0] = h.dt_slot[1] = 0x7FF0000000000000ULL;
        rc = ck(cudaMemsetAsync(x.buf[0], 0, 2 * x.buf_elems * sizeof(float), B->stream), "memset");
        if (!rc) rc = ck(cudaMemcpyAsync(x.zt_f, zf.data(), nz * sizeof(float), cudaMemcpyHostToDevice, B->stream), "upload");
        if (!rc) rc = ck(cudaMemcpyAsync(x.zt_d, prof.z.data(), nz * sizeof(double), cudaMemcpyHostToDevice, B->stream), "upload");
        if (!rc) rc = ck(cudaMemcpyAsync(x.Tc, prof.Tc.data(), nz * sizeof(double), cudaMemcpyHostToDevice, B->stream), "upload");
        if (!rc) rc = ck(cudaMemcpyAsync(x.pc, prof.pc.data(), nz * sizeof(double), cudaMemcpyHostToDevice, B->stream), "upload");
        if (!rc) rc = ck(cudaMemcpyAsync(x.ctl, &h, sizeof h, cudaMemcpyHostToDevice, B->stream), "upload");
        if (!rc && any_st)
            rc = ck(cudaMemcpyAsync(x.zp_f, tf.data(), nz * sizeof(Plane<float>), cudaMemcpyHostToDevice, B->stream), "upload");
        if (!rc && any_st)
            rc = ck(cudaMemcpyAsync(x.zp_d, td.data(), nz * sizeof(Plane<double>), cudaMemcpyHostToDevice, B->stream), "upload");
        InitArgs A;
        A.Tc = x.Tc;
        A.pc = x.pc;
        A.zt = x.zt_d;
        A.a = K.a;
        A.b = K.b;
        A.g = K.g;
        A.amp = P.pert_amp;
        A.seed = P.seed + (unsigned long long)b;
        if (!rc) rc = ck(Launch<float>::init(x.buf[0], x.C, A, B->stream), "init launch");
        if (!rc) rc = ck(Launch<float>::dt(x.buf[0], x.zt_f, x.C, x.ctl, 0, B->stream), "dt launch");
        if (!rc) rc = ck(cudaStreamSynchronize(B->stream), "init");  // host tables above are freed on return
        if (!rc) {
            // the first dt, and the explicit-diffusion bound cm_init applies
            DevCtl hc;
            rc = ck(cudaMemcpy(&hc, x.ctl, sizeof hc, cudaMemcpyDeviceToHost), "control block read");
            double hmin = 0.0;
            std::memcpy(&hmin, &hc.dt_slot[0], sizeof hmin);
            const double dt0 = P.dt_fixed > 0 ? P.dt_fixed : P.cfl * hmin;
            char msg[200];
            if (!rc && (!(dt0 > 0) || !std::isfinite(dt0) || (hc.status & 1))) {
                snprintf(msg, sizeof msg, "cm_batch_init: box %d: non-finite initial state", b);
                rc = set_error(CM_ENAN, msg);
            }
            const double dnum = rc ? 0.0 : diffusion_number(x.grid, planes[b], x.Ra, Pr, P, K, prof.rho_min, dt0);
            if (dnum > 0.5) {
                snprintf(msg, sizeof msg,
                         "cm_batch_init: box %d: explicit diffusion number %.3g > 0.5 at dt = %.3g: refine dt "
                         "(dt_fixed) or raise Ra", b, dnum, dt0);
                rc = set_error(CM_EUNSTABLE, msg);
            }
        }
        desc[b].C = x.C;
        desc[b].buf[0] = x.buf[0];
        desc[b].buf[1] = x.buf[1];
        desc[b].ctl = x.ctl;
        B->launches += 2;
    }
    if (!rc) rc = ck(cudaMemcpyAsync(B->d_boxes, desc.data(), nbox * sizeof(BoxDesc), cudaMemcpyHostToDevice, B->stream), "upload");
    B->const_coefs = nbox <= kConstBoxes;
    if (!rc && B->const_coefs) {
        std::vector<Coef<float>> coefs(nbox);
        for (int b = 0; b < nbox; ++b) coefs[b] = desc[b].C;
        rc = ck(set_batch_coefs(coefs.data(), nbox, B->stream), "coefficient upload");
        if (!rc) rc = ck(cudaStreamSynchronize(B->stream), "coefficient upload");  // coefs is freed on return
    }
    if (!rc) rc = upload_work(*B);
    if (!rc) rc = autotune(*B);
    if (!rc) rc = ck(cudaStreamSynchronize(B->stream), "batch init");
    if (rc) return bail(rc);
    g_batch = B;
    return CM_OK;
}

int cm_batch_step(int n)
{
    if (!g_batch) return set_error(CM_ENOTINIT, "no batch: call cm_batch_init first");
    if (n < 0) return set_error(CM_EINVAL, "n must be >= 0");
    Batch& B = *g_batch;
    const int G = 50;  // steps per captured graph (even: the dt slot parity repeats)
    int rc;
    if ((B.step & 1) && n > 0) {
        if ((rc = queue_steps(B, 1))) return rc;
        --n;
    }
    if (n >= G && !B.graph) {
        cudaGraph_t g;
        CKB(cudaStreamBeginCapture(B.stream, cudaStreamCaptureModeThreadLocal));
        const long long s0 = B.step, l0 = B.launches;
        const int c0 = B.cur;
        rc = queue_steps(B, G);
        cudaError_t e = cudaStreamEndCapture(B.stream, &g);
        B.step = s0;  // capture only records the launches
        B.launches = l0;
        B.cur = c0;
        if (rc) return rc;
        CKB(e);
        e = cudaGraphInstantiate(&B.graph, g, 0);
        cudaGraphDestroy(g);
        CKB(e);
        B.graph_steps = G;
    }
    while (n >= G && B.graph) {
        CKB(cudaGraphLaunch(B.graph, B.stream));
        B.step += G;
        B.launches += 4LL * G;
        n -= G;
    }
    return queue_steps(B, n);
}

int cm_batch_diagnostics(cm_diag* out)
{
    if (!g_batch) return set_error(CM_ENOTINIT, "no batch: call cm_batch_init first");
    if (!out) return set_error(CM_EINVAL, "out is NULL");
    Batch& B = *g_batch;
    const Closure K(B.gamma, B.prm);
    for (int b = 0; b < (int)B.boxes.size(); ++b) {
        Box& x = B.boxes[b];
        DiagArgs A;
        A.zt = x.zt_d;
        A.a = K.a;
        A.b = K.b;
        A.g = K.g;
        A.D = B.prm.D;
        A.cs2 = K.cs2;
        CKB(Launch<float>::diag_planes(x.buf[B.cur], x.C, A, x.scratch, x.ctl, B.stream));
        DiagFinal F{};
        F.Ra = x.Ra;
        F.Pr = B.Pr;
        F.eps = B.prm.eps;
        F.D = B.prm.D;
        F.cfl = B.prm.cfl;
        F.dt_fixed = B.prm.dt_fixed;
        F.cells = (double)x.grid.nx;
        F.nz = x.grid.nz;
        F.slot = (int)(B.step & 1);
        F.zp = x.zp_d;
        CKB(launch_diag_final(x.scratch, x.zt_d, F, x.ctl, B.d_recs + b, B.stream));
        B.launches += 2;
    }
    CKB(cudaMemcpyAsync(out, B.d_recs, B.boxes.size() * sizeof(cm_diag), cudaMemcpyDeviceToHost, B.stream));
    CKB(cudaStreamSynchronize(B.stream));
    for (size_t b = 0; b < B.boxes.size(); ++b)
        if (out[b].status != CM_OK) return set_error(CM_ENAN, "a box met a non-finite value");
    return CM_OK;
}

int cm_batch_get_state(int box, double* host)
{
    if (!g_batch) return set_error(CM_ENOTINIT, "no batch: call cm_batch_init first");
    Batch& B = *g_batch;
    if (box < 0 || box >= (int)B.boxes.size() || !host) return set_error(CM_EINVAL, "bad box or host pointer");
    const Box& x = B.boxes[box];
    std::vector<float> tmp(4 * (size_t)x.grid.nz * x.grid.nx);
    CKB(cudaMemcpy2DAsync(tmp.data(), x.grid.nx * sizeof(float), x.buf[B.cur], x.pitch * sizeof(float),
                          x.grid.nx * sizeof(float), 4 * (size_t)x.grid.nz, cudaMemcpyDeviceToHost, B.stream));
    CKB(cudaStreamSynchronize(B.stream));
    for (size_t q = 0; q < tmp.size(); ++q) host[q] = (double)tmp[q];
    return CM_OK;
}

int cm_batch_tuning(int* seg_z, int* seg_x)
{
    if (!g_batch) return set_error(CM_ENOTINIT, "no batch: call cm_batch_init first");
    for (size_t b = 0; b < g_batch->boxes.size(); ++b) {
        if (seg_z) seg_z[b] = g_batch->boxes[b].seg_z;
        if (seg_x) seg_x[b] = g_batch->boxes[b].seg_x;
    }
    return CM_OK;
}

int cm_batch_profile_steps(int n, unsigned long long flush_bytes, double* total_ms)
{
    if (!g_batch) return set_error(CM_ENOTINIT, "no batch: call cm_batch_init first");
    if (n < 1 || !total_ms) return set_error(CM_EINVAL, "need n >= 1 and total_ms");
    Batch& B = *g_batch;
    void* flush = nullptr;
    if (flush_bytes && cudaMalloc(&flush, flush_bytes) != cudaSuccess) {
        cudaGetLastError();
        return set_error(CM_ENOMEM, "flush buffer allocation failed");
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    if (flush) cudaMemsetAsync(flush, 1, flush_bytes, B.stream);
    cudaEventRecord(e0, B.stream);
    int rc = cm_batch_step(n);
    cudaEventRecord(e1, B.stream);
    float ms = 0.f;
    if (!rc) rc = ck(cudaEventSynchronize(e1), "profiled batch steps");
    if (!rc) rc = ck(cudaEventElapsedTime(&ms, e0, e1), "event time");
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (flush) cudaFree(flush);
    *total_ms = ms;
    return rc;
}

long long cm_batch_launch_count(void) { return g_batch ? g_batch->launches : 0; }

int cm_batch_finalize(void)
{
    if (g_batch) {
        free_batch(g_batch);
        g_batch = nullptr;
    }
    return CM_OK;
}

}  // extern "C"
