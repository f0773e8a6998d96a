/*
 * cm.h -- C ABI of the GB300 MacCormack-TVD compressible-convection solver.
 *
 * The library advances the nondimensional, fully compressible Navier-Stokes-
 * energy equations of arXiv 2411.10372 (Sec. 2: continuity, momentum with
 * gravity -rho/eps, energy with conduction 1/(eps D sqrt(Ra Pr)) and viscous
 * work; ideal gas p = (gamma-1)/(gamma eps D) rho T) in a box of aspect ratio
 * Gamma with periodic side walls and no-slip, fixed-temperature plates, with
 * the operator-split MacCormack predictor-corrector scheme plus TVD correction
 * of Sec. 3.1 (Eq. time_step), on a uniform grid, on one GPU.
 *
 * Conventions shared by every entry point:
 *  - Every function returns an int status: CM_OK (0) or a negative CM_E* code;
 *    cm_last_error() gives a one-line message for the last failure.  No C++
 *    exception crosses this boundary.
 *  - There is one implicit solver context per process (not thread-safe).
 *    cm_init() creates it (replacing any previous one), cm_finalize() frees it.
 *  - Pointers marked "host" are ordinary CPU memory owned by the caller;
 *    pointers marked "device" are CUDA device memory.
 *  - Dense host state arrays are float64, field-major: field f, plane k
 *    (z, k = 0 bottom plate .. nz-1 top plate), row j (y, 3D only), column i
 *    (x) at ((f*nz + k)*ny + j)*nx + i.  2D fields: rho, m_x, m_z, E.
 *    3D fields: rho, m_x, m_y, m_z, E.  (m = rho u, E total energy density.)
 *  - Work is queued on the stream given in cm_params.stream (NULL = the
 *    legacy default stream) and runs asynchronously unless stated.
 *  - After any error other than CM_EINVAL from argument checks, call
 *    cm_finalize() and cm_init() again.
 */
#ifndef CM_H
#define CM_H

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define CM_OK 0
#define CM_EINVAL (-1)      /* bad argument */
#define CM_ECUDA (-2)       /* a CUDA runtime call failed */
#define CM_ENOTINIT (-3)    /* no context: call cm_init first */
#define CM_ENAN (-4)        /* non-finite value met in a reduction */
#define CM_EUNSTABLE (-7)   /* explicit diffusion number above 1/2 at init */
#define CM_ENOMEM (-8)      /* device allocation failed */
#define CM_EBADCKPT (-9)    /* checkpoint file unreadable or for another grid */

/* arithmetic of the state and of the stencil (reductions are always FP64) */
#define CM_FP64 0
#define CM_FP32 1

/* form of the TVD term of Sec. 3.1 */
#define CM_TVD_DAVIS 0      /* [G(r+_k) + G(r-_{k+1})] dX_{k+1/2}: default   */
#define CM_TVD_SUM 1        /* G(r+_k + r-_{k+1}) dX_{k+1/2}: as printed     */
#define CM_TVD_OFF 2        /* no TVD term (plain MacCormack; tests only)    */

/* derivative of the TVD limiter phi(r) of Sec. 3.1 in the reverse pass */
#define CM_ADJ_PHI_EXACT 0  /* phi'(r) = 2 on 0 < 2r < 1, else 0: the derivative of the
                               discrete step wherever it exists (default) */
#define CM_ADJ_PHI_FROZEN 1 /* phi' = 0: no derivative through the ratios r (the limiter's
                               values held fixed; C(Co) still differentiated) */

/* order of the half-step sweeps L_alpha(dt/2) within one step (Sec. 3.1, Eq. time_step) */
#define CM_SPLIT_PRINTED 0   /* z, (y), x, z, (y), x: X^{n+1} = L_x L_y L_z L_x L_y L_z X^n as printed */
#define CM_SPLIT_SYMMETRIC 1 /* x, (y), z, z, (y), x: the palindrome of the same half steps */

typedef struct cm_grid {
    int ndim;       /* 2 or 3 */
    int nx, ny, nz; /* nodes; x (and y) periodic; nz counts both plates (ny ignored in 2D) */
    double aspect;  /* Gamma = L/d: the box is Gamma (x Gamma) x 1 */
    /* z-grid (Sec. 3: uniform in x, y; a tangent-hyperbolic grid in z that
     * refines the plate boundary layers).  zstretch = beta > 0 puts plane k at
     *   z_k = (1 + tanh(beta (2k/K - 1)) / tanh(beta)) / 2,  K = nz - 1
     * (the paper does not print beta); 0 = uniform planes k/K.  znodes, if not
     * NULL, gives the nz plane heights instead (host, read during cm_init only;
     * z_0 = 0 < z_1 < ... < z_K = 1 exactly).  On such a grid the z sweep is
     * written in conservative form over cells of width w_k = (z_{k+1} -
     * z_{k-1})/2 (half cells on the plates), derivatives divide by the
     * distance of the planes they use, volume averages use the trapezoid
     * rule on the planes and the plate Nusselt numbers the derivative of the
     * quadratic through three planes.  Stretched grids: single contexts (2D
     * and 3D, the adjoint included), the boxes of a batch and
     * cm_diag_noalloc. */
    double zstretch;
    const double* znodes;
} cm_grid;

typedef struct cm_params {
    double eps;          /* superadiabaticity epsilon (Sec. 2); default 0.1 */
    double D;            /* dissipation number (Sec. 2); default 0.5 */
    double cfl;          /* dt = cfl * min over nodes, directions of h/(|u|+c); default 0.5 */
    double dt_fixed;     /* > 0: use this dt instead of the CFL rule */
    double gravity;      /* factor on g = 1/eps; 1 = the paper, 0 = no gravity */
    double t_bot, t_top; /* plate temperatures; default 1 and 1 - eps - D (Sec. 2) */
    double pert_amp;     /* amplitude A of the initial temperature perturbation; default 1e-3 */
    double stokes;       /* coefficient of (div u) delta_ij in tau/mu; default -2/3 */
    unsigned long long seed; /* seed of the SplitMix64 perturbation field */
    int precision;       /* CM_FP64 or CM_FP32 */
    int tvd_form;        /* CM_TVD_* */
    int diag_every;      /* queue a diagnostics sample every n steps (0 = never) */
    int diag_capacity;   /* samples kept on the device between cm_diagnostics calls */
    void* stream;        /* cudaStream_t to queue work on (NULL = legacy default stream) */
    void* state_buf;     /* optional caller-owned device memory for the two state
                            buffers (>= cm_state_bytes bytes, 256-byte aligned);
                            NULL = the library allocates.  Must outlive cm_finalize. */
    int adj_limiter;     /* CM_ADJ_PHI_*: derivative of the TVD limiter in cm_adj_backward */
    int layout_exact;    /* FP32 2D sweeps (single box and batch): 0 (default) = fastest form,
                            reproducible bit for bit for a given segment length (cm_tuning), but a
                            node may round differently by an ulp with the segment length that the
                            timing tuner at init picks; 1 = results bit for bit independent of the
                            segment lengths (about 6% slower at 4096 x 1024).  No paper passage. */
    int split;           /* CM_SPLIT_* (default CM_SPLIT_PRINTED); single contexts and batches;
                            the adjoint takes CM_SPLIT_PRINTED only (CM_EINVAL otherwise) */
    int reserved_;       /* set to 0 */
} cm_params;

/* One diagnostics sample (Sec. 2, Eqs. volume_Nu, mean_Nu, Re), FP64.
 * Volume averages <.>_V use the trapezoid rule in z (half weight on the
 * plates) and the plain mean in x, y; T_sa = T - (1 - D z). */
typedef struct cm_diag {
    long long step;   /* steps completed when sampled */
    double t;         /* simulated time */
    double dt;        /* time step of the next step */
    double Nu;        /* 1 + Nu_conv + Nu_K */
    double Nu_conv;   /* sqrt(Ra Pr)/eps <rho u_z T_sa>_V */
    double Nu_K;      /* D sqrt(Ra Pr)/2 <rho u_z u^2>_V */
    double Nu_bot;    /* -(1/eps) d<T_sa>_A/dz at z = 0 (second-order forward difference) */
    double Nu_top;    /* same at z = 1 (second-order backward difference) */
    double Nu_bar;    /* (Nu_bot + Nu_top)/2 */
    double Re;        /* sqrt(Ra/Pr) sqrt(<u^2>_V) (instantaneous) */
    double KE;        /* <rho u^2/2>_V */
    double mass;      /* <rho>_V (conserved to round-off) */
    double energy;    /* <E>_V */
    double mach_max;  /* max |u|/c */
    int status;       /* CM_OK, or CM_ENAN if a non-finite value was met */
    int pad_;
} cm_diag;

/* Fill *p with the defaults listed in cm_params (eps, D, plate temperatures
 * and the Stokes coefficient of Sec. 2; CFL and TVD form are the readings of
 * Sec. 3.1 stated in cm_params).  Never fails for p != NULL. */
int cm_default_params(cm_params* p);

/* Bytes of device memory the two state buffers need (for cm_params.state_buf);
 * the state is the conserved vector (rho, m, E) of Sec. 3.1 in the layout of
 * cm_state_layout.  grid: host; precision: CM_FP64 or CM_FP32; bytes: host out.
 * CM_EINVAL for a bad grid or precision. */
int cm_state_bytes(const cm_grid* grid, int precision, unsigned long long* bytes);

/* Create the context and write the initial state: the
 * conduction / hydrostatic profile of constant K (T linear between the plate
 * temperatures, dp/dz = -g rho, rho(0) = 1) plus an isobaric temperature
 * perturbation A*xi at interior nodes, xi uniform in [-1, 1) from SplitMix64
 * of (seed, dense node index); u = 0.  Also computes the first dt.
 * grid, params: host (params may be NULL for the defaults).  Ra, Pr, gamma:
 * Rayleigh and Prandtl numbers and cp/cv (Sec. 2).  Returns CM_EINVAL for a
 * bad grid or parameter, CM_EUNSTABLE if the explicit diffusion number at the
 * first dt exceeds 1/2, CM_ENOMEM / CM_ECUDA on device failures. */
int cm_init(const cm_grid* grid, double Ra, double Pr, double gamma, const cm_params* params);

/* Queue n full time steps (Sec. 3.1, Eq. time_step):
 *   X^{n+1} = L_x L_y L_z L_x L_y L_z X^n, each L_alpha at dt/2 (rightmost first),
 * where L_alpha is the fused predictor / plate fill / corrector / average /
 * TVD sweep along alpha and dt comes from the state at the start of the step
 * (computed on the device by the previous step; the host never reads it).
 * Asynchronous on the context's stream.  n >= 0. */
int cm_step(int n);

/* Queue one diagnostics sample of the current state now (Sec. 2 definitions). */
int cm_sample(void);

/* Horizontal (x, y) means of the current state on every z plane, the
 * profiles of Sec. 4-5: out (host, nz x 8 doubles, plane k at out[8k..8k+7])
 * receives <rho>_A, <E>_A, <rho u_z T_sa>_A (convective heat flux),
 * <rho u_z |u|^2>_A, <|u|^2>_A, <rho |u|^2 / 2>_A, <T>_A and the plane's
 * maximum Mach number, T_sa = T - (1 - D z); sums in FP64 (FP32 states: the
 * per-node quantities in FP32).  Blocking. */
int cm_profiles(double* out);

/* Wait for the stream, then copy up to max queued samples (oldest first) to
 * out (host, max entries) and drop them; *n_out (host) receives the count.
 * Each record holds Nu (Eq. volume_Nu), Nu_0, Nu_1 and Nu_bar (Eq. mean_Nu),
 * Re (Eq. Re, instantaneous) and the budgets of Sec. 2, reduced in FP64.
 * Returns CM_ENAN if any copied sample saw a non-finite value. */
int cm_diagnostics(cm_diag* out, int max, int* n_out);

/* Device pointer to field f (0 <= f < nfields) of the current state vector
 * (Sec. 3.1: rho, m_x, (m_y,) m_z, E), or NULL if there is no context or f is
 * out of range.  Layout: see cm_state_layout.  The library owns the memory
 * unless cm_params.state_buf was given. */
void* cm_state_ptr(int field);

/* Layout of the current state on the device: element (k, j, i) of field f is
 * at cm_state_ptr(f)[(k*ny + j)*pitch + i]; elem_bytes is 8 (FP64) or 4 (FP32).
 * All arguments are host out-pointers; any may be NULL. */
int cm_state_layout(int* pitch, int* nfields, int* elem_bytes);

/* Wait for the stream and copy the current state vector (Sec. 3.1) into host
 * (dense float64, nfields*nz*ny*nx values, layout in the header comment).
 * State-sized host arrays, here and in every entry point below, are either
 * pageable memory or inside one pinned allocation; an array that spans
 * several pinned allocations (or pinned and pageable pages), which CUDA's
 * copies reject, is refused with CM_EINVAL before any transfer. */
int cm_get_state(double* host);

/* Replace the current state by host (dense float64, same layout; converted
 * to the context's precision) and recompute dt from it, in one pass.  A
 * pinned host array (cudaHostAlloc / cudaHostRegister, one mapped range) is
 * read in place over the host link by that pass; other host memory is copied
 * in plane chunks, each packed while the next is copied.  Blocking. */
int cm_set_state(const double* host);

/* Replace the current state by the initial condition of cm_init built on a
 * given temperature field: T (host, dense float64 [nz][ny][nx], read during
 * the call) at the interior planes, the plate temperatures on the plates, the
 * conduction pressure p_c(z) of each plane (rho = p_c / (a T)) and u = 0;
 * then dt is recomputed from it.  cm_init is this with T = T_c(z) + A xi.
 * Time and step count are kept.  CM_EINVAL if T is NULL or an interior value
 * is not a positive finite number.  Blocking. */
int cm_set_temperature(const double* T);

/* End-to-end call with host buffers: upload state_in (host, dense float64,
 * may be NULL to keep the device state; as cm_set_state, so pinned memory is
 * the fast path), run nsteps steps of Eq. time_step
 * (as cm_step), then write the
 * final state to state_out (host, may be NULL) and one diagnostics sample of
 * the final state to diag_out (host, may be NULL).  Blocking. */
int cm_run_host(const double* state_in, int nsteps, double* state_out, cm_diag* diag_out);

/* cm_run_host for an FP32 context with dense float32 host buffers (the
 * state's own precision: half the bytes over the host link).  CM_EINVAL on
 * an FP64 context.  Blocking. */
int cm_run_host_f32(const float* state_in, int nsteps, float* state_out, cm_diag* diag_out);

/* Queue exactly one directional sweep L_dir(Delta) (dir 0 = x, 1 = y, 2 = z)
 * on the current state (Sec. 3.1 predictor, corrector, average and TVD term),
 * without touching dt or time.  For tests of single operators. */
int cm_sweep(int dir, double Delta);

/* Wait for the stream; *dt (host) = the dt the next step will use: CFL times
 * the minimum over nodes and directions of h/(|u_alpha| + c), c^2 = gamma p/rho
 * (the paper leaves dt to the Courant condition of Sec. 3.1; this is the
 * stated reading), or dt_fixed. */
int cm_get_dt(double* dt);

/* Wait for the stream; simulated time (the sum of the steps' dt, Eq.
 * time_step) and completed steps (host out). */
int cm_get_time(double* t, long long* steps);

/* Measurement: queue n steps exactly as cm_step does, with CUDA events
 * recorded on the context's stream around every sweep launch.  Before each
 * step (outside the event brackets) a device buffer of flush_bytes is
 * overwritten with cudaMemsetAsync to evict the L2 cache (0 = no flush).
 * Waits once at the end.  ms_out (host, 4 entries in 2D: positions z, x, z,
 * x of a step; 6 in 3D: z, y, x, z, y, x) receives the mean device duration
 * in ms of the sweeps at each position; step_ms (host, n entries, may be
 * NULL) the device duration of each step.  ms_out may be NULL (then step_ms
 * may not): each step is then bracketed by two events and no event sits
 * between its sweeps, so consecutive sweeps overlap their launches as in
 * cm_step.  n >= 1. */
int cm_profile_steps(int n, unsigned long long flush_bytes, double* ms_out, double* step_ms);

/* Rows per warp segment that cm_init chose for the FP32 sweeps along z and x
 * by timing a fixed list of lengths (0 = the occupancy model: FP64, odd nx in
 * 2D, or CM_SEG_ROWS set).  The work split only; no paper passage.  Host
 * out-pointers, may be NULL. */
int cm_tuning(int* seg_z, int* seg_x);

/* Extended diagnostics of the current state (the analyses of Secs. 4-6).
 * z derivatives: of the quadratic through three planes (central on uniform
 * planes); x, y: central.  Volume averages as in cm_diag. */
typedef struct cm_ext {
    double C;          /* <rho u_z T_sa>_V / sqrt(<(rho u_z)^2>_V <T_sa^2>_V) (Eq. Corr_Ra); NaN at rest */
    double rho_uz_sq;  /* <(rho u_z)^2>_V */
    double Tsa_sq;     /* <T_sa^2>_V, T_sa = T - (1 - D z) */
    double lambda_b;   /* bottom thermal boundary layer (Sec. 4), as the tangent construction: superadiabatic
                          drop from the plate to the bulk over the plate gradient,
                          (Tb - <T_sa>_A(0)) / (d<T_sa>_A/dz at 0), Tb the trapezoid mean of <T_sa>_A
                          over 1/4 <= z <= 3/4, the plate derivative that of the plate Nusselt number */
    double lambda_top; /* the same at the top plate: (<T_sa>_A(1) - Tb) / (d<T_sa>_A/dz at 1) */
    double F_n, F_p, F_b, F_v; /* averages over the interior planes (weights of the trapezoid rule) of
                          rho (u.grad) u_z, -dp/dz, rho g and d_i tau_iz (Sec. 6, z momentum) */
    double r_max;      /* max over nodes of K_e/I_e = (rho u^2/2)/(rho C_v T) */
    double lambda_b_slope;   /* bottom layer read by the slope criterion of Sec. 4: the first distance
                                from the plate where |d<T>_A/dz + D| = |d<T_sa>_A/dz| has fallen to
                                0.1 D (slopes from the quadratic through three planes, the crossing
                                interpolated linearly between planes); NaN if it never does */
    double lambda_top_slope; /* the same from the top plate */
} cm_ext;

/* Plane means of F_n, F_p, F_b, F_v (0 on the plates), (rho u_z)^2 and
 * T_sa^2, and the vertical profiles of Sec. 4: <T_sa>_A = <T>_A - T_A(z),
 * <rho>_A - rho_A(z) with the adiabatic profiles T_A = 1 - D z and
 * rho_A = (1 - D z)^(1/(gamma-1)), and the rms velocity U(z) = sqrt(<u^2>_A):
 * out (host) receives nz x 9 doubles, plane-major.  FP64 arithmetic
 * on the state (FP32 states widened).  The first call allocates device work
 * space of 40 bytes per node (FP64 primitives), kept until cm_finalize.
 * Blocking.  CM_ENOTINIT / CM_EINVAL (out NULL) / CM_ENOMEM / CM_ECUDA. */
int cm_ext_profiles(double* out);

/* The quantities of cm_ext for the current state, and, if hist != NULL, the
 * histogram of log10 (K_e/I_e) over all nodes: hist (host, nbins counts,
 * 1 <= nbins <= 1024) counts values in [lo + q w, lo + (q+1) w), w =
 * (hi - lo)/nbins, values below lo (and nodes at rest) in bin 0, values at
 * or above hi in the last bin.  Blocking.  CM_EINVAL for out NULL, a bad
 * nbins or hi <= lo. */
int cm_extended(cm_ext* out, long long* hist, int nbins, double log10_lo, double log10_hi);

/* Copy the nz plane heights z_k of the context's z-grid (uniform, tanh or
 * given; see cm_grid) to z (host, nz doubles).  CM_ENOTINIT without a context,
 * CM_EINVAL for z = NULL. */
int cm_znodes(double* z);

/* Number of CUDA kernel launches this context has queued since cm_init
 * (measurement; no paper passage). */
long long cm_launch_count(void);

/* Wait for all queued work of the context (no paper passage). */
int cm_sync(void);

/* Write / read a checkpoint: a header {magic, version, grid, precision,
 * parameter hash, step, t} followed by the dense state in the context's
 * precision.  cm_load needs a context created with the same grid, precision
 * and parameters; it returns CM_EBADCKPT otherwise.  Blocking.  path: host. */
int cm_save(const char* path);
int cm_load(const char* path);

/* ---- Batched ensemble: many independent 2D boxes advanced together ----
 * Each box is the problem of cm_init (Sec. 2 equations, Sec. 3.1 scheme) with
 * its own grid, Ra, dt (per-box device control block), time and seed
 * (params->seed + box index).  FP32 state with FP64 dt and reductions.  One
 * kernel launch per sweep covers every box (warp work items of box, column
 * strip, row segment); the segment length of each box size class is chosen
 * at init by timing the batched sweeps (autotuner); runs of 50 steps are
 * replayed from a captured CUDA graph.  A separate context from cm_init's. */

/* nbox >= 1; grids, Ra: host arrays of nbox (2D grids, even nx); params:
 * host (precision must be CM_FP32; stream NULL = a stream the batch creates,
 * otherwise a stream that can be captured).  Each box gets the initial state
 * of cm_init (seed + box index) and is advanced by Eq. time_step (Sec. 3.1)
 * with its own dt.  A box may have a stretched z-grid (zstretch or znodes,
 * read during this call only, as in cm_init); then every box of the batch is
 * stepped by the stretched-grid sweeps, a uniform box with the plane table
 * of its planes k/K (the result of cm_init with znodes = k/K).  CM_EINVAL for
 * an odd nx, an FP64 precision or a bad grid (before any device work);
 * CM_EUNSTABLE if a box's explicit diffusion number at its first dt is above
 * 1/2 (the bound of cm_init; the message names the box).  Blocking. */
int cm_batch_init(int nbox, const cm_grid* grids, const double* Ra, double Pr, double gamma, const cm_params* params);

/* Queue n steps (Eq. time_step) of every box (asynchronous). */
int cm_batch_step(int n);

/* One diagnostics sample of every box now (Sec. 2 definitions); out: host,
 * nbox records.  Blocking.  CM_ENAN if a box met a non-finite value. */
int cm_batch_diagnostics(cm_diag* out);

/* Dense float64 state of one box (layout of cm_get_state); host out.  Blocking. */
int cm_batch_get_state(int box, double* host);

/* Segment lengths the autotuner chose per box for the z and x sweeps (host
 * arrays of nbox; either may be NULL). */
int cm_batch_tuning(int* seg_z, int* seg_x);

/* Measurement: L2 flush of flush_bytes (0 = none), then n steps bracketed by
 * CUDA events on the batch stream; *total_ms (host) = their device time. */
int cm_batch_profile_steps(int n, unsigned long long flush_bytes, double* total_ms);

/* Kernel launches the batch has queued since cm_batch_init. */
long long cm_batch_launch_count(void);

/* Free the batch context. */
int cm_batch_finalize(void);

/* Diagnostics of a caller's state with no allocation at all.  The paper has
 * no counterpart: this entry point exists for callers that must not allocate
 * device memory, e.g. an in-situ analysis hook called from another
 * application's time loop, whose memory pool owns the device memory and where
 * a cudaMalloc could fail or synchronise the device under the host's streams.
 * Computes the same record as cm_sample without a context: the scratch lives
 * in a fixed ~2.8 MB __device__ array inside the library, so nz may not
 * exceed 16384 planes (CM_EINVAL beyond).  The array is device memory of
 * the library's module: it is placed on a device when the module is loaded
 * there, which under CUDA's default lazy loading is the first call of this
 * entry point on that device (CUDA_MODULE_LOADING=EAGER: when the library's
 * first CUDA call creates the context); it stays until the process exits.
 * A host whose pool claims most of HBM should therefore make one call (or
 * load the library eagerly) during its setup, before the pool grows.  That
 * first call on a device also looks up the array's device address; make it
 * before any stream capture.  A stretched grid (zstretch or znodes, as for
 * cm_init) gets its plane table built in host memory and copied into that
 * array (the stretched-grid weights of cm_sample).
 * All calls share the array: calls that overlap on the GPU race.
 * state: device pointer to field 0 of a state in the layout of
 *   cm_state_layout (fields nz*ny*pitch elements apart), precision CM_FP64 or
 *   CM_FP32; grid, params: host; t, dt, step: copied into the record;
 * stream: cudaStream_t (NULL = legacy default); out: host.  Blocking. */
int cm_diag_noalloc(const void* state, int precision, const cm_grid* grid, int pitch, double Ra, double Pr,
                    double gamma, const cm_params* params, double t, double dt, long long step, void* stream,
                    cm_diag* out);

/* ---- Adjoint: gradients of a time-averaged plate Nusselt number ----
 * J = (1/N_w) sum over steps n = win_begin..nsteps of Nu_bar(X^n), Nu_bar =
 * (Nu_0 + Nu_1)/2 of Eq. mean_Nu (second-order one-sided plate differences
 * of the plane-averaged temperature, as cm_diag.Nu_bar; on a stretched grid
 * the derivative of the quadratic through three planes), X^n the state after
 * step n of the run started by cm_adj_forward.  Each step's dt is a constant
 * of J (the CFL dt the forward run took; dt is not differentiated).
 * Reverse mode of Sec. 3.1's sweeps, hand-written, with non-smooth points
 * taking fixed one-sided derivatives: phi'(r) = 2 on 0 < 2r < 1 else 0,
 * d|u|/du = 0 at u = 0, the Co(1 - Co) branch at Co = 1/2, and on a tie in
 * max(A_k, A_k+1) the first argument.  2D FP64 contexts only (CM_EINVAL
 * otherwise), uniform or stretched z-grid.
 * The limiter's ratio r = <dX_-, dX_+>/<dX_+, dX_+> over the conserved
 * components is not Lipschitz in X (where dX_+ -> 0 and dX_- is not parallel
 * to it), so the exact derivative (cm_params.adj_limiter = CM_ADJ_PHI_EXACT)
 * of a long run can grow far beyond the response of J to any finite change;
 * CM_ADJ_PHI_FROZEN (phi' = 0) drops the derivative through r and stays
 * bounded.  The reading is taken from the context's cm_params at
 * cm_adj_backward. */

/* Replay: the next cm_adj_forward runs of exactly n steps take step s's dt
 * from dts[s] (host, n values > 0, copied) instead of the CFL rule or
 * dt_fixed, so that a run from a perturbed state or at another Ra (a finite
 * difference of J) uses the dts of the run it is compared with.  n = 0 (dts
 * may be NULL) clears it.  CM_EINVAL for n < 0 or a dt that is not a positive
 * finite number. */
int cm_adj_set_dts(const double* dts, int n);

/* The dt of each step of the last cm_adj_forward (host out, n values; n must
 * equal its nsteps).  CM_EINVAL otherwise. */
int cm_adj_get_dts(double* dts, int n);

/* Run nsteps steps from the current state (advancing it, t and the step
 * count as cm_step does), record each step's dt, keep a device copy of the
 * state every K steps (ceil(nsteps/K) states), and write J (host) once the
 * run is done.  1 <= win_begin <= nsteps.  Blocking.  The reverse pass later
 * holds 4K+1 more states and recomputes each K-step segment: K trades memory
 * for recomputation.  K = 0 keeps every sweep input of this run instead
 * (4 nsteps + 1 states, e.g. 67 GB for 2000 steps of 1024 x 256) and the
 * reverse pass recomputes nothing.  The diagnostics ring is not sampled
 * during a K = 0 run. */
int cm_adj_forward(int nsteps, int K, int win_begin, double* J);

/* Reverse pass of the last cm_adj_forward: recompute each K-step segment
 * from its checkpoint (same kernels, same dt: bit-identical states; nothing
 * to recompute when K = 0), then apply the vector-Jacobian products of the
 * sweeps in reverse order.
 * Outputs (each may be NULL; host or device pointers):
 *   grad_X0  dJ/dX^0, dense float64 in the cm_get_state layout (4 fields);
 *   grad_T0  dJ/dT at the interior nodes of X^0 for a temperature change at
 *            fixed pressure and velocity (the isobaric perturbation of the
 *            initial condition), dense float64 [nz][nx], 0 on the plates;
 *   grad_Ra  dJ/dRa through mu = sqrt(Pr/Ra) and K = 1/(eps D sqrt(Ra Pr)).
 * Blocking; may be called again (it recomputes from the checkpoints). */
int cm_adj_backward(double* grad_X0, double* grad_T0, double* grad_Ra);

/* Free the context and its device memory (not caller-owned state_buf). */
int cm_finalize(void);

/* Message of the last failure (static storage; never NULL). */
const char* cm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CM_H */
