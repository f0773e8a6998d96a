/*
 * cm_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU implementation of the explicit MacCormack
 * predictor-corrector step with TVD correction for the nondimensional fully
 * compressible Navier-Stokes-energy equations of arXiv 2411.10372
 * (Tiwari, Sharma & Verma), plus the Nusselt / Reynolds diagnostics.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * leg may load this library.  The product path (paper_2411_10372_gb300) never
 * calls it; the two share no code, headers or tables.
 *
 * Everything is written as separate whole-grid arrays (X, F, X^P, F^P, X^C,
 * TVD fluxes) and plain nested loops, in the order the paper states the
 * scheme, so that it can be checked against the paper by eye.
 *
 * The per-node loops of a sweep carry "omp parallel for" pragmas: every
 * iteration writes its own nodes only, so a build with -fopenmp (the all-cores
 * CPU baseline) computes the same values bit for bit; the default build
 * ignores them.  Reductions (dt, diagnostics) stay serial.
 *
 * Passages followed (paper sections / equations):
 *   Sec. 2, nondimensional continuity / momentum / energy equations and the
 *     closures for p, E and tau ........................ prims(), flux()
 *   Sec. 2, Eq. volume_Nu (bulk Nu), Eq. mean_Nu (plate Nu), Eq. Re ... orc_diag()
 *   Sec. 3.1, vector form X_t + sum_a dF_a/dx_a = sum_a S_a ........ flux()
 *   Sec. 3.1, Eq. time_step (operator splitting) ................... orc_step()
 *   Sec. 3.1, predictor / corrector / average + TVD term, limiter G,
 *     minmod phi, coefficient C(Co) ........................ sweep_z(), sweep_h()
 *   Sec. 3.1, "second-order forward and backward differences at the
 *     plates" ................................................ orc_diag() (plate Nu)
 *
 * Readings where the paper is silent, ambiguous or garbled (each pinned by
 * the tests named in oracle/__init__.py):
 *   - stress tensor: the divergence term enters with coefficient cfg->stokes
 *     (default -2/3, Stokes' hypothesis; the paper prints +2/3);
 *   - corrector uses F^P at both k+1 and k (the printed F^(n)_{k+1} is
 *     inconsistent);
 *   - pressure sits in the alpha-momentum row of F_alpha (p delta_{i alpha});
 *   - derivatives inside F: along the sweep direction forward in the
 *     predictor and backward in the corrector, cross derivatives central;
 *   - TVD: cfg->tvd_form selects G(r+)+G(r-) (Davis form, default, chosen
 *     by the total-variation test) or the literal G(r+ + r-), or none;
 *   - plates: no-slip, fixed temperature; plate density advanced as a half
 *     cell with zero wall mass flux; TVD fluxes through the two interfaces
 *     next to each plate are zero; horizontal sweeps leave plate rows alone;
 *   - time step dt = cfl * min over nodes and directions of h/(|u|+c), from
 *     the state at the start of the step; local Courant number of interface
 *     k+1/2 uses the larger |u|+c of its two nodes and the sweep's dt/2;
 *   - initial state: exact conduction/hydrostatic profile for constant K,
 *     isobaric temperature perturbation at interior nodes;
 *   - the tanh z-grid (Sec. 3 names it, without its formula or stretching):
 *     z_k = (1 + tanh(beta (2k/K - 1))/tanh(beta))/2, or any given planes;
 *     the z flux differences are conservative over cells of width w_k, the
 *     derivatives inside F divide by the distance of the planes they use,
 *     the TVD flux of an interface is weighted by its spacing over w_k, the
 *     CFL step uses the smaller spacing next to a plane, and the plate
 *     derivative is that of the quadratic through three planes.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- configuration (mirrored by oracle/__init__.py, field for field) ---- */
typedef struct {
    int ndim;            /* 2 or 3 */
    int nx, ny, nz;      /* nodes; ny = 1 in 2D; nz counts both plates */
    int tvd_form;        /* 0: G(r+)+G(r-), 1: G(r+ + r-), 2: no TVD term */
    int split;           /* 0: Eq. time_step as printed; 1: the palindrome of its half steps */
    double aspect;       /* Gamma = L/d */
    double Ra, Pr, gamma, eps, D;
    double cfl;          /* dt = cfl * min h/(|u|+c) */
    double dt_fixed;     /* > 0 overrides the CFL rule */
    double gravity;      /* multiplies g = 1/eps (1 = the paper) */
    double t_bot, t_top; /* plate temperatures (paper: 1 and 1-eps-D) */
    double pert_amp;     /* amplitude of the temperature perturbation */
    double stokes;       /* coefficient of (div u) delta_ij inside tau/mu */
    uint64_t seed;
    double zstretch;     /* beta of the tanh z-grid; 0 = uniform planes */
    const double* znodes; /* optional: the nz plane heights (0 .. 1), overriding zstretch */
} orc_cfg;

/* derived constants */
typedef struct {
    int ndim, nx, ny, nz, tvd_form, split;
    size_t n;
    double h[3];         /* dx, dy, dz */
    double a;            /* p = a rho T,        a = (gamma-1)/(gamma eps D) */
    double b;            /* T = b (E/rho - u^2/2 - g z), b = gamma eps D     */
    double g;            /* gravity / eps                                    */
    double mu;           /* sqrt(Pr/Ra)                                      */
    double kth;          /* 1/(eps D sqrt(Ra Pr))                            */
    double stokes, gam;
    double t_bot, t_top;
    double cfl, dt_fixed;
    double Ra, Pr, eps, D, aspect;
    /* z-grid (Sec. 3: tanh planes in z, uniform in x and y).  z[k]: height of
     * plane k; hp[k] = z[k+1] - z[k], the spacing above plane k; w[k]: the
     * width of plane k's cell, (hp[k-1] + hp[k])/2 inside and hp/2 on the
     * plates (so that sum_k w[k] = 1 and the trapezoid rule in z is
     * sum_k w[k] f_k).  On the uniform grid hp = dz and w = dz, dz/2 exactly. */
    int stretched;
    double *z, *hp, *w;
} P;

/* plane k of the tanh grid with nz - 1 = K intervals:
 * z_k = (1 + tanh(beta (2k/K - 1)) / tanh(beta)) / 2, plates exactly 0 and 1 */
static double tanh_plane(double beta, int k, int K)
{
    if (k == 0) return 0.0;
    if (k == K) return 1.0;
    double s = 2.0 * k / K - 1.0;
    return 0.5 * (1.0 + tanh(beta * s) / tanh(beta));
}

static void derive(const orc_cfg* c, P* p)
{
    p->ndim = c->ndim;
    p->nx = c->nx;
    p->ny = (c->ndim == 3) ? c->ny : 1;
    p->nz = c->nz;
    p->tvd_form = c->tvd_form;
    p->split = c->split;
    p->n = (size_t)p->nx * p->ny * p->nz;
    p->h[0] = c->aspect / c->nx;
    p->h[1] = c->aspect / p->ny;
    p->h[2] = 1.0 / (c->nz - 1);
    p->gam = c->gamma;
    p->a = (c->gamma - 1.0) / (c->gamma * c->eps * c->D);
    p->b = c->gamma * c->eps * c->D;
    p->g = c->gravity / c->eps;
    p->mu = sqrt(c->Pr / c->Ra);
    p->kth = 1.0 / (c->eps * c->D * sqrt(c->Ra * c->Pr));
    p->stokes = c->stokes;
    p->t_bot = c->t_bot;
    p->t_top = c->t_top;
    p->cfl = c->cfl;
    p->dt_fixed = c->dt_fixed;
    p->Ra = c->Ra; p->Pr = c->Pr; p->eps = c->eps; p->D = c->D;
    p->aspect = c->aspect;

    int nz = c->nz, K = nz - 1;
    p->stretched = c->znodes != NULL || c->zstretch != 0.0;
    p->z = malloc(nz * sizeof(double));
    p->hp = malloc(nz * sizeof(double));
    p->w = malloc(nz * sizeof(double));
    for (int k = 0; k < nz; k++) {
        if (c->znodes) p->z[k] = c->znodes[k];
        else if (c->zstretch != 0.0) p->z[k] = tanh_plane(c->zstretch, k, K);
        else p->z[k] = (double)k / (double)K;
    }
    if (!p->stretched) {
        for (int k = 0; k < nz; k++) {
            p->hp[k] = p->h[2];
            p->w[k] = (k == 0 || k == K) ? p->h[2] / 2.0 : p->h[2];
        }
    } else {
        for (int k = 0; k < K; k++) p->hp[k] = p->z[k + 1] - p->z[k];
        p->hp[K] = p->hp[K - 1]; /* never used */
        p->w[0] = p->hp[0] / 2.0;
        p->w[K] = p->hp[K - 1] / 2.0;
        for (int k = 1; k < K; k++) p->w[k] = (p->hp[k - 1] + p->hp[k]) / 2.0;
    }
}

static void release(P* p)
{
    free(p->z); free(p->hp); free(p->w);
}

/* z of plane k: nodes on both plates, z_0 = 0 and z_{nz-1} = 1 */
static double zk(const P* p, int k) { return p->z[k]; }

/* smallest spacing next to plane k, the z step of the CFL rule there */
static double hmin_z(const P* p, int k)
{
    int K = p->nz - 1;
    if (k == 0) return p->hp[0];
    if (k == K) return p->hp[K - 1];
    return fmin(p->hp[k - 1], p->hp[k]);
}

static size_t idx(const P* p, int i, int j, int k)
{
    return ((size_t)k * p->ny + j) * p->nx + i;
}

/* neighbour of (i,j,k) one step along direction d (s = +1 or -1);
 * x and y are periodic, z is only asked for interior neighbours. */
static size_t nbr(const P* p, int i, int j, int k, int d, int s)
{
    if (d == 0) i = (i + s + p->nx) % p->nx;
    else if (d == 1) j = (j + s + p->ny) % p->ny;
    else k = k + s;
    return idx(p, i, j, k);
}

/* Internal state: 5 components (rho, m_x, m_y, m_z, E), component c of node n
 * at X[c*N + n].  In 2D m_y stays identically zero. */

/* Primitive variables from the closures of Sec. 2:
 * u = m/rho, T = gamma eps D (E/rho - u^2/2 - z/eps), p = (gamma-1)/(gamma eps D) rho T */
static void prims(const P* p, const double* X, double* U, double* T, double* Pr)
{
    size_t N = p->n;
    #pragma omp parallel for
    for (int k = 0; k < p->nz; k++)
        for (int j = 0; j < p->ny; j++)
            for (int i = 0; i < p->nx; i++) {
                size_t n = idx(p, i, j, k);
                double rho = X[n];
                double u = X[1 * N + n] / rho;
                double v = X[2 * N + n] / rho;
                double w = X[3 * N + n] / rho;
                U[0 * N + n] = u;
                U[1 * N + n] = v;
                U[2 * N + n] = w;
                T[n] = p->b * (X[4 * N + n] / rho - 0.5 * (u * u + v * v + w * w) - p->g * zk(p, k));
                Pr[n] = p->a * rho * T[n];
            }
}

/* Velocity and temperature gradients at node (i,j,k) for a sweep along al:
 * along al a one-sided difference (forward if fwd, else backward), across
 * al central differences.  du[c][d] = d u_c / d x_d.  In z every difference
 * is divided by the distance between the two planes it uses (exact for a
 * linear profile on any grid). */
static void grad(const P* p, const double* U, const double* T, int i, int j, int k,
                 int al, int fwd, double du[3][3], double dT[3])
{
    size_t N = p->n;
    size_t self = idx(p, i, j, k);
    for (int d = 0; d < 3; d++) {
        size_t np, nm;
        double span;
        if (d == al) {
            np = fwd ? nbr(p, i, j, k, d, +1) : self;
            nm = fwd ? self : nbr(p, i, j, k, d, -1);
            span = (d == 2) ? (fwd ? p->hp[k] : p->hp[k - 1]) : p->h[d];
        } else {
            np = nbr(p, i, j, k, d, +1);
            nm = nbr(p, i, j, k, d, -1);
            span = (d == 2) ? p->hp[k - 1] + p->hp[k] : 2.0 * p->h[d];
        }
        for (int c = 0; c < 3; c++)
            du[c][d] = (U[c * N + np] - U[c * N + nm]) / span;
        dT[d] = (T[np] - T[nm]) / span;
    }
}

/* Flux F_al of Sec. 3.1 at one node:
 *   [ rho u_al ;
 *     m_i u_al - tau_{i al} + p delta_{i al}  (i = x, y, z) ;
 *     u_al (E + p) - K dT/dx_al - sum_b u_b tau_{b al} ]
 * with tau_ij = mu (d_j u_i + d_i u_j + stokes (div u) delta_ij). */
static void flux(const P* p, int al, const double q[5], const double u[3], double pr,
                 double du[3][3], const double dT[3], double F[5])
{
    double div = du[0][0] + du[1][1] + du[2][2];
    double tau[3];
    for (int i = 0; i < 3; i++)
        tau[i] = p->mu * (du[i][al] + du[al][i] + (i == al ? p->stokes * div : 0.0));
    F[0] = q[1 + al];
    for (int i = 0; i < 3; i++)
        F[1 + i] = q[1 + i] * u[al] - tau[i] + (i == al ? pr : 0.0);
    double work = u[0] * tau[0] + u[1] * tau[1] + u[2] * tau[2];
    F[4] = u[al] * (q[4] + pr) - p->kth * dT[al] - work;
}

static void node_flux(const P* p, int al, int fwd, const double* X, const double* U,
                      const double* T, const double* Pr, int i, int j, int k, double F[5])
{
    size_t N = p->n, n = idx(p, i, j, k);
    double q[5], u[3], du[3][3], dT[3];
    for (int c = 0; c < 5; c++) q[c] = X[c * N + n];
    for (int c = 0; c < 3; c++) u[c] = U[c * N + n];
    grad(p, U, T, i, j, k, al, fwd, du, dT);
    flux(p, al, q, u, Pr[n], du, dT, F);
}

/* ---- TVD limiter (Sec. 3.1) ---- */
static double phi_minmod(double r) { return fmax(0.0, fmin(2.0 * r, 1.0)); }
static double coefC(double Co) { return Co <= 0.5 ? Co * (1.0 - Co) : 0.25; }
static double Gfun(double r, double C) { return 0.5 * C * (1.0 - phi_minmod(r)); }

/* TVD flux through the interface between nodes n0 and n1 = n0 + e_al, with
 * nm = n0 - e_al and n2 = n1 + e_al, from the sweep's INPUT state X:
 *   D = [G(r+_{n0}) + G(r-_{n1})] dX_{n0+1/2}   (tvd_form 0)
 *   D =  G(r+_{n0} + r-_{n1})     dX_{n0+1/2}   (tvd_form 1)
 * r+_{n0} = (dX_{n0-1/2}, dX_{n0+1/2}) / (dX_{n0+1/2}, dX_{n0+1/2})
 * r-_{n1} = (dX_{n0+1/2}, dX_{n0+3/2}) / (dX_{n0+1/2}, dX_{n0+1/2})
 * Co = (dt/2) max(|u_al|+c over n0, n1) / h, h the spacing of the interface. */
static void tvd_flux(const P* p, const double* X, const double* A, double Delta, double h,
                     size_t nm, size_t n0, size_t n1, size_t n2, double D[5])
{
    size_t N = p->n;
    double dm[5], d0[5], dp[5];
    for (int c = 0; c < 5; c++) {
        dm[c] = X[c * N + n0] - X[c * N + nm];
        d0[c] = X[c * N + n1] - X[c * N + n0];
        dp[c] = X[c * N + n2] - X[c * N + n1];
    }
    double s_plus = 0.0, s_minus = 0.0, dd = 0.0;
    for (int c = 0; c < 5; c++) {
        s_plus += dm[c] * d0[c];
        s_minus += d0[c] * dp[c];
        dd += d0[c] * d0[c];
    }
    for (int c = 0; c < 5; c++) D[c] = 0.0;
    if (p->tvd_form == 2 || dd == 0.0) return;
    double rp = s_plus / dd, rm = s_minus / dd;
    double Co = Delta * fmax(A[n0], A[n1]) / h;
    double C = coefC(Co);
    double G = (p->tvd_form == 0) ? Gfun(rp, C) + Gfun(rm, C) : Gfun(rp + rm, C);
    for (int c = 0; c < 5; c++) D[c] = G * d0[c];
}

/* |u_al| + c at every node, c^2 = gamma p / rho = gamma a T */
static void wave_speed(const P* p, int al, const double* U, const double* T, double* A)
{
    size_t N = p->n;
    #pragma omp parallel for
    for (size_t n = 0; n < N; n++) A[n] = fabs(U[al * N + n]) + sqrt(p->gam * p->a * T[n]);
}

typedef struct {
    double *U, *T, *Pr, *A, *F, *XP, *UP, *TP, *PP, *FP, *XC, *D;
} Work;

static void work_alloc(const P* p, Work* w)
{
    size_t N = p->n;
    w->U = malloc(3 * N * sizeof(double));
    w->T = malloc(N * sizeof(double));
    w->Pr = malloc(N * sizeof(double));
    w->A = malloc(N * sizeof(double));
    w->F = calloc(5 * N, sizeof(double));
    w->XP = malloc(5 * N * sizeof(double));
    w->UP = malloc(3 * N * sizeof(double));
    w->TP = malloc(N * sizeof(double));
    w->PP = malloc(N * sizeof(double));
    w->FP = calloc(5 * N, sizeof(double));
    w->XC = malloc(5 * N * sizeof(double));
    w->D = calloc(5 * N, sizeof(double));
}

static void work_free(Work* w)
{
    free(w->U); free(w->T); free(w->Pr); free(w->A); free(w->F); free(w->XP);
    free(w->UP); free(w->TP); free(w->PP); free(w->FP); free(w->XC); free(w->D);
}

/* Plate values: no slip (m = 0) and fixed temperature T_w, so
 * E = rho (T_w / (gamma eps D) + z_w / eps). */
static void set_plate(const P* p, double* X, size_t n, int top)
{
    size_t N = p->n;
    double Tw = top ? p->t_top : p->t_bot;
    double zw = top ? 1.0 : 0.0;
    X[1 * N + n] = 0.0;
    X[2 * N + n] = 0.0;
    X[3 * N + n] = 0.0;
    X[4 * N + n] = X[n] * (Tw / p->b + p->g * zw);
}

/* L_z(Delta): one predictor-corrector-TVD sweep along z (Sec. 3.1), in the
 * conservative form of a non-uniform grid: plane k is a cell of width w[k],
 * so the flux differences of the predictor and corrector are divided by
 * w[k] and the TVD flux through interface k+1/2, a difference over hp[k], is
 * scaled by hp[k]/w[k].  On the uniform grid every ratio is exactly 1 and
 * Delta/w[k] is Delta/dz (2 Delta/dz on the plates). */
static void sweep_z(const P* p, double Delta, const double* X, double* Y, Work* w)
{
    size_t N = p->n;
    int nz = p->nz, K = nz - 1;

    prims(p, X, w->U, w->T, w->Pr);
    wave_speed(p, 2, w->U, w->T, w->A);

    /* predictor fluxes F^n_k, k = 0..nz-2 (forward z-derivatives) */
    #pragma omp parallel for
    for (int k = 0; k < K; k++)
        for (int j = 0; j < p->ny; j++)
            for (int i = 0; i < p->nx; i++) {
                double F[5];
                node_flux(p, 2, 1, X, w->U, w->T, w->Pr, i, j, k, F);
                size_t n = idx(p, i, j, k);
                for (int c = 0; c < 5; c++) w->F[c * N + n] = F[c];
            }
    /* predictor at interior nodes: X^P = X - (Delta/w_k)(F_k - F_{k-1}) + Delta S,
     * S = (0, 0, 0, -g rho, 0) */
    #pragma omp parallel for
    for (int k = 1; k < K; k++)
        for (int j = 0; j < p->ny; j++)
            for (int i = 0; i < p->nx; i++) {
                double lam = Delta / p->w[k];
                size_t n = idx(p, i, j, k), nm = idx(p, i, j, k - 1);
                for (int c = 0; c < 5; c++) {
                    double S = (c == 3) ? -p->g * X[n] : 0.0;
                    w->XP[c * N + n] = X[c * N + n] - lam * (w->F[c * N + n] - w->F[c * N + nm]) + Delta * S;
                }
            }
    /* plates: half cell with zero wall mass flux; m = 0; T = T_w */
    for (int j = 0; j < p->ny; j++)
        for (int i = 0; i < p->nx; i++) {
            size_t n0 = idx(p, i, j, 0), nK = idx(p, i, j, K), nK1 = idx(p, i, j, K - 1);
            w->XP[n0] = X[n0] - (Delta / p->w[0]) * w->F[n0];
            w->XP[nK] = X[nK] + (Delta / p->w[K]) * w->F[nK1];
            set_plate(p, w->XP, n0, 0);
            set_plate(p, w->XP, nK, 1);
        }

    prims(p, w->XP, w->UP, w->TP, w->PP);

    /* corrector fluxes F^P_k, k = 1..nz-1 (backward z-derivatives) */
    #pragma omp parallel for
    for (int k = 1; k < nz; k++)
        for (int j = 0; j < p->ny; j++)
            for (int i = 0; i < p->nx; i++) {
                double F[5];
                node_flux(p, 2, 0, w->XP, w->UP, w->TP, w->PP, i, j, k, F);
                size_t n = idx(p, i, j, k);
                for (int c = 0; c < 5; c++) w->FP[c * N + n] = F[c];
            }
    /* corrector at interior nodes: X^C = X - (Delta/w_k)(F^P_{k+1} - F^P_k) + Delta S^P;
     * then the average (X^P + X^C)/2 */
    #pragma omp parallel for
    for (int k = 1; k < K; k++)
        for (int j = 0; j < p->ny; j++)
            for (int i = 0; i < p->nx; i++) {
                double lam = Delta / p->w[k];
                size_t n = idx(p, i, j, k), np = idx(p, i, j, k + 1);
                for (int c = 0; c < 5; c++) {
                    double S = (c == 3) ? -p->g * w->XP[n] : 0.0;
                    w->XC[c * N + n] = X[c * N + n] - lam * (w->FP[c * N + np] - w->FP[c * N + n]) + Delta * S;
                    Y[c * N + n] = (w->XP[c * N + n] + w->XC[c * N + n]) / 2.0;
                }
            }
    /* plate densities: corrector half cells, then average */
    for (int j = 0; j < p->ny; j++)
        for (int i = 0; i < p->nx; i++) {
            size_t n0 = idx(p, i, j, 0), n1 = idx(p, i, j, 1), nK = idx(p, i, j, K);
            double rc0 = X[n0] - (Delta / p->w[0]) * w->FP[n1];
            double rcK = X[nK]; /* F^P at the top plate is m_z = 0 */
            Y[n0] = (w->XP[n0] + rc0) / 2.0;
            Y[nK] = (w->XP[nK] + rcK) / 2.0;
        }

    /* TVD fluxes D_{k+1/2} for k = 1..nz-3 (zero at the two plate-adjacent interfaces) */
    memset(w->D, 0, 5 * N * sizeof(double));
    #pragma omp parallel for
    for (int k = 1; k <= nz - 3; k++)
        for (int j = 0; j < p->ny; j++)
            for (int i = 0; i < p->nx; i++) {
                double D[5];
                tvd_flux(p, X, w->A, Delta, p->hp[k], idx(p, i, j, k - 1), idx(p, i, j, k),
                         idx(p, i, j, k + 1), idx(p, i, j, k + 2), D);
                size_t n = idx(p, i, j, k);
                for (int c = 0; c < 5; c++) w->D[c * N + n] = D[c];
            }
    /* X^{new} = (X^P + X^C)/2 + ((hp_k/w_k) D_{k+1/2} - (hp_{k-1}/w_k) D_{k-1/2}) */
    #pragma omp parallel for
    for (int k = 1; k < K; k++) {
        double rp = p->hp[k] / p->w[k], rm = p->hp[k - 1] / p->w[k];
        for (int j = 0; j < p->ny; j++)
            for (int i = 0; i < p->nx; i++) {
                size_t n = idx(p, i, j, k), nm = idx(p, i, j, k - 1);
                for (int c = 0; c < 5; c++)
                    Y[c * N + n] = Y[c * N + n] + (rp * w->D[c * N + n] - rm * w->D[c * N + nm]);
            }
    }
    for (int j = 0; j < p->ny; j++)
        for (int i = 0; i < p->nx; i++) {
            set_plate(p, Y, idx(p, i, j, 0), 0);
            set_plate(p, Y, idx(p, i, j, K), 1);
        }
}

/* L_x(Delta) or L_y(Delta): a periodic horizontal sweep on the interior
 * rows; the plate rows pass through unchanged (no mass flux along a no-slip
 * wall). */
static void sweep_h(const P* p, int al, double Delta, const double* X, double* Y, Work* w)
{
    size_t N = p->n;
    int nz = p->nz, K = nz - 1;
    double lam = Delta / p->h[al];

    prims(p, X, w->U, w->T, w->Pr);
    wave_speed(p, al, w->U, w->T, w->A);

    #pragma omp parallel for
    for (int k = 1; k < K; k++)
        for (int j = 0; j < p->ny; j++)
            for (int i = 0; i < p->nx; i++) {
                double F[5];
                node_flux(p, al, 1, X, w->U, w->T, w->Pr, i, j, k, F);
                size_t n = idx(p, i, j, k);
                for (int c = 0; c < 5; c++) w->F[c * N + n] = F[c];
            }
    memcpy(w->XP, X, 5 * N * sizeof(double));
    #pragma omp parallel for
    for (int k = 1; k < K; k++)
        for (int j = 0; j < p->ny; j++)
            for (int i = 0; i < p->nx; i++) {
                size_t n = idx(p, i, j, k), nm = nbr(p, i, j, k, al, -1);
                for (int c = 0; c < 5; c++)
                    w->XP[c * N + n] = X[c * N + n] - lam * (w->F[c * N + n] - w->F[c * N + nm]);
            }

    prims(p, w->XP, w->UP, w->TP, w->PP);

    #pragma omp parallel for
    for (int k = 1; k < K; k++)
        for (int j = 0; j < p->ny; j++)
            for (int i = 0; i < p->nx; i++) {
                double F[5];
                node_flux(p, al, 0, w->XP, w->UP, w->TP, w->PP, i, j, k, F);
                size_t n = idx(p, i, j, k);
                for (int c = 0; c < 5; c++) w->FP[c * N + n] = F[c];
            }
    memcpy(Y, X, 5 * N * sizeof(double));
    #pragma omp parallel for
    for (int k = 1; k < K; k++)
        for (int j = 0; j < p->ny; j++)
            for (int i = 0; i < p->nx; i++) {
                size_t n = idx(p, i, j, k), np = nbr(p, i, j, k, al, +1);
                for (int c = 0; c < 5; c++) {
                    w->XC[c * N + n] = X[c * N + n] - lam * (w->FP[c * N + np] - w->FP[c * N + n]);
                    Y[c * N + n] = (w->XP[c * N + n] + w->XC[c * N + n]) / 2.0;
                }
            }
    /* TVD flux D at interface n+1/2 stored at n; all interfaces of interior rows */
    #pragma omp parallel for
    for (int k = 1; k < K; k++)
        for (int j = 0; j < p->ny; j++)
            for (int i = 0; i < p->nx; i++) {
                size_t n0 = idx(p, i, j, k);
                size_t nm = nbr(p, i, j, k, al, -1);
                size_t n1 = nbr(p, i, j, k, al, +1);
                int i1 = (al == 0) ? (i + 1) % p->nx : i;
                int j1 = (al == 1) ? (j + 1) % p->ny : j;
                size_t n2 = nbr(p, i1, j1, k, al, +1);
                double D[5];
                tvd_flux(p, X, w->A, Delta, p->h[al], nm, n0, n1, n2, D);
                for (int c = 0; c < 5; c++) w->D[c * N + n0] = D[c];
            }
    #pragma omp parallel for
    for (int k = 1; k < K; k++)
        for (int j = 0; j < p->ny; j++)
            for (int i = 0; i < p->nx; i++) {
                size_t n = idx(p, i, j, k), nm = nbr(p, i, j, k, al, -1);
                for (int c = 0; c < 5; c++)
                    Y[c * N + n] = Y[c * N + n] + (w->D[c * N + n] - w->D[c * N + nm]);
            }
}

/* ---- conversion between the external layout and the 5-component one ----
 * external 2D: [rho, m_x, m_z, E]; external 3D: [rho, m_x, m_y, m_z, E];
 * field f is the contiguous block f*N .. f*N+N-1, node index ((k*ny)+j)*nx+i */
static void to_internal(const P* p, const double* ext, double* X)
{
    size_t N = p->n;
    if (p->ndim == 3) { memcpy(X, ext, 5 * N * sizeof(double)); return; }
    memcpy(X, ext, 2 * N * sizeof(double));
    memset(X + 2 * N, 0, N * sizeof(double));
    memcpy(X + 3 * N, ext + 2 * N, 2 * N * sizeof(double));
}

static void to_external(const P* p, const double* X, double* ext)
{
    size_t N = p->n;
    if (p->ndim == 3) { memcpy(ext, X, 5 * N * sizeof(double)); return; }
    memcpy(ext, X, 2 * N * sizeof(double));
    memcpy(ext + 2 * N, X + 3 * N, 2 * N * sizeof(double));
}

/* ---- time step ---- */
static double dt_of(const P* p, const double* X, Work* w)
{
    if (p->dt_fixed > 0.0) return p->dt_fixed;
    prims(p, X, w->U, w->T, w->Pr);
    size_t N = p->n;
    double best = INFINITY;
    for (size_t n = 0; n < N; n++) {
        double c = sqrt(p->gam * p->a * w->T[n]);
        int k = (int)(n / ((size_t)p->nx * p->ny));
        for (int d = 0; d < 3; d++) {
            if (d == 1 && p->ndim == 2) continue;
            double h = (d == 2) ? hmin_z(p, k) : p->h[d];
            double v = h / (fabs(w->U[d * N + n]) + c);
            if (v < best) best = v;
        }
    }
    return p->cfl * best;
}

/* ======================= exported entry points ======================= */

int orc_nfields(const orc_cfg* c) { return c->ndim == 3 ? 5 : 4; }

/* Conduction / hydrostatic profile for constant K (reading of the paper's
 * "hydrostatic base state"): T_c = t_bot + (t_top - t_bot) z, dp/dz = -g rho,
 * p = a rho T, rho(0) = 1, so p_c = a t_bot (T_c/t_bot)^(g/(a Lambda)),
 * Lambda = t_bot - t_top; isothermal limit p_c = a t_bot exp(-g z /(a t_bot)). */
void orc_profile(const orc_cfg* c, double* Tc, double* pc, double* rhoc)
{
    P p;
    derive(c, &p);
    double Lam = p.t_bot - p.t_top;
    for (int k = 0; k < p.nz; k++) {
        double z = zk(&p, k);
        double T = p.t_bot - Lam * z;
        double pr;
        if (Lam != 0.0)
            pr = p.a * p.t_bot * pow(T / p.t_bot, p.g / (p.a * Lam));
        else
            pr = p.a * p.t_bot * exp(-p.g * z / (p.a * p.t_bot));
        if (Tc) Tc[k] = T;
        if (pc) pc[k] = pr;
        if (rhoc) rhoc[k] = pr / (p.a * T);
    }
    release(&p);
}

/* the nz plane heights the oracle uses for c (uniform, tanh or given) */
void orc_znodes(const orc_cfg* c, double* z)
{
    P p;
    derive(c, &p);
    for (int k = 0; k < p.nz; k++) z[k] = p.z[k];
    release(&p);
}

/* SplitMix64 (Steele, Lea & Flood 2014): output number idx+1 of the
 * generator seeded with `seed`, i.e. the mix of seed + (idx+1)*golden_gamma. */
uint64_t orc_splitmix64(uint64_t seed, uint64_t idx)
{
    uint64_t z = seed + (idx + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* uniform in [-1, 1): 53 high bits scaled to [0,1), then 2u - 1 */
static double xi_of(uint64_t seed, uint64_t idx)
{
    double u = (double)(orc_splitmix64(seed, idx) >> 11) * 0x1.0p-53;
    return 2.0 * u - 1.0;
}

/* Initial state: the conduction profile with an isobaric temperature
 * perturbation pert_amp * xi at interior nodes, u = 0; plates unperturbed. */
void orc_init(const orc_cfg* c, double* ext)
{
    P p;
    derive(c, &p);
    size_t N = p.n;
    double* Tc = malloc(p.nz * sizeof(double));
    double* pc = malloc(p.nz * sizeof(double));
    orc_profile(c, Tc, pc, NULL);
    double* X = calloc(5 * N, sizeof(double));
    for (int k = 0; k < p.nz; k++)
        for (int j = 0; j < p.ny; j++)
            for (int i = 0; i < p.nx; i++) {
                size_t n = idx(&p, i, j, k);
                double T = Tc[k];
                if (k > 0 && k < p.nz - 1) T = Tc[k] + c->pert_amp * xi_of(c->seed, n);
                double rho = pc[k] / (p.a * T);
                X[n] = rho;
                X[4 * N + n] = rho * (T / p.b + p.g * zk(&p, k));
            }
    to_external(&p, X, ext);
    free(X); free(Tc); free(pc);
    release(&p);
}

/* one directional sweep L_dir(Delta) applied to ext (in place); dir 0=x 1=y 2=z */
void orc_sweep(const orc_cfg* c, int dir, double Delta, double* ext)
{
    P p;
    derive(c, &p);
    size_t N = p.n;
    double* X = malloc(5 * N * sizeof(double));
    double* Y = malloc(5 * N * sizeof(double));
    Work w;
    work_alloc(&p, &w);
    to_internal(&p, ext, X);
    if (dir == 2) sweep_z(&p, Delta, X, Y, &w);
    else sweep_h(&p, dir, Delta, X, Y, &w);
    to_external(&p, Y, ext);
    work_free(&w);
    free(X); free(Y);
    release(&p);
}

double orc_dt(const orc_cfg* c, const double* ext)
{
    P p;
    derive(c, &p);
    double* X = malloc(5 * p.n * sizeof(double));
    Work w;
    work_alloc(&p, &w);
    to_internal(&p, ext, X);
    double dt = dt_of(&p, X, &w);
    work_free(&w);
    free(X);
    release(&p);
    return dt;
}

/* nsteps full steps of Eq. time_step:
 * X^{n+1} = L_x L_y L_z L_x L_y L_z X^n with every L at dt/2 (rightmost first:
 * z, y, x, z, y, x; 2D drops y); dt from the state at the start of each step.
 * cfg->split = 1 applies the same half steps as the palindrome x, y, z, z, y, x
 * instead (the symmetric ordering a second-order splitting would use; reading
 * A4 takes the printed one).  Writes each step's dt to dts (if not NULL) and
 * advances *t. */
void orc_step(const orc_cfg* c, double* ext, int nsteps, double* t, double* dts)
{
    P p;
    derive(c, &p);
    size_t N = p.n;
    double* X = malloc(5 * N * sizeof(double));
    double* Y = malloc(5 * N * sizeof(double));
    Work w;
    work_alloc(&p, &w);
    to_internal(&p, ext, X);
    /* sweep directions in the order applied: 0 = x, 1 = y, 2 = z */
    static const int printed3[6] = {2, 1, 0, 2, 1, 0}, palindrome3[6] = {0, 1, 2, 2, 1, 0};
    static const int printed2[4] = {2, 0, 2, 0}, palindrome2[4] = {0, 2, 2, 0};
    const int* order = (p.ndim == 3) ? (p.split ? palindrome3 : printed3) : (p.split ? palindrome2 : printed2);
    const int nsweeps = (p.ndim == 3) ? 6 : 4;
    for (int s = 0; s < nsteps; s++) {
        double dt = dt_of(&p, X, &w);
        double Delta = 0.5 * dt;
        for (int q = 0; q < nsweeps; q++) {
            if (order[q] == 2) sweep_z(&p, Delta, X, Y, &w);
            else sweep_h(&p, order[q], Delta, X, Y, &w);
            double* tmp = X; X = Y; Y = tmp;   /* the result is in X again */
        }
        if (dts) dts[s] = dt;
        if (t) *t += dt;
    }
    to_external(&p, X, ext);
    work_free(&w);
    free(X); free(Y);
    release(&p);
}

/* Diagnostics (Sec. 2).  Volume averages use the trapezoid rule in z (half
 * weight on the plate planes; on a stretched grid the weight of plane k is
 * its cell width w[k]) and the plain mean in x, y.
 * out[0]  Nu      = 1 + Nu_conv + Nu_K                       (Eq. volume_Nu)
 * out[1]  Nu_conv = sqrt(Ra Pr)/eps <rho u_z T_sa>_V
 * out[2]  Nu_K    = D sqrt(Ra Pr)/2 <rho u_z u^2>_V
 * out[3]  Nu_bot  = -(1/eps) d<T_sa>_A/dz at z=0, second-order forward difference
 * out[4]  Nu_top  = same at z=1, second-order backward difference   (Eq. mean_Nu)
 *         (on a stretched grid: the derivative of the quadratic through
 *         the three planes next to the plate)
 * out[5]  Nu_bar  = (Nu_bot + Nu_top)/2
 * out[6]  Re      = sqrt(Ra/Pr) sqrt(<u^2>_V)  (instantaneous; Eq. Re before the time mean)
 * out[7]  KE      = <rho u^2 / 2>_V
 * out[8]  mass    = <rho>_V
 * out[9]  energy  = <E>_V
 * out[10] max Mach number |u|/c
 * T_sa = T - (1 - D z) (superadiabatic temperature). */
void orc_diag(const orc_cfg* c, const double* ext, double* out)
{
    P p;
    derive(c, &p);
    size_t N = p.n;
    double* X = malloc(5 * N * sizeof(double));
    to_internal(&p, ext, X);
    double s_conv = 0, s_k = 0, s_u2 = 0, s_ke = 0, s_m = 0, s_e = 0, mach = 0;
    double* TA = calloc(p.nz, sizeof(double));
    for (int k = 0; k < p.nz; k++) {
        double wgt = p.stretched ? p.w[k] : ((k == 0 || k == p.nz - 1) ? 0.5 : 1.0);
        double z = zk(&p, k);
        for (int j = 0; j < p.ny; j++)
            for (int i = 0; i < p.nx; i++) {
                size_t n = idx(&p, i, j, k);
                double rho = X[n];
                double u = X[1 * N + n] / rho, v = X[2 * N + n] / rho, w = X[3 * N + n] / rho;
                double u2 = u * u + v * v + w * w;
                double T = p.b * (X[4 * N + n] / rho - 0.5 * u2 - p.g * z);
                double Tsa = T - (1.0 - p.D * z);
                s_conv += wgt * rho * w * Tsa;
                s_k += wgt * rho * w * u2;
                s_u2 += wgt * u2;
                s_ke += wgt * 0.5 * rho * u2;
                s_m += wgt * rho;
                s_e += wgt * X[4 * N + n];
                TA[k] += T;
                double M = sqrt(u2) / sqrt(p.gam * p.a * T);
                if (M > mach) mach = M;
            }
    }
    double vol = p.stretched ? (double)p.nx * p.ny : (double)p.nx * p.ny * (p.nz - 1);
    double sRP = sqrt(p.Ra * p.Pr);
    out[1] = sRP / p.eps * (s_conv / vol);
    out[2] = p.D * sRP / 2.0 * (s_k / vol);
    out[0] = 1.0 + out[1] + out[2];
    double f[3], g[3];
    int K = p.nz - 1;
    for (int q = 0; q < 3; q++) {
        f[q] = TA[q] / ((double)p.nx * p.ny) - (1.0 - p.D * zk(&p, q));
        g[q] = TA[K - q] / ((double)p.nx * p.ny) - (1.0 - p.D * zk(&p, K - q));
    }
    if (!p.stretched) {
        double dz = p.h[2];
        out[3] = -(1.0 / p.eps) * (-3.0 * f[0] + 4.0 * f[1] - f[2]) / (2.0 * dz);
        out[4] = -(1.0 / p.eps) * (3.0 * g[0] - 4.0 * g[1] + g[2]) / (2.0 * dz);
    } else {
        /* derivative at the plate of the quadratic through the three planes:
         * spacings h1 (plate to the next plane) and h2 (the one after) */
        double h1 = p.z[1] - p.z[0], h2 = p.z[2] - p.z[1];
        double db = -(2.0 * h1 + h2) / (h1 * (h1 + h2)) * f[0] + (h1 + h2) / (h1 * h2) * f[1]
                    - h1 / (h2 * (h1 + h2)) * f[2];
        h1 = p.z[K] - p.z[K - 1];
        h2 = p.z[K - 1] - p.z[K - 2];
        double dt_ = (2.0 * h1 + h2) / (h1 * (h1 + h2)) * g[0] - (h1 + h2) / (h1 * h2) * g[1]
                     + h1 / (h2 * (h1 + h2)) * g[2];
        out[3] = -(1.0 / p.eps) * db;
        out[4] = -(1.0 / p.eps) * dt_;
    }
    out[5] = (out[3] + out[4]) / 2.0;
    out[6] = sqrt(p.Ra / p.Pr) * sqrt(s_u2 / vol);
    out[7] = s_ke / vol;
    out[8] = s_m / vol;
    out[9] = s_e / vol;
    out[10] = mach;
    free(TA);
    free(X);
    release(&p);
}

/* 1D scalar periodic linear advection u_t + a u_x = 0 (a > 0) with the same
 * predictor / corrector / average / TVD sequence (Sec. 3.1) and the same
 * limiter, for the total-variation test of the TVD-term reading.  Here the
 * dot products are plain products, F = a u, and Co = a dt/h. */
void orc_advect1d(int n, double a, double dt, double h, int nsteps, int tvd_form, double* u)
{
    double* F = malloc(n * sizeof(double));
    double* uP = malloc(n * sizeof(double));
    double* FP = malloc(n * sizeof(double));
    double* y = malloc(n * sizeof(double));
    double* D = malloc(n * sizeof(double));
    double lam = dt / h, Co = a * dt / h, C = coefC(Co);
    for (int s = 0; s < nsteps; s++) {
        for (int i = 0; i < n; i++) F[i] = a * u[i];
        for (int i = 0; i < n; i++) uP[i] = u[i] - lam * (F[i] - F[(i - 1 + n) % n]);
        for (int i = 0; i < n; i++) FP[i] = a * uP[i];
        for (int i = 0; i < n; i++) {
            double uC = u[i] - lam * (FP[(i + 1) % n] - FP[i]);
            y[i] = (uP[i] + uC) / 2.0;
        }
        for (int i = 0; i < n; i++) {
            double dm = u[i] - u[(i - 1 + n) % n];
            double d0 = u[(i + 1) % n] - u[i];
            double dp = u[(i + 2) % n] - u[(i + 1) % n];
            double dd = d0 * d0;
            D[i] = 0.0;
            if (tvd_form == 2 || dd == 0.0) continue;
            double rp = dm * d0 / dd, rm = d0 * dp / dd;
            double G = (tvd_form == 0) ? Gfun(rp, C) + Gfun(rm, C) : Gfun(rp + rm, C);
            D[i] = G * d0;
        }
        for (int i = 0; i < n; i++) u[i] = y[i] + (D[i] - D[(i - 1 + n) % n]);
    }
    free(F); free(uP); free(FP); free(y); free(D);
}

/* ---- extended diagnostics (the analyses of Sec. 4-6) ----
 *
 * z derivatives at an interior plane k use the three planes k-1, k, k+1
 * (spacings hm below, hp above): the derivative and second derivative of
 * the quadratic through them (exact for quadratics on any planes; the
 * central differences on uniform planes).  x and y derivatives are central
 * (periodic). */
static double dz3(const P* p, int k, double fm, double f0, double fp)
{
    double hm = p->z[k] - p->z[k - 1], hp = p->z[k + 1] - p->z[k];
    return (hm * hm * fp - hp * hp * fm + (hp * hp - hm * hm) * f0) / (hm * hp * (hm + hp));
}

static double dzz3(const P* p, int k, double fm, double f0, double fp)
{
    double hm = p->z[k] - p->z[k - 1], hp = p->z[k + 1] - p->z[k];
    return 2.0 * ((fp - f0) / hp - (f0 - fm) / hm) / (hm + hp);
}

/* Plane means of the terms of the z-momentum equation, of the two squares
 * in the correlation C(Ra) and the vertical profiles of Sec. 4:
 *   out[k*9+0] <F_n>_A = <rho (u . grad) u_z>_A        (nonlinear term)
 *   out[k*9+1] <F_p>_A = <-dp/dz>_A                   (pressure gradient)
 *   out[k*9+2] <F_b>_A = <rho g>_A                    (buoyancy, g = gravity/eps)
 *   out[k*9+3] <F_v>_A = <d_i tau_iz>_A               (viscous force)
 *   out[k*9+4] <(rho u_z)^2>_A,  out[k*9+5] <T_sa^2>_A, T_sa = T - (1 - D z)
 *   out[k*9+6] <T_sa>_A = <T>_A - T_A(z), T_A = 1 - D z
 *   out[k*9+7] <rho>_A - rho_A(z), rho_A = (1 - D z)^(1/(gamma-1))
 *   out[k*9+8] U(z) = sqrt(<u^2>_A), the plane's rms velocity
 * The force terms need neighbouring planes: on the plates they are 0.
 * d_i tau_iz = mu (d_xx u_z + d_yy u_z + (2 + s) d_zz u_z + (1 + s)(d_x d_z u_x + d_y d_z u_y)),
 * s the Stokes coefficient (tau_ij = mu (d_j u_i + d_i u_j + s (div u) delta_ij)). */
void orc_ext_profiles(const orc_cfg* c, const double* ext, double* out)
{
    P p;
    derive(c, &p);
    size_t N = p.n;
    double* X = malloc(5 * N * sizeof(double));
    double *U = malloc(3 * N * sizeof(double)), *T = malloc(N * sizeof(double)), *Pr = malloc(N * sizeof(double));
    to_internal(&p, ext, X);
    prims(&p, X, U, T, Pr);
    double cells = (double)p.nx * p.ny;
    int K = p.nz - 1;
    for (int k = 0; k < p.nz; k++) {
        double s[6] = {0, 0, 0, 0, 0, 0}, tsum = 0.0, rsum = 0.0, usum = 0.0;
        double z = zk(&p, k);
        for (int j = 0; j < p.ny; j++)
            for (int i = 0; i < p.nx; i++) {
                size_t n = idx(&p, i, j, k);
                double rho = X[n];
                double ux = U[n], uy = U[N + n], uz = U[2 * N + n];
                double Tsa = T[n] - (1.0 - p.D * z);
                s[4] += (rho * uz) * (rho * uz);
                s[5] += Tsa * Tsa;
                tsum += T[n];
                rsum += rho;
                usum += (ux * ux + uy * uy) + uz * uz;
                if (k == 0 || k == K) continue;
                size_t xp = nbr(&p, i, j, k, 0, +1), xm = nbr(&p, i, j, k, 0, -1);
                size_t yp = nbr(&p, i, j, k, 1, +1), ym = nbr(&p, i, j, k, 1, -1);
                size_t zp = idx(&p, i, j, k + 1), zm = idx(&p, i, j, k - 1);
                double dx = p.h[0], dy = p.h[1];
                double dxuz = (U[2 * N + xp] - U[2 * N + xm]) / (2.0 * dx);
                double dyuz = (U[2 * N + yp] - U[2 * N + ym]) / (2.0 * dy);
                double dzuz = dz3(&p, k, U[2 * N + zm], uz, U[2 * N + zp]);
                s[0] += rho * ((ux * dxuz + uy * dyuz) + uz * dzuz);
                s[1] += -dz3(&p, k, Pr[zm], Pr[n], Pr[zp]);
                s[2] += rho * p.g;
                double dxx = (U[2 * N + xp] - 2.0 * uz + U[2 * N + xm]) / (dx * dx);
                double dyy = (U[2 * N + yp] - 2.0 * uz + U[2 * N + ym]) / (dy * dy);
                double dzz = dzz3(&p, k, U[2 * N + zm], uz, U[2 * N + zp]);
                /* d_x d_z u_x: x-central of the z-derivative on the planes */
                size_t xpzp = idx(&p, (i + 1) % p.nx, j, k + 1), xmzp = idx(&p, (i - 1 + p.nx) % p.nx, j, k + 1);
                size_t xpzm = idx(&p, (i + 1) % p.nx, j, k - 1), xmzm = idx(&p, (i - 1 + p.nx) % p.nx, j, k - 1);
                double dxdzux = (dz3(&p, k, U[xpzm], U[xp], U[xpzp]) - dz3(&p, k, U[xmzm], U[xm], U[xmzp])) / (2.0 * dx);
                double dydzuy = 0.0;
                if (p.ndim == 3) {
                    size_t ypzp = idx(&p, i, (j + 1) % p.ny, k + 1), ymzp = idx(&p, i, (j - 1 + p.ny) % p.ny, k + 1);
                    size_t ypzm = idx(&p, i, (j + 1) % p.ny, k - 1), ymzm = idx(&p, i, (j - 1 + p.ny) % p.ny, k - 1);
                    dydzuy = (dz3(&p, k, U[N + ypzm], U[N + yp], U[N + ypzp]) -
                              dz3(&p, k, U[N + ymzm], U[N + ym], U[N + ymzp])) / (2.0 * dy);
                }
                s[3] += p.mu * ((dxx + dyy) + (2.0 + p.stokes) * dzz + (1.0 + p.stokes) * (dxdzux + dydzuy));
            }
        for (int q = 0; q < 6; q++) out[(size_t)k * 9 + q] = s[q] / cells;
        out[(size_t)k * 9 + 6] = tsum / cells - (1.0 - p.D * z);
        out[(size_t)k * 9 + 7] = rsum / cells - pow(1.0 - p.D * z, 1.0 / (p.gam - 1.0));
        out[(size_t)k * 9 + 8] = sqrt(usum / cells);
    }
    free(X); free(U); free(T); free(Pr);
    release(&p);
}

/* Quantities derived from the plane means:
 *   out[0] C = <rho u_z T_sa>_V / sqrt(<(rho u_z)^2>_V <T_sa^2>_V)   (Eq. Corr_Ra)
 *   out[1] <(rho u_z)^2>_V, out[2] <T_sa^2>_V
 *   out[3] lambda_b, out[4] lambda_t: thermal boundary-layer thicknesses,
 *          read as the classical tangent construction: the depth at which the
 *          plate tangent of <T_sa>_A meets the adiabatic bulk, i.e. the
 *          superadiabatic drop across the layer over the plate gradient,
 *          lambda_b = (Tb - f_0) / (d<T_sa>_A/dz at z = 0),
 *          lambda_t = (f_K - Tb) / (d<T_sa>_A/dz at z = 1),
 *          with the plate derivatives of the plate Nusselt numbers (the
 *          three-plane quadratic) and Tb the trapezoid mean of <T_sa>_A over
 *          the planes with 1/4 <= z <= 3/4 (the bulk, where <T>_A follows
 *          the adiabat).
 *   out[5..8] <F_n>, <F_p>, <F_b>, <F_v> over the interior planes (weights
 *          w_k of the interior planes, normalised by their sum)
 *   out[9] max over nodes of r = K_e / I_e = (rho u^2/2) / (rho C_v T) = b u^2 / (2 T)
 *   out[10] lambda_b_slope, out[11] lambda_t_slope: the boundary layers by the
 *          slope criterion of slope_lambda (tol 0.1), the second reading
 * hist[q] (q < nbins): nodes with log10 r in [lo + q w, lo + (q+1) w),
 *          w = (hi - lo)/nbins; below lo (or r = 0) in bin 0, at or above hi
 *          in bin nbins - 1. */
/* slope of <T_sa>_A at plane k from the quadratic through three planes:
 * one-sided (planes 0, 1, 2 or K, K-1, K-2) on the plates, central inside */
static double tsa_slope(const P* p, const double* sa, int k)
{
    int K = p->nz - 1;
    const double* z = p->z;
    if (k == 0) {
        double h1 = z[1] - z[0], h2 = z[2] - z[1];
        return -(2.0 * h1 + h2) / (h1 * (h1 + h2)) * sa[0] + (h1 + h2) / (h1 * h2) * sa[1] - h1 / (h2 * (h1 + h2)) * sa[2];
    }
    if (k == K) {
        double h1 = z[K] - z[K - 1], h2 = z[K - 1] - z[K - 2];
        return (2.0 * h1 + h2) / (h1 * (h1 + h2)) * sa[K] - (h1 + h2) / (h1 * h2) * sa[K - 1] + h1 / (h2 * (h1 + h2)) * sa[K - 2];
    }
    double h1 = z[k] - z[k - 1], h2 = z[k + 1] - z[k];
    return -h2 / (h1 * (h1 + h2)) * sa[k - 1] + (h2 - h1) / (h1 * h2) * sa[k] + h1 / (h2 * (h1 + h2)) * sa[k + 1];
}

/* Boundary layer by the words of Sec. 4 (the height where the slope of
 * <T>_A approximates the adiabatic gradient -D), read with a tolerance: the
 * first distance from the plate at which |d<T>_A/dz + D| = |d<T_sa>_A/dz|
 * has fallen to tol * D, linearly interpolated between the two planes around
 * the crossing; NaN if it never does (the conduction state) */
static double slope_lambda(const P* p, const double* sa, int top, double tol)
{
    int K = p->nz - 1;
    double target = tol * p->D, dprev = 0.0, sprev = 0.0;
    for (int q = 0; q <= K; q++) {
        int k = top ? K - q : q;
        double s = fabs(tsa_slope(p, sa, k));
        double d = top ? 1.0 - p->z[k] : p->z[k];
        if (s <= target) {
            if (q == 0) return 0.0;
            return dprev + (sprev - target) / (sprev - s) * (d - dprev);
        }
        dprev = d;
        sprev = s;
    }
    return NAN;
}

#define ORC_LAMBDA_SLOPE_TOL 0.1

void orc_extended(const orc_cfg* c, const double* ext, double* out, long long* hist, int nbins, double lo, double hi)
{
    P p;
    derive(c, &p);
    size_t N = p.n;
    int K = p.nz - 1;
    double* prof = malloc((size_t)p.nz * 9 * sizeof(double));
    orc_ext_profiles(c, ext, prof);
    double* X = malloc(5 * N * sizeof(double));
    double *U = malloc(3 * N * sizeof(double)), *T = malloc(N * sizeof(double)), *Pr = malloc(N * sizeof(double));
    to_internal(&p, ext, X);
    prims(&p, X, U, T, Pr);
    double cells = (double)p.nx * p.ny;
    double s_conv = 0, s_m2 = 0, s_t2 = 0, wsum = 0, f[4] = {0, 0, 0, 0};
    double* TA = calloc(p.nz, sizeof(double));
    for (int k = 0; k < p.nz; k++) {
        double wgt = p.stretched ? p.w[k] : ((k == 0 || k == K) ? 0.5 : 1.0);
        double z = zk(&p, k), conv = 0.0;
        for (int j = 0; j < p.ny; j++)
            for (int i = 0; i < p.nx; i++) {
                size_t n = idx(&p, i, j, k);
                conv += X[n] * U[2 * N + n] * (T[n] - (1.0 - p.D * z));
                TA[k] += T[n];
            }
        s_conv += wgt * conv / cells;
        s_m2 += wgt * prof[(size_t)k * 9 + 4];
        s_t2 += wgt * prof[(size_t)k * 9 + 5];
        TA[k] /= cells;
        if (k > 0 && k < K) {
            wsum += wgt;
            for (int q = 0; q < 4; q++) f[q] += wgt * prof[(size_t)k * 9 + q];
        }
    }
    double vol = p.stretched ? 1.0 : (double)(p.nz - 1);
    out[1] = s_m2 / vol;
    out[2] = s_t2 / vol;
    out[0] = (s_conv / vol) / sqrt(out[1] * out[2]);
    {
        double sa[3], sb[3], tb = 0.0, tw = 0.0;
        for (int q = 0; q < 3; q++) {
            sa[q] = TA[q] - (1.0 - p.D * p.z[q]);
            sb[q] = TA[K - q] - (1.0 - p.D * p.z[K - q]);
        }
        for (int k = 0; k <= K; k++)
            if (p.z[k] >= 0.25 && p.z[k] <= 0.75) {
                double wk = p.stretched ? p.w[k] : 1.0;
                tb += wk * (TA[k] - (1.0 - p.D * p.z[k]));
                tw += wk;
            }
        tb /= tw;
        double h1 = p.z[1] - p.z[0], h2 = p.z[2] - p.z[1];
        double db = -(2.0 * h1 + h2) / (h1 * (h1 + h2)) * sa[0] + (h1 + h2) / (h1 * h2) * sa[1] - h1 / (h2 * (h1 + h2)) * sa[2];
        h1 = p.z[K] - p.z[K - 1];
        h2 = p.z[K - 1] - p.z[K - 2];
        double dtp = (2.0 * h1 + h2) / (h1 * (h1 + h2)) * sb[0] - (h1 + h2) / (h1 * h2) * sb[1] + h1 / (h2 * (h1 + h2)) * sb[2];
        out[3] = (tb - sa[0]) / db;
        out[4] = (sb[0] - tb) / dtp;
        double* sal = malloc((size_t)p.nz * sizeof(double));
        for (int k = 0; k <= K; k++) sal[k] = TA[k] - (1.0 - p.D * p.z[k]);
        out[10] = slope_lambda(&p, sal, 0, ORC_LAMBDA_SLOPE_TOL);
        out[11] = slope_lambda(&p, sal, 1, ORC_LAMBDA_SLOPE_TOL);
        free(sal);
    }
    for (int q = 0; q < 4; q++) out[5 + q] = f[q] / wsum;
    double rmax = 0.0, bw = (hi - lo) / nbins;
    for (int q = 0; q < nbins; q++) hist[q] = 0;
    for (size_t n = 0; n < N; n++) {
        double u2 = U[n] * U[n] + U[N + n] * U[N + n] + U[2 * N + n] * U[2 * N + n];
        double r = p.b * u2 / (2.0 * T[n]);
        if (r > rmax) rmax = r;
        int q = 0;
        if (r > 0.0) {
            double t = (log10(r) - lo) / bw;
            q = t < 0.0 ? 0 : (t >= nbins ? nbins - 1 : (int)t);
        }
        hist[q]++;
    }
    out[9] = rmax;
    free(prof); free(X); free(U); free(T); free(Pr); free(TA);
    release(&p);
}
