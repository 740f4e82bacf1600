/*
 * oracle.c -- plain serial FP64 CPU oracle of MIUGKS (arXiv 1704.03151).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the CPU
 * baseline leg of the benchmark; never by the product library.  Written for
 * readability against the paper, not for speed: straightforward loops in the
 * order the paper states the steps.  Where the paper is silent the reading
 * taken is stated at the function (and listed in the design notes).
 *
 * The last section differentiates the steady equations by hand (reverse
 * mode) for the adjoint gradient of wall objectives; its pins are
 * finite-difference and high-precision derivatives and converged forward
 * solves (tests/test_oracle_adjoint.py).
 *
 * Bodies (solid cells, the square cylinder of Sec. 4.3) are handled by face
 * ids: a face between a fluid and a solid cell is a boundary face of the fluid
 * cell, and cells in a body hold no residual, update or correction (pins in
 * tests/test_oracle_solid.py).  The adjoint section refuses meshes with
 * bodies.
 *
 * Parity pins (tests/test_oracle_*.py) cover every function here except the
 * physical time step rule of face_dt(), which the paper leaves open and which
 * is therefore "parity unpinned" (both implementations follow the same rule),
 * and the three positivity rules of the prediction and the update (a cell
 * whose corrected or updated state would have non-positive density or
 * internal energy keeps its state), which never trigger in smooth flow and
 * are pinned only by the Ma 5 square-cylinder start staying physical.
 */
#include "oracle.h"
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

/* Optional OpenMP build (-fopenmp, a separate library): faces, cells and the
 * cells of one anti-diagonal of a sweep are spread over threads; each face or
 * cell is computed by one thread with the serial build's arithmetic in the
 * serial build's order, so the two builds give the same bits.  Scratch is
 * per thread. */
#ifdef _OPENMP
#include <omp.h>
#define ORC_TID omp_get_thread_num()
#define ORC_MAXTHR omp_get_max_threads()
#else
#define ORC_TID 0
#define ORC_MAXTHR 1
#endif

#define KINT 1      /* internal (z-translational) degrees of freedom of the 2-D reduced model */
#define MAXL 8
#define PI 3.14159265358979323846

static char g_err[512];
static int fail(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return 1;
}
const char *oracle_last_error(void) { return g_err; }

typedef struct { int type; double rho, u, v, t; } obc_t;

typedef struct {
    int nx, ny, nc, nfx, nfy;
    double *xn, *yn, *xc, *yc, *dx, *dy;
    int *fbx, *fby;
    unsigned char *solid; /* per cell: 1 inside a body (no state, never updated) */
    int nfluid;
    /* FAS work (nc x 4) and CS work (2 x nc x nv) */
    double *Wn, *Wc, *Rc, *P, *RE, *dW, *Wtil;
    double *r, *df, *dl, *Ad, *inv_tau;
} olev_t;

/* Adaptive multigrid cycle (Sec. 3.4 names it without a rule; reading): a
 * level visits its coarser level a second time when the first visit left more
 * than a ratio (ADAPT_RATIO unless set) of the coarse residual it started from
 * (L2 norms over all values), at most ADAPT_MAX_VISITS visits.  With ratio 0
 * every level visits twice (the W cycle); with a ratio above any reduction,
 * once (the V cycle). */
#define ADAPT_RATIO 0.2
#define ADAPT_MAX_VISITS 2
#define ADAPT_LOG 4096

/* one boundary face of a cell, as seen from that cell */
typedef struct { int bc, axis, outsign; double S, V; } bface_t;

struct oracle_solver {
    int L;
    olev_t lev[MAXL];
    int nu, nvv, nv;
    double *u, *v, *w;
    int *mxk, *myk;
    double umax_abs, vmax_abs;
    double kn, omega, pr, mu_ref;
    int nbc;
    obc_t *bc;
    double *Cw; /* per BC: unit-density Maxwellian at the BC state, G part */
    int nu1, nu2, nuc;
    int cycle; /* 0 V, 1 W, 2 F, 3 adaptive (Sec. 3.4: V, W, F and adaptive cycles) */
    int shock; /* pressure-jump collision time at interior faces (0 off) */
    double adapt_ratio;                   /* ADAPT_RATIO unless set */
    int adapt_n;                          /* adaptive-cycle decisions taken so far */
    unsigned char adapt_log[ADAPT_LOG];   /* each: 1 = a second coarse visit (ring of ADAPT_LOG) */
    double cfl, dtn_growth, dtp_min;
    int iter;
    double *f, *W, *q, *R;
    double *phx, *phy, *Fx, *Fy;
    int nthr;                   /* threads of the parallel loops (1 in the serial build) */
    double *tmp0, *tmp1, *tmp2; /* per-face / per-cell velocity scratch (2 x nv per thread each) */
    double *sD, *sbase, *sxc;   /* sweep scratch (nv, 2 nv, 2 nv per thread) */
};

/* ------------------------------------------------------------------ */
/* Gas model and quadrature                                            */
/* ------------------------------------------------------------------ */

/* VHS reference viscosity for a given Knudsen number (alpha = 1), in units of
 * rho0*L*sqrt(2RT0).  The paper relates Kn and viscosity through the VHS model
 * (Sec. 4.1, 4.3) without printing the constant; this is the standard VHS
 * mean-free-path relation. */
double oracle_mu_ref(double kn, double omega)
{
    return 15.0 * sqrt(PI) * kn / (2.0 * (5.0 - 2.0 * omega) * (7.0 - 2.0 * omega));
}

/* Discrete velocity nodes and weights on [a, b] (Sec. 4.1: trapezoidal rule;
 * Sec. 4.3: Newton-Cotes).  rule 0 = trapezoid, rule 1 = composite Boole
 * (closed Newton-Cotes of degree 4, needs (n-1) % 4 == 0).  Nodes are placed
 * symmetrically about the centre so that mirrored nodes negate exactly. */
int oracle_vgrid(int n, double a, double b, int rule, double *x, double *w)
{
    if (n < 2 || !(b > a)) return fail("vgrid: need n >= 2 and b > a");
    double h = (b - a) / (n - 1), c = 0.5 * (a + b);
    for (int i = 0; i < n; ++i) x[i] = c + (i - 0.5 * (n - 1)) * h;
    if (rule == 0) {
        for (int i = 0; i < n; ++i) w[i] = h;
        w[0] = w[n - 1] = 0.5 * h;
    } else if (rule == 1) {
        if ((n - 1) % 4) return fail("vgrid: Boole rule needs (n-1) %% 4 == 0");
        for (int i = 0; i < n; ++i) w[i] = 0.0;
        for (int p = 0; p + 4 < n; p += 4) {
            w[p] += 7.0; w[p + 1] += 32.0; w[p + 2] += 12.0; w[p + 3] += 32.0; w[p + 4] += 7.0;
        }
        for (int i = 0; i < n; ++i) w[i] *= 2.0 * h / 45.0;
    } else {
        return fail("vgrid: unknown rule %d", rule);
    }
    return 0;
}

/* conservative -> primitive (rho, U, V, lambda); rho*eps = rho|U|^2/2 + (K+2) rho/(4 lambda) */
static void prim(const double *W, double *rho, double *U, double *V, double *lam)
{
    *rho = W[0];
    *U = W[1] / W[0];
    *V = W[2] / W[0];
    double eint = W[3] - 0.5 * (W[1] * W[1] + W[2] * W[2]) / W[0];
    *lam = (KINT + 2) * W[0] / (4.0 * eint);
}

/* tau = mu/p with mu = mu_ref T^omega, p = rho T / 2 (Sec. 4.1) */
static double tau_of(const oracle_solver *s, double rho, double lam)
{
    double T = 1.0 / lam;
    return s->mu_ref * pow(T, s->omega) / (0.5 * rho * T);
}

/* reduced Maxwellian G at node k (Eq. f_on_wall form with R = 1/2) */
static double maxw(double rho, double U, double V, double lam, double u, double v)
{
    return rho * (lam / PI) * exp(-lam * ((u - U) * (u - U) + (v - V) * (v - V)));
}

/* Shakhov equilibrium at node (u, v) (Sec. 2.1, the Shakhov-type model that
 * gives the Prandtl number): the 3-D model f_M [1 + (1-Pr) c.q (c^2/RT - 5) /
 * (5 p R T)] reduced over xi_z with <xi_z^2> = RT, <xi_z^4> = 3 (RT)^2 and
 * R = 1/2, p = rho/(2 lambda):
 *   G+ = G_M [1 + (1-Pr) (4 lambda^2 / (5 rho)) (c.q) (2 lambda c^2 - 4)],
 *   H+ = H_M [1 + (1-Pr) (4 lambda^2 / (5 rho)) (c.q) (2 lambda c^2 - 2)],
 * c = (u - U, v - V), H_M = G_M K_int / (4 lambda).  The correction carries no
 * mass, momentum or energy, and the heat flux of (G+, H+) is (1-Pr) q. */
static void shakhov(double rho, double U, double V, double lam, double qx, double qy, double pr, double u, double v,
                    double *gP, double *hP)
{
    double cx = u - U, cy = v - V, c2 = cx * cx + cy * cy;
    double gM = maxw(rho, U, V, lam, u, v), hM = gM * KINT / (4.0 * lam);
    double Fq = (1.0 - pr) * 4.0 * lam * lam / (5.0 * rho) * (cx * qx + cy * qy);
    *gP = gM * (1.0 + Fq * (2.0 * lam * c2 - 4.0));
    *hP = hM * (1.0 + Fq * (2.0 * lam * c2 - 2.0));
}

void oracle_shakhov(double rho, double U, double V, double lam, double qx, double qy, double pr, int n,
                    const double *u, const double *v, double *G, double *H)
{
    for (int k = 0; k < n; ++k) shakhov(rho, U, V, lam, qx, qy, pr, u[k], v[k], &G[k], &H[k]);
}

/* ------------------------------------------------------------------ */
/* UGKS building blocks (the explicit flux is deferred by the paper to  */
/* its references; these are the standard UGKS forms)                   */
/* ------------------------------------------------------------------ */

/* Time integrals of the integral solution over [0, dt] with collision time
 * tau (x = dt/tau, e = exp(-x)):
 *   q1 = dt - tau(1-e)                 (equilibrium)
 *   q2 = -tau dt (1+e) + 2 tau^2 (1-e) (equilibrium spatial slope)
 *   q3 = dt^2/2 - tau dt + tau^2 (1-e) (equilibrium time slope)
 *   q4 = tau (1-e)                     (initial distribution)
 *   q5 = tau dt e - tau^2 (1-e)        (initial slope)
 * For x < 1 the cancelling forms are summed as power series in x. */
void oracle_time_coeffs(double dt, double tau, double q[5])
{
    double x = dt / tau;
    if (x < 1.0) {
        double p[27];
        p[0] = 1.0;
        for (int n = 1; n < 27; ++n) p[n] = p[n - 1] * x / n; /* x^n / n! */
        double s1 = 0, s2 = 0, s3 = 0, s4 = 0, s5 = 0;
        for (int n = 0; n < 26; ++n) {
            double sg = (n % 2) ? -1.0 : 1.0;      /* (-1)^n */
            s4 += sg * p[n] / (n + 1);             /* sum_{n>=0} (-1)^n x^n/(n+1)! */
            if (n >= 1) {
                s1 += -sg * p[n] / (n + 1);                     /* (-1)^{n+1} x^n/(n+1)! */
                s3 += -sg * p[n] / ((double)(n + 1) * (n + 2)); /* (-1)^{n+1} x^n/(n+2)! */
            }
            int m = n + 1;                                      /* m >= 1 */
            double sm = (m % 2) ? -1.0 : 1.0;                   /* (-1)^m */
            s5 += sm * p[m - 1] / (m + 1);                      /* (-1)^m m x^{m-1}/(m+1)! */
            if (m >= 2) s2 += sm * (1.0 - m) * p[m - 1] / ((double)m * (m + 1));
        }
        q[0] = dt * s1;
        q[1] = dt * dt * s2;
        q[2] = dt * dt * s3;
        q[3] = dt * s4;
        q[4] = dt * dt * s5;
    } else {
        double e = exp(-x), E1 = -expm1(-x);
        q[0] = dt - tau * E1;
        q[1] = -tau * dt * (1.0 + e) + 2.0 * tau * tau * E1;
        q[2] = 0.5 * dt * dt - tau * dt + tau * tau * E1;
        q[3] = tau * E1;
        q[4] = tau * dt * e - tau * tau * E1;
    }
}

/* Micro-slope inversion: given the derivative of W divided by rho, dw, find
 * a = (a1..a4) such that the (continuous) moments of (a1 + a2 u + a3 v +
 * a4 (u^2+v^2+xi^2)/2) g reproduce it, g the Maxwellian at (U, V, lam). */
void oracle_micro_slope(const double dw[4], double U, double V, double lam, double a[4])
{
    double Kp2 = KINT + 2.0;
    double R4 = 2.0 * dw[3] - (U * U + V * V + Kp2 / (2.0 * lam)) * dw[0];
    double R3 = dw[2] - V * dw[0];
    double R2 = dw[1] - U * dw[0];
    a[3] = 4.0 * lam * lam / Kp2 * (R4 - 2.0 * U * R2 - 2.0 * V * R3);
    a[2] = 2.0 * lam * R3 - V * a[3];
    a[1] = 2.0 * lam * R2 - U * a[3];
    a[0] = dw[0] - U * a[1] - V * a[2] - 0.5 * a[3] * (U * U + V * V + Kp2 / (2.0 * lam));
}

/* van Leer limiter of two one-sided slopes */
double oracle_vanleer(double s1, double s2)
{
    double p = s1 * s2;
    return p > 0.0 ? 2.0 * p / (s1 + s2) : 0.0;
}

/* Physical time step of one face: CFL number times the smaller normal cell
 * width over the largest normal discrete speed (Sec. 2.1: Delta t_p from a CFL
 * condition with Courant number below 1; the exact rule is not printed). */
static double face_dt(const oracle_solver *s, int axis, double hL, double hR)
{
    double um = axis == 0 ? s->umax_abs : s->vmax_abs;
    return s->cfl * (hL < hR ? hL : hR) / um;
}

/* (a . psi) g split into the two reduced components, with
 * b = a1 + a2 u + a3 v + a4 (u^2+v^2)/2:
 *   G part: b gM + a4 hM,  H part: b hM + a4 <xi^4>/4 gM */
static void slope_moments(const double a[4], double u, double v, double gM, double hM,
                          double lam, double *mG, double *mH)
{
    double b = a[0] + a[1] * u + a[2] * v + 0.5 * a[3] * (u * u + v * v);
    double xi4q = KINT * (KINT + 2.0) / (16.0 * lam * lam);
    *mG = b * gM + a[3] * hM;
    *mH = b * hM + a[3] * xi4q * gM;
}

/* ------------------------------------------------------------------ */
/* Mesh levels                                                          */
/* ------------------------------------------------------------------ */

static double *dalloc(size_t n) { return (double *)calloc(n ? n : 1, sizeof(double)); }

static int level_alloc(oracle_solver *s, olev_t *Lv)
{
    size_t nc = Lv->nc, nv = s->nv;
    Lv->Wn = dalloc(4 * nc); Lv->Wc = dalloc(4 * nc); Lv->Rc = dalloc(4 * nc);
    Lv->P = dalloc(4 * nc); Lv->RE = dalloc(4 * nc); Lv->dW = dalloc(4 * nc); Lv->Wtil = dalloc(4 * nc);
    Lv->r = dalloc(2 * nc * nv); Lv->df = dalloc(2 * nc * nv); Lv->dl = dalloc(2 * nc * nv);
    Lv->Ad = dalloc(2 * nc * nv); Lv->inv_tau = dalloc(nc);
    if (!Lv->Wn || !Lv->Wc || !Lv->Rc || !Lv->P || !Lv->RE || !Lv->dW || !Lv->Wtil || !Lv->r ||
        !Lv->df || !Lv->dl || !Lv->Ad || !Lv->inv_tau)
        return fail("out of memory");
    return 0;
}

static int level_geom(olev_t *Lv)
{
    int nx = Lv->nx, ny = Lv->ny;
    Lv->xc = dalloc(nx); Lv->dx = dalloc(nx); Lv->yc = dalloc(ny); Lv->dy = dalloc(ny);
    for (int i = 0; i < nx; ++i) {
        Lv->dx[i] = Lv->xn[i + 1] - Lv->xn[i];
        Lv->xc[i] = 0.5 * (Lv->xn[i] + Lv->xn[i + 1]);
        if (!(Lv->dx[i] > 0)) return fail("x nodes must increase");
    }
    for (int j = 0; j < ny; ++j) {
        Lv->dy[j] = Lv->yn[j + 1] - Lv->yn[j];
        Lv->yc[j] = 0.5 * (Lv->yn[j] + Lv->yn[j + 1]);
        if (!(Lv->dy[j] > 0)) return fail("y nodes must increase");
    }
    return 0;
}

/* Coarse grid by deleting every second grid line in each direction (Sec. 3.1). */
static int coarsen(const olev_t *F, olev_t *C)
{
    if (F->nx % 2 || F->ny % 2) return fail("cannot coarsen %dx%d", F->nx, F->ny);
    C->nx = F->nx / 2; C->ny = F->ny / 2; C->nc = C->nx * C->ny;
    C->nfx = (C->nx + 1) * C->ny; C->nfy = C->nx * (C->ny + 1);
    C->xn = dalloc(C->nx + 1); C->yn = dalloc(C->ny + 1);
    for (int I = 0; I <= C->nx; ++I) C->xn[I] = F->xn[2 * I];
    for (int J = 0; J <= C->ny; ++J) C->yn[J] = F->yn[2 * J];
    C->fbx = (int *)calloc(C->nfx, sizeof(int));
    C->fby = (int *)calloc(C->nfy, sizeof(int));
    C->solid = (unsigned char *)calloc(C->nc, 1);
    C->nfluid = 0;
    for (int J = 0; J < C->ny; ++J)
        for (int I = 0; I < C->nx; ++I) {
            int ns = 0;
            for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a) ns += F->solid[(2 * J + b) * F->nx + 2 * I + a];
            if (ns != 0 && ns != 4) return fail("solid cells must fill whole coarse cells (coarse cell %d,%d)", I, J);
            C->solid[J * C->nx + I] = ns == 4;
            C->nfluid += ns == 0;
        }
    for (int J = 0; J < C->ny; ++J)
        for (int I = 0; I <= C->nx; ++I) {
            int a = F->fbx[(2 * J) * (F->nx + 1) + 2 * I], b = F->fbx[(2 * J + 1) * (F->nx + 1) + 2 * I];
            if (a != b) return fail("coarse x-face (%d,%d) spans two boundary ids", I, J);
            C->fbx[J * (C->nx + 1) + I] = a;
        }
    for (int J = 0; J <= C->ny; ++J)
        for (int I = 0; I < C->nx; ++I) {
            int a = F->fby[(2 * J) * F->nx + 2 * I], b = F->fby[(2 * J) * F->nx + 2 * I + 1];
            if (a != b) return fail("coarse y-face (%d,%d) spans two boundary ids", I, J);
            C->fby[J * C->nx + I] = a;
        }
    return level_geom(C);
}

/* Boundary faces of cell (i, j) on one sweep side: side 0 = lower (west, south),
 * side 1 = upper (east, north), side 2 = all. */
static int cell_bfaces(const olev_t *Lv, int i, int j, int side, bface_t *bf)
{
    int n = 0, nx = Lv->nx;
    double V = Lv->dx[i] * Lv->dy[j];
    int w = Lv->fbx[j * (nx + 1) + i], e = Lv->fbx[j * (nx + 1) + i + 1];
    int so = Lv->fby[j * nx + i], no = Lv->fby[(j + 1) * nx + i];
    if (side != 1 && w >= 0) bf[n++] = (bface_t){w, 0, -1, Lv->dy[j], V};
    if (side != 1 && so >= 0) bf[n++] = (bface_t){so, 1, -1, Lv->dx[i], V};
    if (side != 0 && e >= 0) bf[n++] = (bface_t){e, 0, +1, Lv->dy[j], V};
    if (side != 0 && no >= 0) bf[n++] = (bface_t){no, 1, +1, Lv->dx[i], V};
    return n;
}

/* The fluid cell of boundary face (i, j) along `axis` (x-face i in 0..nx, or
 * y-face j in 0..ny) and the sign of the face's outward normal seen from it:
 * the face lies on the domain edge or between a fluid and a solid cell. */
static void face_side(const olev_t *Lv, int axis, int i, int j, int *c, int *outsign)
{
    int nx = Lv->nx;
    if (axis == 0) {
        int lo_fluid = i > 0 && !Lv->solid[j * nx + i - 1];
        *c = lo_fluid ? j * nx + i - 1 : j * nx + i;
        *outsign = lo_fluid ? +1 : -1;
    } else {
        int lo_fluid = j > 0 && !Lv->solid[(j - 1) * nx + i];
        *c = lo_fluid ? (j - 1) * nx + i : j * nx + i;
        *outsign = lo_fluid ? +1 : -1;
    }
}

/* ------------------------------------------------------------------ */
/* Step 1: explicit UGKS fluxes and residuals (Eqs. macroResidualDef,   */
/* macroResidualCalc, microResidualDef)                                 */
/* ------------------------------------------------------------------ */

#define FIX(s, comp, c, k) ((s)->f[((size_t)(comp) * (s)->lev[0].nc + (c)) * (s)->nv + (k)])

/* Interior face between cells cL (lower) and cR (upper) along `axis`; cLL /
 * cRR are the next cells outward (-1 where the neighbour is a boundary ghost:
 * first order there).  Writes the time-averaged micro flux per velocity
 * (G, H) and the macro flux F = sum_k w psi flux.  */
static void interior_face(oracle_solver *s, int axis, int cLL, int cL, int cR, int cRR,
                          double dLLL, double dLR, double dRRR, double hL, double hR,
                          double wL, double wR, double *phG, double *phH, double F[4])
{
    int nv = s->nv;
    const double *u = s->u, *v = s->v, *w = s->w;
    double *f0 = s->tmp0 + (size_t)ORC_TID * 2 * nv, *sg = s->tmp1 + (size_t)ORC_TID * 2 * nv; /* [comp][k] */
    /* reconstruction (van Leer) and upwinding of the initial distribution */
    for (int k = 0; k < nv; ++k) {
        double un = axis == 0 ? u[k] : v[k];
        for (int cp = 0; cp < 2; ++cp) {
            double fL = FIX(s, cp, cL, k), fR = FIX(s, cp, cR, k);
            double sL = 0.0, sR = 0.0;
            if (cLL >= 0) sL = oracle_vanleer((fL - FIX(s, cp, cLL, k)) / dLLL, (fR - fL) / dLR);
            if (cRR >= 0) sR = oracle_vanleer((fR - fL) / dLR, (FIX(s, cp, cRR, k) - fR) / dRRR);
            double faceL = fL + sL * hL, faceR = fR - sR * hR;
            if (un > 0) { f0[cp * nv + k] = faceL; sg[cp * nv + k] = sL; }
            else if (un < 0) { f0[cp * nv + k] = faceR; sg[cp * nv + k] = sR; }
            else { f0[cp * nv + k] = 0.5 * (faceL + faceR); sg[cp * nv + k] = 0.5 * (sL + sR); }
        }
    }
    /* interface conservative variables from the upwinded distribution */
    double W0[4] = {0, 0, 0, 0};
    for (int k = 0; k < nv; ++k) {
        double g = f0[k], h = f0[nv + k];
        W0[0] += w[k] * g;
        W0[1] += w[k] * u[k] * g;
        W0[2] += w[k] * v[k] * g;
        W0[3] += w[k] * (0.5 * (u[k] * u[k] + v[k] * v[k]) * g + h);
    }
    double rho0, U0, V0, lam0;
    prim(W0, &rho0, &U0, &V0, &lam0);
    double tau0 = tau_of(s, rho0, lam0);
    double dt = face_dt(s, axis, wL, wR);
    /* equilibrium slopes on either side from the cell averages */
    const double *WL = s->W + 4 * cL, *WR = s->W + 4 * cR;
    if (s->shock) {
        /* shock capturing (off by default; the paper is silent, reading): the
         * interface collision time gains the pressure-jump term of the gas-kinetic
         * schemes, dt |p_L - p_R| / (p_L + p_R), p = rho / (2 lambda) of the cells */
        double rl, ul, vl, ll, rr, ur, vr, lr;
        prim(WL, &rl, &ul, &vl, &ll);
        prim(WR, &rr, &ur, &vr, &lr);
        double pl = rl / (2.0 * ll), pr = rr / (2.0 * lr);
        tau0 += dt * fabs(pl - pr) / (pl + pr);
    }
    double dwl[4], dwr[4], aL[4], aR[4];
    for (int m = 0; m < 4; ++m) {
        dwl[m] = (W0[m] - WL[m]) / hL / rho0;
        dwr[m] = (WR[m] - W0[m]) / hR / rho0;
    }
    oracle_micro_slope(dwl, U0, V0, lam0, aL);
    oracle_micro_slope(dwr, U0, V0, lam0, aR);
    /* heat flux of the interface distribution (Shakhov) and the time slope A
     * from compatibility: sum_k w psi (u_n a + A) g0 = 0 */
    double q0[2] = {0, 0}, Mt[4] = {0, 0, 0, 0};
    for (int k = 0; k < nv; ++k) {
        double cx = u[k] - U0, cy = v[k] - V0, c2 = cx * cx + cy * cy;
        double g = f0[k], h = f0[nv + k];
        q0[0] += w[k] * cx * (0.5 * c2 * g + h);
        q0[1] += w[k] * cy * (0.5 * c2 * g + h);
        double un = axis == 0 ? u[k] : v[k];
        if (un == 0.0) continue;
        double gM = maxw(rho0, U0, V0, lam0, u[k], v[k]), hM = gM * KINT / (4.0 * lam0);
        double mG, mH;
        slope_moments(un > 0 ? aL : aR, u[k], v[k], gM, hM, lam0, &mG, &mH);
        Mt[0] += w[k] * un * mG;
        Mt[1] += w[k] * un * u[k] * mG;
        Mt[2] += w[k] * un * v[k] * mG;
        Mt[3] += w[k] * un * (0.5 * (u[k] * u[k] + v[k] * v[k]) * mG + mH);
    }
    double dwt[4], A[4];
    for (int m = 0; m < 4; ++m) dwt[m] = -Mt[m] / rho0;
    oracle_micro_slope(dwt, U0, V0, lam0, A);
    double qc[5];
    oracle_time_coeffs(dt, tau0, qc);
    for (int m = 0; m < 4; ++m) F[m] = 0.0;
    for (int k = 0; k < nv; ++k) {
        double un = axis == 0 ? u[k] : v[k];
        double gM = maxw(rho0, U0, V0, lam0, u[k], v[k]), hM = gM * KINT / (4.0 * lam0);
        double gP, hP;
        shakhov(rho0, U0, V0, lam0, q0[0], q0[1], s->pr, u[k], v[k], &gP, &hP);
        double mGa, mHa, mGA, mHA;
        slope_moments(un > 0 ? aL : aR, u[k], v[k], gM, hM, lam0, &mGa, &mHa);
        slope_moments(A, u[k], v[k], gM, hM, lam0, &mGA, &mHA);
        double PG = un * (qc[0] * gP + qc[1] * un * mGa + qc[2] * mGA + qc[3] * f0[k] + qc[4] * un * sg[k]);
        double PH = un * (qc[0] * hP + qc[1] * un * mHa + qc[2] * mHA + qc[3] * f0[nv + k] + qc[4] * un * sg[nv + k]);
        phG[k] = PG / dt;
        phH[k] = PH / dt;
        F[0] += w[k] * phG[k];
        F[1] += w[k] * u[k] * phG[k];
        F[2] += w[k] * v[k] * phG[k];
        F[3] += w[k] * (0.5 * (u[k] * u[k] + v[k] * v[k]) * phG[k] + phH[k]);
    }
}

/* Distribution on a boundary face as seen from interior cell c (Sec. 3.2):
 * wall: diffuse reflection, incoming rho_w C_k with rho_w from zero mass flux,
 * both sums discrete; symmetry: mirrored velocity; farfield: freestream
 * Maxwellian incoming; outflow: zero gradient.  Outgoing velocities carry the
 * cell value (first order at boundaries). */
static void boundary_face_f(const oracle_solver *s, int bcid, int axis, int outsign, int c,
                            double *fG, double *fH)
{
    int nv = s->nv;
    const obc_t *b = &s->bc[bcid];
    double rhow = 0.0, lamw = 1.0 / b->t;
    if (b->type == ORC_BC_WALL) {
        double num = 0.0, den = 0.0;
        for (int k = 0; k < nv; ++k) {
            double uo = outsign * (axis == 0 ? s->u[k] : s->v[k]);
            if (uo > 0) num += s->w[k] * uo * FIX(s, 0, c, k);
            else if (uo < 0) den += s->w[k] * uo * s->Cw[(size_t)bcid * nv + k];
        }
        rhow = -num / den;
    }
    for (int k = 0; k < nv; ++k) {
        double uo = outsign * (axis == 0 ? s->u[k] : s->v[k]);
        if (uo >= 0 || b->type == ORC_BC_OUTFLOW) {
            fG[k] = FIX(s, 0, c, k); fH[k] = FIX(s, 1, c, k);
        } else if (b->type == ORC_BC_WALL) {
            double C = s->Cw[(size_t)bcid * nv + k];
            fG[k] = rhow * C; fH[k] = rhow * C * KINT / (4.0 * lamw);
        } else if (b->type == ORC_BC_SYMMETRY) {
            int km = axis == 0 ? s->mxk[k] : s->myk[k];
            fG[k] = FIX(s, 0, c, km); fH[k] = FIX(s, 1, c, km);
        } else { /* farfield */
            double g = maxw(b->rho, b->u, b->v, lamw, s->u[k], s->v[k]);
            fG[k] = g; fH[k] = g * KINT / (4.0 * lamw);
        }
    }
}

/* Boundary face flux: free transport of the face distribution, time-averaged,
 * oriented along +axis like the interior faces. */
static void boundary_face(oracle_solver *s, int bcid, int axis, int outsign, int c,
                          double *phG, double *phH, double F[4])
{
    int nv = s->nv;
    double *fG = s->tmp2 + (size_t)ORC_TID * 2 * nv, *fH = fG + nv;
    boundary_face_f(s, bcid, axis, outsign, c, fG, fH);
    for (int m = 0; m < 4; ++m) F[m] = 0.0;
    for (int k = 0; k < nv; ++k) {
        double un = axis == 0 ? s->u[k] : s->v[k];
        phG[k] = un * fG[k];
        phH[k] = un * fH[k];
        F[0] += s->w[k] * phG[k];
        F[1] += s->w[k] * s->u[k] * phG[k];
        F[2] += s->w[k] * s->v[k] * phG[k];
        F[3] += s->w[k] * (0.5 * (s->u[k] * s->u[k] + s->v[k] * s->v[k]) * phG[k] + phH[k]);
    }
}

/* All face fluxes on level 0 and the macroscopic residual
 * R_i = -(1/V_i) sum_j S_ij F_ij (Eq. macroResidualDef). */
static void flux_stage(oracle_solver *s)
{
    olev_t *Lv = &s->lev[0];
    int nx = Lv->nx, ny = Lv->ny, nv = s->nv;
    size_t nfx = Lv->nfx, nfy = Lv->nfy;
#pragma omp parallel for num_threads(s->nthr) schedule(dynamic, 1)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i <= nx; ++i) {
            int fi = j * (nx + 1) + i;
            double *pG = s->phx + (size_t)fi * nv, *pH = s->phx + (nfx + fi) * (size_t)nv;
            int bcid = Lv->fbx[fi];
            if (bcid >= 0) {
                int c, os;
                face_side(Lv, 0, i, j, &c, &os);
                boundary_face(s, bcid, 0, os, c, pG, pH, s->Fx + 4 * fi);
                continue;
            }
            int cL = j * nx + i - 1, cR = j * nx + i;
            if (i == 0 || i == nx || Lv->solid[cL] || Lv->solid[cR]) { /* a face inside a body */
                memset(s->Fx + 4 * fi, 0, 4 * sizeof(double));
                for (int k = 0; k < nv; ++k) pG[k] = pH[k] = 0.0;
                continue;
            }
            int hasLL = (i - 1 > 0) && Lv->fbx[fi - 1] < 0;
            int hasRR = (i + 1 < nx) && Lv->fbx[fi + 1] < 0;
            interior_face(s, 0, hasLL ? cL - 1 : -1, cL, cR, hasRR ? cR + 1 : -1,
                          hasLL ? Lv->xc[i - 1] - Lv->xc[i - 2] : 1.0, Lv->xc[i] - Lv->xc[i - 1],
                          hasRR ? Lv->xc[i + 1] - Lv->xc[i] : 1.0,
                          Lv->xn[i] - Lv->xc[i - 1], Lv->xc[i] - Lv->xn[i],
                          Lv->dx[i - 1], Lv->dx[i], pG, pH, s->Fx + 4 * fi);
        }
#pragma omp parallel for num_threads(s->nthr) schedule(dynamic, 1)
    for (int j = 0; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int fi = j * nx + i;
            double *pG = s->phy + (size_t)fi * nv, *pH = s->phy + (nfy + fi) * (size_t)nv;
            int bcid = Lv->fby[fi];
            if (bcid >= 0) {
                int c, os;
                face_side(Lv, 1, i, j, &c, &os);
                boundary_face(s, bcid, 1, os, c, pG, pH, s->Fy + 4 * fi);
                continue;
            }
            int cL = (j - 1) * nx + i, cR = j * nx + i;
            if (j == 0 || j == ny || Lv->solid[cL] || Lv->solid[cR]) {
                memset(s->Fy + 4 * fi, 0, 4 * sizeof(double));
                for (int k = 0; k < nv; ++k) pG[k] = pH[k] = 0.0;
                continue;
            }
            int hasLL = (j - 1 > 0) && Lv->fby[fi - nx] < 0;
            int hasRR = (j + 1 < ny) && Lv->fby[fi + nx] < 0;
            interior_face(s, 1, hasLL ? cL - nx : -1, cL, cR, hasRR ? cR + nx : -1,
                          hasLL ? Lv->yc[j - 1] - Lv->yc[j - 2] : 1.0, Lv->yc[j] - Lv->yc[j - 1],
                          hasRR ? Lv->yc[j + 1] - Lv->yc[j] : 1.0,
                          Lv->yn[j] - Lv->yc[j - 1], Lv->yc[j] - Lv->yn[j],
                          Lv->dy[j - 1], Lv->dy[j], pG, pH, s->Fy + 4 * fi);
        }
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int c = j * nx + i;
            double V = Lv->dx[i] * Lv->dy[j];
            const double *FW = s->Fx + 4 * (j * (nx + 1) + i), *FE = FW + 4;
            const double *FS = s->Fy + 4 * (j * nx + i), *FN = s->Fy + 4 * ((j + 1) * nx + i);
            for (int m = 0; m < 4; ++m)
                s->R[4 * c + m] = Lv->solid[c] ? 0.0 : -(Lv->dy[j] * (FE[m] - FW[m]) + Lv->dx[i] * (FN[m] - FS[m])) / V;
        }
}

/* ------------------------------------------------------------------ */
/* Prediction step: split Euler flux, FAS (Secs. 2.1.1, 2.3, 2.4, 3.2) */
/* ------------------------------------------------------------------ */

/* Euler flux T(W).n */
static void euler_flux(const double *W, int axis, double sgn, double T[4])
{
    double rho, U, V, lam;
    prim(W, &rho, &U, &V, &lam);
    double p = rho / (2.0 * lam);
    double nx_ = axis == 0 ? sgn : 0.0, ny_ = axis == 1 ? sgn : 0.0;
    double Un = U * nx_ + V * ny_;
    T[0] = rho * Un;
    T[1] = W[1] * Un + p * nx_;
    T[2] = W[2] * Un + p * ny_;
    T[3] = (W[3] + p) * Un;
}

/* Ghost state W_j = B(W_i) of a boundary face and its Jacobian dB/dW
 * (Eqs. boundaryRelation, boundaryWall, example_results).  Reading of the
 * garbled wall relation: rho_j V_j = 2 rho_i V_w - rho_i V_i, and U_0, V_0 in
 * the Jacobian are the wall velocity. */
void oracle_wall_ghost(const double W[4], double Uw, double Vw, double Tw, double Wg[4])
{
    double rho, U, V, lam;
    prim(W, &rho, &U, &V, &lam);
    double lamg = 2.0 / Tw - lam, Ug = 2.0 * Uw - U, Vg = 2.0 * Vw - V;
    Wg[0] = rho;
    Wg[1] = rho * Ug;
    Wg[2] = rho * Vg;
    Wg[3] = 0.5 * rho * (Ug * Ug + Vg * Vg) + (KINT + 2) * rho / (4.0 * lamg);
}

void oracle_wall_jacobian(const double W[4], double Uw, double Vw, double Tw, double M[16])
{
    double rho, U, V, lam;
    prim(W, &rho, &U, &V, &lam);
    double lamw = 1.0 / Tw, Y = lam / (lam - 2.0 * lamw), K = KINT + 2.0;
    memset(M, 0, 16 * sizeof(double));
    M[0] = 1.0;
    M[4] = 2.0 * Uw; M[5] = -1.0;
    M[8] = 2.0 * Vw; M[10] = -1.0;
    M[12] = 2.0 * (Uw * Uw + Vw * Vw) - 0.5 * (U * U + V * V) * (1.0 + Y * Y) + K / (4.0 * lam) * (Y * Y - Y);
    M[13] = U - 2.0 * Uw + U * Y * Y;
    M[14] = V - 2.0 * Vw + V * Y * Y;
    M[15] = -Y * Y;
}

static void macro_ghost(const oracle_solver *s, int bcid, int axis, const double *Wi, double Wg[4], double M[16])
{
    const obc_t *b = &s->bc[bcid];
    if (b->type == ORC_BC_WALL) {
        oracle_wall_ghost(Wi, b->u, b->v, b->t, Wg);
        if (M) oracle_wall_jacobian(Wi, b->u, b->v, b->t, M);
    } else if (b->type == ORC_BC_SYMMETRY) {
        for (int m = 0; m < 4; ++m) Wg[m] = Wi[m];
        Wg[1 + axis] = -Wi[1 + axis];
        if (M) {
            memset(M, 0, 16 * sizeof(double));
            for (int m = 0; m < 4; ++m) M[5 * m] = 1.0;
            M[5 * (1 + axis)] = -1.0;
        }
    } else if (b->type == ORC_BC_FARFIELD) {
        double lam = 1.0 / b->t;
        Wg[0] = b->rho; Wg[1] = b->rho * b->u; Wg[2] = b->rho * b->v;
        Wg[3] = 0.5 * b->rho * (b->u * b->u + b->v * b->v) + (KINT + 2) * b->rho / (4.0 * lam);
        if (M) memset(M, 0, 16 * sizeof(double));
    } else {
        for (int m = 0; m < 4; ++m) Wg[m] = Wi[m];
        if (M) {
            memset(M, 0, 16 * sizeof(double));
            for (int m = 0; m < 4; ++m) M[5 * m] = 1.0;
        }
    }
}

/* Gamma_ij = |U_ij . n| + a_s + 2 nu / (n . (x_j - x_i)) at the arithmetic mean
 * of the two conservative states (Eq. predictionSpectralRadius). */
static double gamma_face(const oracle_solver *s, const double *Wa, const double *Wb, int axis, double dist)
{
    double Wm[4], rho, U, V, lam;
    for (int m = 0; m < 4; ++m) Wm[m] = 0.5 * (Wa[m] + Wb[m]);
    prim(Wm, &rho, &U, &V, &lam);
    double gam = (KINT + 4.0) / (KINT + 2.0);
    double as = sqrt(gam / (2.0 * lam));
    double nu = s->mu_ref * pow(1.0 / lam, s->omega) / rho;
    return fabs(axis == 0 ? U : V) + as + 2.0 * nu / dist;
}

/* split flux 1/2 [T_a + T_b + Gamma (W_a - W_b)] along the normal from a to b (Eq. macroFluxSplitting) */
static void split_flux(const double *Wa, const double *Wb, int axis, double sgn, double gam, double F[4])
{
    double Ta[4], Tb[4];
    euler_flux(Wa, axis, sgn, Ta);
    euler_flux(Wb, axis, sgn, Tb);
    for (int m = 0; m < 4; ++m) F[m] = 0.5 * (Ta[m] + Tb[m] + gam * (Wa[m] - Wb[m]));
}

/* Gamma of the four faces of cell c on level Lv, from the frozen state Wg */
static void cell_gammas(const oracle_solver *s, const olev_t *Lv, const double *Wg, int i, int j, double gm[4])
{
    int nx = Lv->nx, ny = Lv->ny, c = j * nx + i;
    double G[4];
    /* west, east, south, north */
    for (int f = 0; f < 4; ++f) {
        int axis = f / 2, up = f % 2;
        int bcid = axis == 0 ? Lv->fbx[j * (nx + 1) + i + up] : Lv->fby[(j + up) * nx + i];
        if (bcid >= 0) {
            macro_ghost(s, bcid, axis, Wg + 4 * c, G, NULL);
            gm[f] = gamma_face(s, Wg + 4 * c, G, axis, axis == 0 ? Lv->dx[i] : Lv->dy[j]);
        } else {
            int nb = axis == 0 ? c + (up ? 1 : -1) : c + (up ? nx : -nx);
            double dist = axis == 0 ? fabs(Lv->xc[i + (up ? 1 : -1)] - Lv->xc[i])
                                    : fabs(Lv->yc[j + (up ? 1 : -1)] - Lv->yc[j]);
            gm[f] = gamma_face(s, Wg + 4 * c, Wg + 4 * nb, axis, dist);
        }
    }
    (void)ny;
}

/* R_E(W) = -(1/V_i) sum_j S_ij F_split(W_i, W_j), Gamma frozen at Wg (Eq. forcingFunction) */
static void resid_macro(const oracle_solver *s, const olev_t *Lv, const double *W, const double *Wg, double *RE)
{
    int nx = Lv->nx, ny = Lv->ny;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int c = j * nx + i;
            if (Lv->solid[c]) { for (int m = 0; m < 4; ++m) RE[4 * c + m] = 0.0; continue; }
            double V = Lv->dx[i] * Lv->dy[j], gm[4], acc[4] = {0, 0, 0, 0};
            cell_gammas(s, Lv, Wg, i, j, gm);
            for (int f = 0; f < 4; ++f) {
                int axis = f / 2, up = f % 2;
                double sgn = up ? 1.0 : -1.0, S = axis == 0 ? Lv->dy[j] : Lv->dx[i], F[4], G[4];
                int bcid = axis == 0 ? Lv->fbx[j * (nx + 1) + i + up] : Lv->fby[(j + up) * nx + i];
                if (bcid >= 0) {
                    macro_ghost(s, bcid, axis, W + 4 * c, G, NULL);
                    split_flux(W + 4 * c, G, axis, sgn, gm[f], F);
                } else {
                    int nb = axis == 0 ? c + (up ? 1 : -1) : c + (up ? nx : -nx);
                    split_flux(W + 4 * c, W + 4 * nb, axis, sgn, gm[f], F);
                }
                for (int m = 0; m < 4; ++m) acc[m] += S * F[m];
            }
            for (int m = 0; m < 4; ++m) RE[4 * c + m] = -acc[m] / V;
        }
}

static double dtn_inv(const oracle_solver *s)
{
    if (!(s->dtn_growth > 0.0)) return 0.0;
    return 1.0 / (pow(s->dtn_growth, (double)s->iter) * s->dtp_min);
}

/* One LU-SGS pass of Eq. macroFinalDefect with the split flux: forward sweep
 * with the lower neighbours (west, south), backward sweep with the upper ones
 * (east, north).  Boundary ghosts dW_j = (dB/dW) dW_i take dW_i from the
 * previous half sweep (zero in the forward sweep).  order 1 runs the same
 * sweeps over anti-diagonals (identical arithmetic per cell). */
static void sgs_macro(const oracle_solver *s, const olev_t *Lv, const double *W, const double *Wg,
                      const double *R, double *dW, int order)
{
    int nx = Lv->nx, ny = Lv->ny, nd = nx + ny - 1;
    double add = dtn_inv(s);
    for (int pass = 0; pass < 2; ++pass) {
        int ncell = nx * ny;
        for (int t = 0; t < ncell; ++t) {
            int i, j;
            if (order == 0) {
                int tt = pass == 0 ? t : ncell - 1 - t;
                i = tt % nx; j = tt / nx;
            } else {
                /* t-th cell in diagonal order */
                int cnt = 0, found = 0;
                for (int d0 = 0; d0 < nd && !found; ++d0) {
                    int d = pass == 0 ? d0 : nd - 1 - d0;
                    int ilo = d - (ny - 1) > 0 ? d - (ny - 1) : 0, ihi = d < nx - 1 ? d : nx - 1;
                    if (t < cnt + (ihi - ilo + 1)) {
                        int off = t - cnt;
                        i = pass == 0 ? ilo + off : ihi - off;
                        j = d - i;
                        found = 1;
                    }
                    cnt += ihi - ilo + 1;
                }
            }
            int c = j * nx + i;
            if (Lv->solid[c]) { for (int m = 0; m < 4; ++m) dW[4 * c + m] = 0.0; continue; }
            double V = Lv->dx[i] * Lv->dy[j], gm[4];
            cell_gammas(s, Lv, Wg, i, j, gm);
            double diag = 0.0;
            for (int f = 0; f < 4; ++f) diag += (f / 2 == 0 ? Lv->dy[j] : Lv->dx[i]) * gm[f];
            diag = diag / (2.0 * V) + add;
            double acc[4] = {0, 0, 0, 0};
            for (int f = 0; f < 4; ++f) {
                int axis = f / 2, up = f % 2;
                if (up != pass) continue; /* forward: lower faces, backward: upper faces */
                double sgn = up ? 1.0 : -1.0, S = axis == 0 ? Lv->dy[j] : Lv->dx[i];
                int bcid = axis == 0 ? Lv->fbx[j * (nx + 1) + i + up] : Lv->fby[(j + up) * nx + i];
                double Wn[4], dWn[4], Wp[4], T1[4], T0[4];
                if (bcid >= 0) {
                    double M[16];
                    macro_ghost(s, bcid, axis, W + 4 * c, Wn, M);
                    for (int m = 0; m < 4; ++m) {
                        dWn[m] = 0.0;
                        if (pass == 1)
                            for (int q = 0; q < 4; ++q) dWn[m] += M[4 * m + q] * dW[4 * c + q];
                    }
                } else {
                    int nb = axis == 0 ? c + (up ? 1 : -1) : c + (up ? nx : -nx);
                    for (int m = 0; m < 4; ++m) { Wn[m] = W[4 * nb + m]; dWn[m] = dW[4 * nb + m]; }
                }
                for (int m = 0; m < 4; ++m) Wp[m] = Wn[m] + dWn[m];
                euler_flux(Wp, axis, sgn, T1);
                euler_flux(Wn, axis, sgn, T0);
                for (int m = 0; m < 4; ++m) acc[m] += S * ((T1[m] - T0[m]) - gm[f] * dWn[m]);
            }
            if (pass == 0)
                for (int m = 0; m < 4; ++m) dW[4 * c + m] = (R[4 * c + m] - acc[m] / (2.0 * V)) / diag;
            else
                for (int m = 0; m < 4; ++m) dW[4 * c + m] = dW[4 * c + m] - acc[m] / (2.0 * V * diag);
        }
    }
}

/* ------------------------------------------------------------------ */
/* Transfer operators (Secs. 2.3.1, 2.3.3)                             */
/* ------------------------------------------------------------------ */

/* Volume-weighted restriction of an [cell][m] array from level l to l+1 */
static void restrict_lv(const olev_t *F, const olev_t *C, int m, const double *fine, double *coarse)
{
#pragma omp parallel for schedule(static) if (m > 4)
    for (int J = 0; J < C->ny; ++J)
        for (int I = 0; I < C->nx; ++I) {
            double *out = coarse + (size_t)(J * C->nx + I) * m;
            double vs = 0.0;
            for (int q = 0; q < m; ++q) out[q] = 0.0;
            for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a) {
                    int i = 2 * I + a, j = 2 * J + b;
                    double V = F->dx[i] * F->dy[j];
                    const double *in = fine + (size_t)(j * F->nx + i) * m;
                    for (int q = 0; q < m; ++q) out[q] += in[q] * V;
                    vs += V;
                }
            for (int q = 0; q < m; ++q) out[q] /= vs;
        }
}

static int fluid_at(const olev_t *C, int I, int J)
{
    return I >= 0 && I < C->nx && J >= 0 && J < C->ny && !C->solid[J * C->nx + I];
}

/* Prolongation stencil of fine cell (i, j) in coarse cell (I, J): the coarse
 * neighbour along each axis is the one on the side of the fine centre, or the
 * one on the other side (extrapolation, signed weights) when that one lies
 * outside the domain or in a body; with neither, the axis is constant.  When
 * the diagonal cell of the two chosen neighbours lies in a body (a fine cell
 * diagonal to a body's corner), the first pair of x- and y-options (preferred
 * side first, x outer) whose three cells are fluid is taken; with none, the
 * y-axis is dropped.  Without bodies this is the plain bilinear stencil with
 * one-sided extrapolation at the domain edges. */
static void stencil(const olev_t *F, const olev_t *C, int i, int j, int *IN, int *JN, double *wx, double *wy)
{
    int I = i / 2, J = j / 2;
    double x = F->xc[i], y = F->yc[j];
    int ox[2], oy[2], nox = 0, noy = 0;
    int sx = x < C->xc[I] ? -1 : 1, sy = y < C->yc[J] ? -1 : 1;
    for (int q = 0; q < 2; ++q) {
        int a = I + (q == 0 ? sx : -sx), b = J + (q == 0 ? sy : -sy);
        if (fluid_at(C, a, J)) ox[nox++] = a;
        if (fluid_at(C, I, b)) oy[noy++] = b;
    }
    int ix = nox ? ox[0] : I, jy = noy ? oy[0] : J;
    if (nox && noy && !fluid_at(C, ix, jy)) {
        int found = 0;
        for (int p = 0; p < nox && !found; ++p)
            for (int q = 0; q < noy && !found; ++q)
                if (fluid_at(C, ox[p], oy[q])) { ix = ox[p]; jy = oy[q]; found = 1; }
        if (!found) jy = J;
    }
    *IN = ix; *JN = jy;
    /* 1-D linear weights of the own and the neighbour centre */
    wx[0] = 1.0; wx[1] = 0.0; wy[0] = 1.0; wy[1] = 0.0;
    if (ix != I) { wx[0] = (C->xc[ix] - x) / (C->xc[ix] - C->xc[I]); wx[1] = (x - C->xc[I]) / (C->xc[ix] - C->xc[I]); }
    if (jy != J) { wy[0] = (C->yc[jy] - y) / (C->yc[jy] - C->yc[J]); wy[1] = (y - C->yc[J]) / (C->yc[jy] - C->yc[J]); }
}

/* Bilinear prolongation from level l+1 to l (Eqs. prolongation, prolongationWeight):
 * on a rectilinear mesh the weights h_BC h_CD / S_ABCD etc. are the products of
 * the 1-D linear weights in each direction.  Cells in a body receive zero (a
 * correction), or their coarse cell's value with inject_solid (a state). */
static void prolong_lv_s(const olev_t *F, const olev_t *C, int m, const double *coarse, double *fine, int inject_solid)
{
#pragma omp parallel for schedule(static) if (m > 4)
    for (int j = 0; j < F->ny; ++j)
        for (int i = 0; i < F->nx; ++i) {
            int I = i / 2, J = j / 2, IN, JN;
            double *out = fine + (size_t)(j * F->nx + i) * m;
            const double *A = coarse + (size_t)(J * C->nx + I) * m;
            if (F->solid[j * F->nx + i]) {
                for (int q = 0; q < m; ++q) out[q] = inject_solid ? A[q] : 0.0;
                continue;
            }
            double wx[2], wy[2];
            stencil(F, C, i, j, &IN, &JN, wx, wy);
            const double *B = coarse + (size_t)(J * C->nx + IN) * m;
            const double *D = coarse + (size_t)(JN * C->nx + I) * m, *Cc = coarse + (size_t)(JN * C->nx + IN) * m;
            for (int q = 0; q < m; ++q)
                out[q] = wx[0] * wy[0] * A[q] + wx[1] * wy[0] * B[q] + wx[0] * wy[1] * D[q] + wx[1] * wy[1] * Cc[q];
        }
}
static void prolong_lv(const olev_t *F, const olev_t *C, int m, const double *coarse, double *fine)
{
    prolong_lv_s(F, C, m, coarse, fine, 0);
}

static double sumsq(const double *a, size_t n)
{
    double t = 0.0;
    for (size_t q = 0; q < n; ++q) t += a[q] * a[q];
    return t;
}

/* FAS cycle (Eq. FASCYC): W_l <- FAS(l, W_l^n, R_l); lv->Wn holds W_l^n and
 * lv->Rc the restricted (or UGKS) residual on entry; the result is left in lv->Wc.
 * The cycle type (Sec. 3.4) sets the coarse visits of a level: V one visit, W
 * two W visits, F one F visit then one V visit, adaptive one adaptive visit and
 * a second one when the first did not reduce the coarse residual five-fold.  A visit after the first starts
 * from the coarse state the previous one left, with the same forcing function
 * and the same frozen Gamma. */
static void fas_visit(oracle_solver *s, int l, int type, int first);

static void fas(oracle_solver *s, int l, int type)
{
    olev_t *Lv = &s->lev[l];
    size_t n4 = 4 * (size_t)Lv->nc;
    resid_macro(s, Lv, Lv->Wn, Lv->Wn, Lv->RE);
    for (size_t q = 0; q < n4; ++q) Lv->P[q] = Lv->Rc[q] - Lv->RE[q]; /* forcing function */
    memcpy(Lv->Wc, Lv->Wn, n4 * sizeof(double));
    fas_visit(s, l, type, 1);
}

static void fas_visit(oracle_solver *s, int l, int type, int first)
{
    olev_t *Lv = &s->lev[l];
    size_t n4 = 4 * (size_t)Lv->nc;
    double *R = (double *)malloc(n4 * sizeof(double));
    if (first) {
        memcpy(R, Lv->Rc, n4 * sizeof(double));
    } else {
        resid_macro(s, Lv, Lv->Wc, Lv->Wn, Lv->RE);
        for (size_t q = 0; q < n4; ++q) R[q] = Lv->P[q] + Lv->RE[q];
    }
    int coarsest = (l == s->L - 1);
    int npre = coarsest ? (s->L == 1 ? 1 : s->nuc) : s->nu1;
    for (int m = 0; m < npre; ++m) {
        sgs_macro(s, Lv, Lv->Wc, Lv->Wn, R, Lv->dW, 0);
        for (size_t q = 0; q < n4; ++q) Lv->Wc[q] += Lv->dW[q];
        if (coarsest && m == npre - 1) break;
        resid_macro(s, Lv, Lv->Wc, Lv->Wn, Lv->RE); /* renewal, Eq. renewResiduals */
        for (size_t q = 0; q < n4; ++q) R[q] = Lv->P[q] + Lv->RE[q];
    }
    if (!coarsest) {
        olev_t *Cv = &s->lev[l + 1];
        restrict_lv(Lv, Cv, 4, Lv->Wc, Cv->Wn);
        restrict_lv(Lv, Cv, 4, R, Cv->Rc);
        fas(s, l + 1, type);                                   /* first coarse visit, of this type */
        if (type == 1 || type == 2) fas_visit(s, l + 1, type == 1 ? 1 : 0, 0); /* W: another W visit; F: a V visit */
        if (type == 3) {
            /* adaptive: visit again while a visit leaves more than ADAPT_RATIO of the coarse
             * residual it started from (the coarse residual on entry is the restricted R) */
            size_t c4 = 4 * (size_t)Cv->nc;
            double *Rh = (double *)malloc(c4 * sizeof(double));
            double before = sumsq(Cv->Rc, c4);
            for (int visit = 1; visit < ADAPT_MAX_VISITS; ++visit) {
                resid_macro(s, Cv, Cv->Wc, Cv->Wn, Cv->RE);
                for (size_t q = 0; q < c4; ++q) Rh[q] = Cv->P[q] + Cv->RE[q];
                double after = sumsq(Rh, c4);
                s->adapt_log[s->adapt_n++ % ADAPT_LOG] = after > s->adapt_ratio * s->adapt_ratio * before;
                if (!(after > s->adapt_ratio * s->adapt_ratio * before)) break;
                before = after;
                fas_visit(s, l + 1, 3, 0);
            }
            free(Rh);
        }
        size_t c4 = 4 * (size_t)Cv->nc;
        for (size_t q = 0; q < c4; ++q) Cv->dW[q] = Cv->Wc[q] - Cv->Wn[q];
        double *corr = (double *)malloc(n4 * sizeof(double));
        prolong_lv(Lv, Cv, 4, Cv->dW, corr);
        /* W_l += P dW_H; a correction that would leave a cell without positive
         * density and internal energy is dropped there (reading: the paper is
         * silent; at a strong shock the bilinear correction can overshoot) */
        for (int c = 0; c < Lv->nc; ++c) {
            double w[4];
            for (int m = 0; m < 4; ++m) w[m] = Lv->Wc[4 * c + m] + corr[4 * c + m];
            double e2 = w[3] * w[0] - 0.5 * (w[1] * w[1] + w[2] * w[2]);
            if (w[0] > 0.0 && e2 > 0.0)
                for (int m = 0; m < 4; ++m) Lv->Wc[4 * c + m] = w[m];
        }
        free(corr);
        for (int m = 0; m < s->nu2; ++m) {
            resid_macro(s, Lv, Lv->Wc, Lv->Wn, Lv->RE);
            for (size_t q = 0; q < n4; ++q) R[q] = Lv->P[q] + Lv->RE[q];
            sgs_macro(s, Lv, Lv->Wc, Lv->Wn, R, Lv->dW, 0);
            for (size_t q = 0; q < n4; ++q) Lv->Wc[q] += Lv->dW[q];
        }
    }
    free(R);
}

/* ------------------------------------------------------------------ */
/* Evolution step: upwind micro system, LU-SGS, CS cycle (Secs. 2.1.2,  */
/* 2.3, 2.4, 3.2)                                                       */
/* ------------------------------------------------------------------ */

/* D_{i,k} = 1/tau_i (+1/dt_n) + (1/V_i) sum_{u_n > 0} u_n S_ij (Eq. evolutionCoefficients) */
static double Dii(const oracle_solver *s, const olev_t *Lv, int i, int j, double inv_tau, int k)
{
    double V = Lv->dx[i] * Lv->dy[j];
    return inv_tau + (fabs(s->u[k]) * Lv->dy[j] + fabs(s->v[k]) * Lv->dx[i]) / V;
}

/* D_{j,k} = (1/V_i) u_n S_ij for u_n < 0 through a face with outward normal outsign*axis */
static double Dij(const oracle_solver *s, int axis, int outsign, double S, double V, int k)
{
    double un = outsign * (axis == 0 ? s->u[k] : s->v[k]);
    return un < 0 ? un * S / V : 0.0;
}

static double wallC(const oracle_solver *s, int bcid, int comp, int k)
{
    double C = s->Cw[(size_t)bcid * s->nv + k];
    return comp == 0 ? C : C * KINT * s->bc[bcid].t / 4.0;
}

/* Solve one cell's own equations for one sweep side given base_k:
 *   D_k x_k + sum_{b: k incoming at b} D_bk ghost_bk(x) = base_k
 * Ghosts (Sec. 3.2): wall  rho_b C_k with rho_b = -sum_{out} w u_n x_k,G / sum_{in} w u_n C_k;
 * symmetry x_{k'} (mirror); farfield 0; outflow x_k.  Two walls on the same
 * side (a corner) couple through a 2x2 system for the two densities; every
 * other combination is resolved exactly by three substitution rounds. */
static void cell_solve(const oracle_solver *s, int c, int nb, const bface_t *bf, const double *D,
                       const double *base, double *x)
{
    int nv = s->nv;
    size_t nc = s->lev[0].nc; (void)nc;
    double *den = s->tmp0 + (size_t)ORC_TID * 2 * nv, *xo = s->tmp1 + (size_t)ORC_TID * 2 * nv;
    for (int k = 0; k < nv; ++k) {
        den[k] = D[k];
        for (int b = 0; b < nb; ++b)
            if (s->bc[bf[b].bc].type == ORC_BC_OUTFLOW) den[k] += Dij(s, bf[b].axis, bf[b].outsign, bf[b].S, bf[b].V, k);
    }
    int nwall = 0;
    for (int b = 0; b < nb; ++b) nwall += s->bc[bf[b].bc].type == ORC_BC_WALL;
    double Z[4], rho[4];
    for (int b = 0; b < nb; ++b) {
        Z[b] = 0.0;
        if (s->bc[bf[b].bc].type != ORC_BC_WALL) continue;
        for (int k = 0; k < nv; ++k) {
            double uo = bf[b].outsign * (bf[b].axis == 0 ? s->u[k] : s->v[k]);
            if (uo < 0) Z[b] += s->w[k] * uo * wallC(s, bf[b].bc, 0, k);
        }
    }
    if (nwall == 2 && nb == 2) {
        double cc[2] = {0, 0}, mm[2] = {0, 0}; /* mm[b] couples b to the other wall */
        for (int b = 0; b < 2; ++b) {
            int o = 1 - b;
            for (int k = 0; k < nv; ++k) {
                double uo = bf[b].outsign * (bf[b].axis == 0 ? s->u[k] : s->v[k]);
                if (!(uo > 0)) continue;
                cc[b] += s->w[k] * uo * base[k] / den[k];
                double Do = Dij(s, bf[o].axis, bf[o].outsign, bf[o].S, bf[o].V, k);
                if (Do != 0.0) mm[b] += s->w[k] * uo * Do * wallC(s, bf[o].bc, 0, k) / den[k];
            }
            cc[b] = -cc[b] / Z[b];
            mm[b] = mm[b] / Z[b];
        }
        rho[0] = (cc[0] + mm[0] * cc[1]) / (1.0 - mm[0] * mm[1]);
        rho[1] = cc[1] + mm[1] * rho[0];
        for (int cp = 0; cp < 2; ++cp)
            for (int k = 0; k < nv; ++k) {
                double acc = base[cp * nv + k];
                for (int b = 0; b < 2; ++b) {
                    double Db = Dij(s, bf[b].axis, bf[b].outsign, bf[b].S, bf[b].V, k);
                    if (Db != 0.0) acc -= Db * wallC(s, bf[b].bc, cp, k) * rho[b];
                }
                x[cp * nv + k] = acc / den[k];
            }
        return;
    }
    for (int cp = 0; cp < 2; ++cp)
        for (int k = 0; k < nv; ++k) x[cp * nv + k] = base[cp * nv + k] / den[k];
    double *xs = (double *)malloc(2 * (size_t)nv * sizeof(double));
    for (int round = 0; round < 3; ++round) {
        memcpy(xs, x, 2 * (size_t)nv * sizeof(double));
        for (int b = 0; b < nb; ++b) {
            if (s->bc[bf[b].bc].type != ORC_BC_WALL) continue;
            double num = 0.0;
            for (int k = 0; k < nv; ++k) {
                double uo = bf[b].outsign * (bf[b].axis == 0 ? s->u[k] : s->v[k]);
                if (uo > 0) num += s->w[k] * uo * xs[k];
            }
            rho[b] = -num / Z[b];
        }
        for (int cp = 0; cp < 2; ++cp)
            for (int k = 0; k < nv; ++k) {
                double acc = base[cp * nv + k];
                for (int b = 0; b < nb; ++b) {
                    double Db = Dij(s, bf[b].axis, bf[b].outsign, bf[b].S, bf[b].V, k);
                    if (Db == 0.0) continue;
                    int t = s->bc[bf[b].bc].type;
                    if (t == ORC_BC_WALL) acc -= Db * wallC(s, bf[b].bc, cp, k) * rho[b];
                    else if (t == ORC_BC_SYMMETRY) {
                        int km = bf[b].axis == 0 ? s->mxk[k] : s->myk[k];
                        acc -= Db * xs[cp * nv + km];
                    }
                }
                x[cp * nv + k] = acc / den[k];
            }
    }
    free(xs);
    (void)xo; (void)c;
}

#define AT(arr, nc_, nv_, cp, c, k) ((arr)[((size_t)(cp) * (nc_) + (c)) * (nv_) + (k)])

/* one cell (i, j) of a sweep pass: D, base and xc are scratch of nv, 2 nv, 2 nv */
static void sweep_cell(oracle_solver *s, const olev_t *Lv, const double *inv_tau, const double *r, double *x, int pass,
                       int i, int j, double *D, double *base, double *xc)
{
    int nx = Lv->nx, ny = Lv->ny, nv = s->nv;
    size_t nc = Lv->nc;
    int c = j * nx + i;
    if (Lv->solid[c]) {
        for (int cp = 0; cp < 2; ++cp)
            for (int k = 0; k < nv; ++k) AT(x, nc, nv, cp, c, k) = 0.0;
        return;
    }
    double V = Lv->dx[i] * Lv->dy[j];
    for (int k = 0; k < nv; ++k) D[k] = Dii(s, Lv, i, j, inv_tau[c], k);
    for (int cp = 0; cp < 2; ++cp)
        for (int k = 0; k < nv; ++k) {
            double y = 0.0;
            if (pass == 0) {
                if (i > 0 && Lv->fbx[j * (nx + 1) + i] < 0)
                    y += Dij(s, 0, -1, Lv->dy[j], V, k) * AT(x, nc, nv, cp, c - 1, k);
                if (j > 0 && Lv->fby[j * nx + i] < 0)
                    y += Dij(s, 1, -1, Lv->dx[i], V, k) * AT(x, nc, nv, cp, c - nx, k);
                base[cp * nv + k] = AT(r, nc, nv, cp, c, k) - y;
            } else {
                if (i < nx - 1 && Lv->fbx[j * (nx + 1) + i + 1] < 0)
                    y += Dij(s, 0, +1, Lv->dy[j], V, k) * AT(x, nc, nv, cp, c + 1, k);
                if (j < ny - 1 && Lv->fby[(j + 1) * nx + i] < 0)
                    y += Dij(s, 1, +1, Lv->dx[i], V, k) * AT(x, nc, nv, cp, c + nx, k);
                base[cp * nv + k] = D[k] * AT(x, nc, nv, cp, c, k) - y;
            }
        }
    bface_t bf[4];
    int nb = cell_bfaces(Lv, i, j, pass, bf);
    if (nb == 0) {
        for (int cp = 0; cp < 2; ++cp)
            for (int k = 0; k < nv; ++k) AT(x, nc, nv, cp, c, k) = base[cp * nv + k] / D[k];
    } else {
        cell_solve(s, c, nb, bf, D, base, xc);
        for (int cp = 0; cp < 2; ++cp)
            for (int k = 0; k < nv; ++k) AT(x, nc, nv, cp, c, k) = xc[cp * nv + k];
    }
}

/* One symmetric Gauss-Seidel pass (LU-SGS) on Eq. microFinalDefect:
 * forward  (D + L) x* = r, backward (D + U) x = D x*, lower = west/south
 * neighbours and ghosts, upper = east/north.  order 0 = lexicographic cell
 * order, order 1 = anti-diagonal wavefront order (the cells of a diagonal
 * depend only on the previous diagonal, so the arithmetic per cell is the
 * same; the OpenMP build sweeps in this order, the cells of a diagonal
 * spread over threads). */
static void sgs_micro(oracle_solver *s, const olev_t *Lv, const double *inv_tau, const double *r, double *x, int order)
{
    int nx = Lv->nx, ny = Lv->ny, nv = s->nv, nd = nx + ny - 1;
    if (s->nthr > 1) order = 1;
    for (int pass = 0; pass < 2; ++pass) {
        if (order == 0) {
            int ncell = nx * ny;
            for (int t = 0; t < ncell; ++t) {
                int tt = pass == 0 ? t : ncell - 1 - t;
                sweep_cell(s, Lv, inv_tau, r, x, pass, tt % nx, tt / nx, s->sD, s->sbase, s->sxc);
            }
            continue;
        }
        for (int d0 = 0; d0 < nd; ++d0) {
            int d = pass == 0 ? d0 : nd - 1 - d0;
            int ilo = d - (ny - 1) > 0 ? d - (ny - 1) : 0, ihi = d < nx - 1 ? d : nx - 1;
#pragma omp parallel for num_threads(s->nthr) schedule(static) if (ihi - ilo >= 2)
            for (int i = ilo; i <= ihi; ++i) {
                size_t t = (size_t)ORC_TID;
                sweep_cell(s, Lv, inv_tau, r, x, pass, i, d - i, s->sD + t * nv, s->sbase + t * 2 * nv,
                           s->sxc + t * 2 * nv);
            }
        }
    }
}

/* y = A x, the full evolution operator of Eq. microFinalDefect with every
 * neighbour and every boundary ghost (used to renew residuals, Eq. renewResidualMicro). */
static void apply_micro(const oracle_solver *s, const olev_t *Lv, const double *inv_tau, const double *x, double *y)
{
    int nx = Lv->nx, ny = Lv->ny, nv = s->nv;
    size_t nc = Lv->nc;
#pragma omp parallel for num_threads(s->nthr) schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int c = j * nx + i;
            if (Lv->solid[c]) {
                for (int cp = 0; cp < 2; ++cp)
                    for (int k = 0; k < nv; ++k) AT(y, nc, nv, cp, c, k) = 0.0;
                continue;
            }
            double V = Lv->dx[i] * Lv->dy[j];
            bface_t bf[4];
            int nb = cell_bfaces(Lv, i, j, 2, bf);
            double rho[4];
            for (int b = 0; b < nb; ++b) {
                if (s->bc[bf[b].bc].type != ORC_BC_WALL) continue;
                double num = 0.0, Z = 0.0;
                for (int k = 0; k < nv; ++k) {
                    double uo = bf[b].outsign * (bf[b].axis == 0 ? s->u[k] : s->v[k]);
                    if (uo > 0) num += s->w[k] * uo * AT(x, nc, nv, 0, c, k);
                    else if (uo < 0) Z += s->w[k] * uo * wallC(s, bf[b].bc, 0, k);
                }
                rho[b] = -num / Z;
            }
            for (int cp = 0; cp < 2; ++cp)
                for (int k = 0; k < nv; ++k) {
                    double acc = Dii(s, Lv, i, j, inv_tau[c], k) * AT(x, nc, nv, cp, c, k);
                    if (i > 0 && Lv->fbx[j * (nx + 1) + i] < 0)
                        acc += Dij(s, 0, -1, Lv->dy[j], V, k) * AT(x, nc, nv, cp, c - 1, k);
                    if (i < nx - 1 && Lv->fbx[j * (nx + 1) + i + 1] < 0)
                        acc += Dij(s, 0, +1, Lv->dy[j], V, k) * AT(x, nc, nv, cp, c + 1, k);
                    if (j > 0 && Lv->fby[j * nx + i] < 0)
                        acc += Dij(s, 1, -1, Lv->dx[i], V, k) * AT(x, nc, nv, cp, c - nx, k);
                    if (j < ny - 1 && Lv->fby[(j + 1) * nx + i] < 0)
                        acc += Dij(s, 1, +1, Lv->dx[i], V, k) * AT(x, nc, nv, cp, c + nx, k);
                    for (int b = 0; b < nb; ++b) {
                        double Db = Dij(s, bf[b].axis, bf[b].outsign, bf[b].S, bf[b].V, k);
                        if (Db == 0.0) continue;
                        int t = s->bc[bf[b].bc].type;
                        if (t == ORC_BC_WALL) acc += Db * wallC(s, bf[b].bc, cp, k) * rho[b];
                        else if (t == ORC_BC_SYMMETRY) {
                            int km = bf[b].axis == 0 ? s->mxk[k] : s->myk[k];
                            acc += Db * AT(x, nc, nv, cp, c, km);
                        } else if (t == ORC_BC_OUTFLOW) acc += Db * AT(x, nc, nv, cp, c, k);
                    }
                    AT(y, nc, nv, cp, c, k) = acc;
                }
        }
}

/* CS cycle (Eq. CSCYC): on entry lv->r holds the residual of level l (it is
 * renewed in place); on exit lv->df holds the total correction.  Cycle types
 * as for FAS: a second coarse visit (W: of type W, F: of type V) solves for the
 * coarse residual that the first visit's correction leaves, r_H - A_H df_H,
 * and the two corrections add. */
static void cs(oracle_solver *s, int l, int type)
{
    olev_t *Lv = &s->lev[l];
    size_t n = 2 * (size_t)Lv->nc * s->nv;
    memset(Lv->df, 0, n * sizeof(double));
    int coarsest = (l == s->L - 1);
    int npre = coarsest ? (s->L == 1 ? 1 : s->nuc) : s->nu1;
    for (int m = 0; m < npre; ++m) {
        sgs_micro(s, Lv, Lv->inv_tau, Lv->r, Lv->dl, 0);
#pragma omp parallel for schedule(static)
        for (size_t q = 0; q < n; ++q) Lv->df[q] += Lv->dl[q];
        if (coarsest && m == npre - 1) return;
        apply_micro(s, Lv, Lv->inv_tau, Lv->dl, Lv->Ad); /* Eq. renewResidualMicro */
#pragma omp parallel for schedule(static)
        for (size_t q = 0; q < n; ++q) Lv->r[q] -= Lv->Ad[q];
    }
    olev_t *Cv = &s->lev[l + 1];
    for (int cp = 0; cp < 2; ++cp)
        restrict_lv(Lv, Cv, s->nv, Lv->r + (size_t)cp * Lv->nc * s->nv, Cv->r + (size_t)cp * Cv->nc * s->nv);
    size_t nC = 2 * (size_t)Cv->nc * s->nv;
    double *r0 = type != 0 ? dalloc(nC) : NULL;
    if (r0) memcpy(r0, Cv->r, nC * sizeof(double));
    cs(s, l + 1, type);
    if (type == 3) {
        /* adaptive: another coarse visit, for the coarse residual the corrections so far
         * leave, while a visit leaves more than ADAPT_RATIO of the residual it started from */
        double *acc = dalloc(nC);
        double before = sumsq(r0, nC);
        memcpy(acc, Cv->df, nC * sizeof(double));
        for (int visit = 1; visit < ADAPT_MAX_VISITS; ++visit) {
            apply_micro(s, Cv, Cv->inv_tau, acc, Cv->Ad);
            for (size_t q = 0; q < nC; ++q) Cv->r[q] = r0[q] - Cv->Ad[q];
            double after = sumsq(Cv->r, nC);
            s->adapt_log[s->adapt_n++ % ADAPT_LOG] = after > s->adapt_ratio * s->adapt_ratio * before;
            if (!(after > s->adapt_ratio * s->adapt_ratio * before)) break;
            before = after;
            cs(s, l + 1, 3);
            for (size_t q = 0; q < nC; ++q) acc[q] += Cv->df[q];
        }
        memcpy(Cv->df, acc, nC * sizeof(double));
        free(acc);
        free(r0);
    } else if (type != 0) {
        double *acc = dalloc(nC);
        memcpy(acc, Cv->df, nC * sizeof(double));
        apply_micro(s, Cv, Cv->inv_tau, acc, Cv->Ad);
        for (size_t q = 0; q < nC; ++q) Cv->r[q] = r0[q] - Cv->Ad[q];
        cs(s, l + 1, type == 1 ? 1 : 0);
        for (size_t q = 0; q < nC; ++q) Cv->df[q] += acc[q];
        free(acc);
        free(r0);
    }
    for (int cp = 0; cp < 2; ++cp)
        prolong_lv(Lv, Cv, s->nv, Cv->df + (size_t)cp * Cv->nc * s->nv, Lv->dl + (size_t)cp * Lv->nc * s->nv);
#pragma omp parallel for schedule(static)
    for (size_t q = 0; q < n; ++q) Lv->df[q] += Lv->dl[q];
    for (int m = 0; m < s->nu2; ++m) {
        apply_micro(s, Lv, Lv->inv_tau, Lv->dl, Lv->Ad);
#pragma omp parallel for schedule(static)
        for (size_t q = 0; q < n; ++q) Lv->r[q] -= Lv->Ad[q];
        sgs_micro(s, Lv, Lv->inv_tau, Lv->r, Lv->dl, 0);
#pragma omp parallel for schedule(static)
        for (size_t q = 0; q < n; ++q) Lv->df[q] += Lv->dl[q];
    }
}

/* ------------------------------------------------------------------ */
/* Outer iteration (Steps 1-8)                                          */
/* ------------------------------------------------------------------ */

/* Step 7: W = sum_k w psi f and the heat flux q = sum_k w c (c^2 G/2 + H) */
static void moments(oracle_solver *s)
{
    int nv = s->nv;
    long nc = (long)s->lev[0].nc;
#pragma omp parallel for num_threads(s->nthr) schedule(static)
    for (long c = 0; c < nc; ++c) {
        double W[4] = {0, 0, 0, 0};
        for (int k = 0; k < nv; ++k) {
            double g = FIX(s, 0, c, k), h = FIX(s, 1, c, k);
            W[0] += s->w[k] * g;
            W[1] += s->w[k] * s->u[k] * g;
            W[2] += s->w[k] * s->v[k] * g;
            W[3] += s->w[k] * (0.5 * (s->u[k] * s->u[k] + s->v[k] * s->v[k]) * g + h);
        }
        double rho, U, V, lam, qx = 0.0, qy = 0.0;
        prim(W, &rho, &U, &V, &lam);
        for (int k = 0; k < nv; ++k) {
            double cx = s->u[k] - U, cy = s->v[k] - V, c2 = cx * cx + cy * cy;
            double e = 0.5 * c2 * FIX(s, 0, c, k) + FIX(s, 1, c, k);
            qx += s->w[k] * cx * e;
            qy += s->w[k] * cy * e;
        }
        for (int m = 0; m < 4; ++m) s->W[4 * c + m] = W[m];
        s->q[2 * c] = qx;
        s->q[2 * c + 1] = qy;
    }
}

/* RMS over the fluid cells (Eq. Residual_Def); R is zero in bodies */
static void rms(const oracle_solver *s, double res[4])
{
    size_t nc = s->lev[0].nc;
    for (int m = 0; m < 4; ++m) {
        double a = 0.0;
        for (size_t c = 0; c < nc; ++c) a += s->R[4 * c + m] * s->R[4 * c + m];
        res[m] = sqrt(a / s->lev[0].nfluid);
    }
}

static void one_iteration(oracle_solver *s, double res[4])
{
    olev_t *L0 = &s->lev[0];
    int nx = L0->nx, ny = L0->ny, nv = s->nv;
    size_t nc = L0->nc;
    /* Step 1 */
    flux_stage(s);
    rms(s, res);
    /* Step 2: predicted conservative variables by FAS */
    memcpy(L0->Wn, s->W, 4 * nc * sizeof(double));
    memcpy(L0->Rc, s->R, 4 * nc * sizeof(double));
    fas(s, 0, s->cycle);
    /* the predicted state; a cell where it has non-positive density or
     * internal energy keeps W^n (reading: the paper is silent) */
    for (size_t c = 0; c < nc; ++c) {
        const double *w = L0->Wc + 4 * c;
        double e2 = w[3] * w[0] - 0.5 * (w[1] * w[1] + w[2] * w[2]);
        const double *src = (w[0] > 0.0 && e2 > 0.0) ? w : L0->Wn + 4 * c;
        for (int m = 0; m < 4; ++m) L0->Wtil[4 * c + m] = src[m];
    }
    /* Step 3: predicted equilibrium and collision time; coarse tau from the
     * volume-restricted predicted state */
    double add = dtn_inv(s);
    for (int l = 0; l < s->L; ++l) {
        olev_t *Lv = &s->lev[l];
        if (l > 0) restrict_lv(&s->lev[l - 1], Lv, 4, s->lev[l - 1].Wtil, Lv->Wtil);
        for (int c = 0; c < Lv->nc; ++c) {
            double rho, U, V, lam;
            prim(Lv->Wtil + 4 * c, &rho, &U, &V, &lam);
            Lv->inv_tau[c] = 1.0 / tau_of(s, rho, lam) + add;
        }
    }
    /* Step 4: r = (g~ - f)/tau~ - (1/V) sum S u_n f~ (Eq. microResidualDef) */
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int c = j * nx + i;
            if (L0->solid[c]) {
                for (int cp = 0; cp < 2; ++cp)
                    for (int k = 0; k < nv; ++k) AT(L0->r, nc, nv, cp, c, k) = 0.0;
                continue;
            }
            double rho, U, V, lam;
            prim(L0->Wtil + 4 * c, &rho, &U, &V, &lam);
            double itau = 1.0 / tau_of(s, rho, lam);
            double Vol = L0->dx[i] * L0->dy[j];
            double qx = s->q[2 * c], qy = s->q[2 * c + 1];
            int fW = j * (nx + 1) + i, fE = fW + 1, fS = j * nx + i, fN = (j + 1) * nx + i;
            for (int k = 0; k < nv; ++k) {
                double gt[2];
                shakhov(rho, U, V, lam, qx, qy, s->pr, s->u[k], s->v[k], &gt[0], &gt[1]);
                for (int cp = 0; cp < 2; ++cp) {
                    const double *px = s->phx + (size_t)cp * L0->nfx * nv, *py = s->phy + (size_t)cp * L0->nfy * nv;
                    double div = (L0->dy[j] * (px[(size_t)fE * nv + k] - px[(size_t)fW * nv + k]) +
                                  L0->dx[i] * (py[(size_t)fN * nv + k] - py[(size_t)fS * nv + k])) / Vol;
                    AT(L0->r, nc, nv, cp, c, k) = (gt[cp] - FIX(s, cp, c, k)) * itau - div;
                }
            }
        }
    /* Step 5: total correction by the CS cycle */
    cs(s, 0, s->cycle);
    /* Steps 6-7: f += df, except in a cell where f + df has non-positive
     * density or internal energy, which keeps f (reading: the paper is silent) */
#pragma omp parallel for num_threads(s->nthr) schedule(static)
    for (size_t c = 0; c < nc; ++c) {
        double W[4] = {0, 0, 0, 0};
        for (int k = 0; k < nv; ++k) {
            double g = FIX(s, 0, c, k) + AT(L0->df, nc, nv, 0, c, k);
            double h = FIX(s, 1, c, k) + AT(L0->df, nc, nv, 1, c, k);
            W[0] += s->w[k] * g;
            W[1] += s->w[k] * s->u[k] * g;
            W[2] += s->w[k] * s->v[k] * g;
            W[3] += s->w[k] * (0.5 * (s->u[k] * s->u[k] + s->v[k] * s->v[k]) * g + h);
        }
        if (W[0] > 0.0 && W[3] * W[0] - 0.5 * (W[1] * W[1] + W[2] * W[2]) > 0.0)
            for (int cp = 0; cp < 2; ++cp)
                for (int k = 0; k < nv; ++k) FIX(s, cp, c, k) += AT(L0->df, nc, nv, cp, c, k);
    }
    moments(s);
    s->iter++;
}

/* ------------------------------------------------------------------ */
/* Public API                                                           */
/* ------------------------------------------------------------------ */

oracle_solver *oracle_create(int nx, int ny, const double *xn, const double *yn,
                             const int *face_bc_x, const int *face_bc_y, const unsigned char *solid,
                             int nbc, const int *bc_type, const double *bc_vals,
                             int nu, int nv, double umin, double umax,
                             double vmin, double vmax, int rule,
                             double kn, double omega, double pr,
                             int levels, int nu1, int nu2, int nuc,
                             double cfl, double dtn_growth)
{
    if (nx < 1 || ny < 1 || levels < 1 || levels > MAXL || nbc < 1 || nu < 2 || nv < 2) {
        fail("bad sizes");
        return NULL;
    }
    oracle_solver *s = (oracle_solver *)calloc(1, sizeof *s);
    s->L = levels;
    s->nu = nu; s->nvv = nv; s->nv = nu * nv;
    s->kn = kn; s->omega = omega; s->pr = pr; s->mu_ref = oracle_mu_ref(kn, omega);
    s->nu1 = nu1; s->nu2 = nu2; s->nuc = nuc; s->cfl = cfl; s->dtn_growth = dtn_growth;
    s->adapt_ratio = ADAPT_RATIO;
    double *ux = dalloc(nu), *wu = dalloc(nu), *vy = dalloc(nv), *wv = dalloc(nv);
    if (oracle_vgrid(nu, umin, umax, rule, ux, wu) || oracle_vgrid(nv, vmin, vmax, rule, vy, wv)) {
        free(ux); free(wu); free(vy); free(wv); free(s);
        return NULL;
    }
    int NV = s->nv;
    s->u = dalloc(NV); s->v = dalloc(NV); s->w = dalloc(NV);
    s->mxk = (int *)calloc(NV, sizeof(int)); s->myk = (int *)calloc(NV, sizeof(int));
    int symu = (umin == -umax), symv = (vmin == -vmax);
    for (int a = 0; a < nu; ++a)
        for (int b = 0; b < nv; ++b) {
            int k = a * nv + b;
            s->u[k] = ux[a]; s->v[k] = vy[b]; s->w[k] = wu[a] * wv[b];
            s->mxk[k] = symu ? (nu - 1 - a) * nv + b : -1;
            s->myk[k] = symv ? a * nv + (nv - 1 - b) : -1;
        }
    s->umax_abs = fmax(fabs(umin), fabs(umax));
    s->vmax_abs = fmax(fabs(vmin), fabs(vmax));
    free(ux); free(wu); free(vy); free(wv);
    s->nbc = nbc;
    s->bc = (obc_t *)calloc(nbc, sizeof(obc_t));
    s->Cw = dalloc((size_t)nbc * NV);
    for (int b = 0; b < nbc; ++b) {
        s->bc[b] = (obc_t){bc_type[b], bc_vals[4 * b], bc_vals[4 * b + 1], bc_vals[4 * b + 2], bc_vals[4 * b + 3]};
        if (bc_type[b] < 0 || bc_type[b] > 3 || !(bc_vals[4 * b + 3] > 0)) {
            fail("bad BC %d", b);
            oracle_destroy(s);
            return NULL;
        }
        if (bc_type[b] == ORC_BC_SYMMETRY && (!symu || !symv)) {
            fail("symmetry BC needs a velocity grid symmetric about zero");
            oracle_destroy(s);
            return NULL;
        }
        for (int k = 0; k < NV; ++k)
            s->Cw[(size_t)b * NV + k] = maxw(1.0, s->bc[b].u, s->bc[b].v, 1.0 / s->bc[b].t, s->u[k], s->v[k]);
    }
    olev_t *L0 = &s->lev[0];
    L0->nx = nx; L0->ny = ny; L0->nc = nx * ny; L0->nfx = (nx + 1) * ny; L0->nfy = nx * (ny + 1);
    L0->xn = dalloc(nx + 1); L0->yn = dalloc(ny + 1);
    memcpy(L0->xn, xn, (nx + 1) * sizeof(double));
    memcpy(L0->yn, yn, (ny + 1) * sizeof(double));
    L0->fbx = (int *)malloc(L0->nfx * sizeof(int));
    L0->fby = (int *)malloc(L0->nfy * sizeof(int));
    memcpy(L0->fbx, face_bc_x, L0->nfx * sizeof(int));
    memcpy(L0->fby, face_bc_y, L0->nfy * sizeof(int));
    L0->solid = (unsigned char *)calloc(L0->nc, 1);
    if (solid)
        for (int c = 0; c < L0->nc; ++c) L0->solid[c] = solid[c] != 0;
    L0->nfluid = 0;
    for (int c = 0; c < L0->nc; ++c) L0->nfluid += !L0->solid[c];
    if (L0->nfluid == 0) { fail("no fluid cell"); oracle_destroy(s); return NULL; }
    /* A face between two fluid cells is interior (id -1); a face between a
     * fluid cell and a body or the domain edge needs a BC id; a face with no
     * fluid cell on either side is inactive (set to -1). */
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i <= nx; ++i) {
            int *b = &L0->fbx[j * (nx + 1) + i];
            int fl = i > 0 && !L0->solid[j * nx + i - 1], fr = i < nx && !L0->solid[j * nx + i];
            if (!fl && !fr) { *b = -1; continue; }
            if ((fl && fr) ? (*b != -1) : (*b < 0 || *b >= nbc)) {
                fail("x-face (%d,%d): boundary faces need a BC id, interior faces -1", i, j);
                oracle_destroy(s);
                return NULL;
            }
        }
    for (int j = 0; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int *b = &L0->fby[j * nx + i];
            int fl = j > 0 && !L0->solid[(j - 1) * nx + i], fr = j < ny && !L0->solid[j * nx + i];
            if (!fl && !fr) { *b = -1; continue; }
            if ((fl && fr) ? (*b != -1) : (*b < 0 || *b >= nbc)) {
                fail("y-face (%d,%d): boundary faces need a BC id, interior faces -1", i, j);
                oracle_destroy(s);
                return NULL;
            }
        }
    if (level_geom(L0)) { oracle_destroy(s); return NULL; }
    for (int l = 1; l < levels; ++l)
        if (coarsen(&s->lev[l - 1], &s->lev[l])) { oracle_destroy(s); return NULL; }
    for (int l = 0; l < levels; ++l)
        if (level_alloc(s, &s->lev[l])) { oracle_destroy(s); return NULL; }
    size_t nc = L0->nc;
    s->f = dalloc(2 * nc * NV); s->W = dalloc(4 * nc); s->q = dalloc(2 * nc); s->R = dalloc(4 * nc);
    s->phx = dalloc(2 * (size_t)L0->nfx * NV); s->phy = dalloc(2 * (size_t)L0->nfy * NV);
    s->Fx = dalloc(4 * (size_t)L0->nfx); s->Fy = dalloc(4 * (size_t)L0->nfy);
    s->nthr = ORC_MAXTHR;
    {
        size_t per = 2 * (size_t)NV * s->nthr;
        s->tmp0 = dalloc(per); s->tmp1 = dalloc(per); s->tmp2 = dalloc(per);
        s->sD = dalloc((size_t)NV * s->nthr); s->sbase = dalloc(per); s->sxc = dalloc(per);
    }
    if (!s->f || !s->phx || !s->phy) { fail("out of memory"); oracle_destroy(s); return NULL; }
    /* minimum physical time step over the interior faces (for dt_n) */
    s->dtp_min = 1e300;
    for (int i = 1; i < nx; ++i) s->dtp_min = fmin(s->dtp_min, face_dt(s, 0, L0->dx[i - 1], L0->dx[i]));
    for (int j = 1; j < ny; ++j) s->dtp_min = fmin(s->dtp_min, face_dt(s, 1, L0->dy[j - 1], L0->dy[j]));
    return s;
}

void oracle_destroy(oracle_solver *s)
{
    if (!s) return;
    for (int l = 0; l < MAXL; ++l) {
        olev_t *Lv = &s->lev[l];
        free(Lv->xn); free(Lv->yn); free(Lv->xc); free(Lv->yc); free(Lv->dx); free(Lv->dy);
        free(Lv->fbx); free(Lv->fby); free(Lv->solid);
        free(Lv->Wn); free(Lv->Wc); free(Lv->Rc); free(Lv->P); free(Lv->RE); free(Lv->dW); free(Lv->Wtil);
        free(Lv->r); free(Lv->df); free(Lv->dl); free(Lv->Ad); free(Lv->inv_tau);
    }
    free(s->u); free(s->v); free(s->w); free(s->mxk); free(s->myk); free(s->bc); free(s->Cw);
    free(s->f); free(s->W); free(s->q); free(s->R); free(s->phx); free(s->phy); free(s->Fx); free(s->Fy);
    free(s->tmp0); free(s->tmp1); free(s->tmp2);
    free(s->sD); free(s->sbase); free(s->sxc);
    free(s);
}

int oracle_init_fields(oracle_solver *s, const double *rho, const double *u, const double *v, const double *t)
{
    size_t nc = s->lev[0].nc;
    for (size_t c = 0; c < nc; ++c) {
        if (!(rho[c] > 0) || !(t[c] > 0)) return fail("init: rho and T must be positive");
        double lam = 1.0 / t[c];
        for (int k = 0; k < s->nv; ++k) {
            double g = maxw(rho[c], u[c], v[c], lam, s->u[k], s->v[k]);
            FIX(s, 0, c, k) = g;
            FIX(s, 1, c, k) = g * KINT / (4.0 * lam);
        }
    }
    moments(s);
    s->iter = 0;
    return 0;
}

int oracle_init_uniform(oracle_solver *s, double rho, double u, double v, double t)
{
    size_t nc = s->lev[0].nc;
    double *a = dalloc(4 * nc);
    for (size_t c = 0; c < nc; ++c) { a[c] = rho; a[nc + c] = u; a[2 * nc + c] = v; a[3 * nc + c] = t; }
    int st = oracle_init_fields(s, a, a + nc, a + 2 * nc, a + 3 * nc);
    free(a);
    return st;
}

int oracle_step(oracle_solver *s, int n, double res[4])
{
    double r[4] = {0, 0, 0, 0};
    for (int it = 0; it < n; ++it) {
        one_iteration(s, r);
        for (size_t c = 0; c < (size_t)s->lev[0].nc; ++c) {
            const double *W = s->W + 4 * c;
            double eint = W[3] - 0.5 * (W[1] * W[1] + W[2] * W[2]) / W[0];
            if (!(W[0] > 0) || !(eint > 0)) return fail("diverged at iteration %d", s->iter);
        }
    }
    if (res) memcpy(res, r, sizeof r);
    return 0;
}

int oracle_residual(oracle_solver *s, double *R)
{
    flux_stage(s);
    memcpy(R, s->R, 4 * (size_t)s->lev[0].nc * sizeof(double));
    return 0;
}

int oracle_get_macro(const oracle_solver *s, double *rho, double *u, double *v, double *t, double *qx, double *qy)
{
    for (int c = 0; c < s->lev[0].nc; ++c) {
        double r, U, V, lam;
        prim(s->W + 4 * c, &r, &U, &V, &lam);
        if (rho) rho[c] = r;
        if (u) u[c] = U;
        if (v) v[c] = V;
        if (t) t[c] = 1.0 / lam;
        if (qx) qx[c] = s->q[2 * c];
        if (qy) qy[c] = s->q[2 * c + 1];
    }
    return 0;
}

int oracle_get_f(const oracle_solver *s, double *f)
{
    memcpy(f, s->f, 2 * (size_t)s->lev[0].nc * s->nv * sizeof(double));
    return 0;
}

int oracle_set_f(oracle_solver *s, const double *f)
{
    memcpy(s->f, f, 2 * (size_t)s->lev[0].nc * s->nv * sizeof(double));
    moments(s);
    return 0;
}

int oracle_set_bc(oracle_solver *s, int b, double rho, double u, double v, double t)
{
    if (b < 0 || b >= s->nbc || !(t > 0)) return fail("set_bc: bad arguments");
    s->bc[b].rho = rho; s->bc[b].u = u; s->bc[b].v = v; s->bc[b].t = t;
    for (int k = 0; k < s->nv; ++k) s->Cw[(size_t)b * s->nv + k] = maxw(1.0, u, v, 1.0 / t, s->u[k], s->v[k]);
    return 0;
}

/* Wall pressure, shear stress and heat flux (Secs. 4.2, 4.3): momentum and
 * energy carried into the wall per unit area and time by the face
 * distribution, in the frame of the wall; normal n points from the gas into
 * the wall, the tangent is the other axis. */
int oracle_get_wall(const oracle_solver *s, int bc, int *nf, double *p, double *tau, double *q)
{
    const olev_t *L0 = &s->lev[0];
    int nx = L0->nx, ny = L0->ny, nv = s->nv, cnt = 0, cap = *nf;
    if (bc < 0 || bc >= s->nbc) return fail("get_wall: bad BC id");
    double *fG = dalloc(nv), *fH = dalloc(nv);
    const obc_t *B = &s->bc[bc];
    for (int pass = 0; pass < 2; ++pass) {
        int nfc = pass == 0 ? L0->nfx : L0->nfy;
        for (int fi = 0; fi < nfc; ++fi) {
            int b = pass == 0 ? L0->fbx[fi] : L0->fby[fi];
            if (b != bc) continue;
            int axis = pass, outsign, c;
            if (axis == 0) face_side(L0, 0, fi % (nx + 1), fi / (nx + 1), &c, &outsign);
            else face_side(L0, 1, fi % nx, fi / nx, &c, &outsign);
            boundary_face_f(s, bc, axis, outsign, c, fG, fH);
            double P = 0, T = 0, Q = 0, Uwt = axis == 0 ? B->v : B->u;
            for (int k = 0; k < nv; ++k) {
                double uo = outsign * (axis == 0 ? s->u[k] : s->v[k]);
                double ut = axis == 0 ? s->v[k] : s->u[k];
                double du = s->u[k] - B->u, dv = s->v[k] - B->v;
                P += s->w[k] * uo * uo * fG[k];
                T += s->w[k] * uo * (ut - Uwt) * fG[k];
                Q += s->w[k] * uo * (0.5 * (du * du + dv * dv) * fG[k] + fH[k]);
            }
            if (cnt < cap) { p[cnt] = P; tau[cnt] = T; q[cnt] = Q; }
            cnt++;
        }
    }
    free(fG); free(fH);
    *nf = cnt;
    return cnt > cap ? fail("get_wall: capacity %d < %d faces", cap, cnt) : 0;
}

int oracle_iterations(const oracle_solver *s) { return s->iter; }
int oracle_nv(const oracle_solver *s) { return s->nv; }
int oracle_level_size(const oracle_solver *s, int lev, int *nx, int *ny)
{
    if (lev < 0 || lev >= s->L) return fail("bad level");
    *nx = s->lev[lev].nx; *ny = s->lev[lev].ny;
    return 0;
}

int oracle_stage_flux(oracle_solver *s, double *R, double *phx, double *phy)
{
    flux_stage(s);
    const olev_t *L0 = &s->lev[0];
    if (R) memcpy(R, s->R, 4 * (size_t)L0->nc * sizeof(double));
    if (phx) memcpy(phx, s->phx, 2 * (size_t)L0->nfx * s->nv * sizeof(double));
    if (phy) memcpy(phy, s->phy, 2 * (size_t)L0->nfy * s->nv * sizeof(double));
    return 0;
}

int oracle_stage_sgs_micro(oracle_solver *s, int lev, const double *inv_tau, const double *r, double *x, int order)
{
    if (lev < 0 || lev >= s->L) return fail("bad level");
    sgs_micro(s, &s->lev[lev], inv_tau, r, x, order);
    return 0;
}

int oracle_stage_apply_micro(oracle_solver *s, int lev, const double *inv_tau, const double *x, double *y)
{
    if (lev < 0 || lev >= s->L) return fail("bad level");
    apply_micro(s, &s->lev[lev], inv_tau, x, y);
    return 0;
}

int oracle_stage_sgs_macro(oracle_solver *s, int lev, const double *W, const double *Wg, const double *R, double *dW, int order)
{
    if (lev < 0 || lev >= s->L) return fail("bad level");
    sgs_macro(s, &s->lev[lev], W, Wg, R, dW, order);
    return 0;
}

int oracle_stage_resid_macro(oracle_solver *s, int lev, const double *W, const double *Wg, double *RE)
{
    if (lev < 0 || lev >= s->L) return fail("bad level");
    resid_macro(s, &s->lev[lev], W, Wg, RE);
    return 0;
}

int oracle_stage_restrict(oracle_solver *s, int lev, int m, const double *fine, double *coarse)
{
    if (lev < 0 || lev + 1 >= s->L) return fail("bad level");
    restrict_lv(&s->lev[lev], &s->lev[lev + 1], m, fine, coarse);
    return 0;
}

int oracle_stage_prolong(oracle_solver *s, int lev, int m, const double *coarse, double *fine)
{
    if (lev < 0 || lev + 1 >= s->L) return fail("bad level");
    prolong_lv(&s->lev[lev], &s->lev[lev + 1], m, coarse, fine);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Steady equations and their adjoint.                                  */
/*                                                                      */
/* At convergence the outer iteration has Delta f = 0, which with the   */
/* predicted state equal to the moments of f is the discrete steady     */
/* equation N(f; theta) = 0 of Eq. microResidualDef:                    */
/*   N_i,k = (g+_k(W_i, q_i) - f_i,k)/tau(W_i)                          */
/*           - (1/V_i) sum_j S_ij Phi_ij,k / dt_p,                      */
/* with W_i, q_i the moments of f_i and Phi the UGKS flux of Step 1.    */
/* theta (a wall temperature or velocity) enters only through the       */
/* diffuse wall (Sec. 3.2).  For an objective J(f; theta) the adjoint   */
/* state solves (dN/df)^T lambda = -(dJ/df)^T and                       */
/*   dJ/dtheta = dJ/dtheta|_f + lambda . dN/dtheta|_f.                   */
/* The functions below are hand-written reverse-mode derivatives of     */
/* the forward functions of this file, in the same order of operations. */
/* ------------------------------------------------------------------ */

/* d q_m / d tau of the five time integrals.  Closed form from
 * d e/d tau = e x / tau; for x < 1 the series of oracle_time_coeffs
 * differentiated term by term: q_m = dt^p s_m(x) gives
 * dq_m/dtau = -(dt^p / tau) sum_n n c_mn x^n. */
void oracle_time_coeffs_dtau(double dt, double tau, double dq[5])
{
    double x = dt / tau;
    if (x < 1.0) {
        double p[28];
        p[0] = 1.0;
        for (int n = 1; n < 28; ++n) p[n] = p[n - 1] * x / n; /* x^n / n! */
        double s1 = 0, s2 = 0, s3 = 0, s4 = 0, s5 = 0;
        for (int n = 1; n < 26; ++n) {
            double sg = (n % 2) ? -1.0 : 1.0;                          /* (-1)^n */
            s4 += n * sg * p[n] / (n + 1);                             /* n (-1)^n x^n/(n+1)! */
            s1 += n * -sg * p[n] / (n + 1);                            /* n (-1)^{n+1} x^n/(n+1)! */
            s3 += n * -sg * p[n] / ((double)(n + 1) * (n + 2));        /* n (-1)^{n+1} x^n/(n+2)! */
            s2 += n * sg * n * p[n] / ((double)(n + 1) * (n + 2));     /* n (-1)^n n x^n/(n+2)! */
            s5 += n * -sg * (n + 1) * p[n] / ((double)(n + 1) * (n + 2)); /* n (-1)^{n+1}(n+1) x^n/(n+2)! */
        }
        dq[0] = -dt / tau * s1;
        dq[1] = -dt * dt / tau * s2;
        dq[2] = -dt * dt / tau * s3;
        dq[3] = -dt / tau * s4;
        dq[4] = -dt * dt / tau * s5;
    } else {
        double e = exp(-x), E1 = -expm1(-x);
        dq[0] = -E1 + x * e;
        dq[1] = -dt * (1.0 + e) - dt * x * e + 4.0 * tau * E1 - 2.0 * tau * x * e;
        dq[2] = -dt + 2.0 * tau * E1 - tau * x * e;
        dq[3] = E1 - x * e;
        dq[4] = dt * e + dt * x * e - 2.0 * tau * E1 + tau * x * e;
    }
}

/* Reverse of oracle_micro_slope: given abar = dL/da, accumulate dL/d(dw)
 * into dwb and dL/d(U, V, lam) into pb[0..2]. */
void oracle_micro_slope_adj(const double dw[4], double U, double V, double lam, const double abar[4],
                            double dwb[4], double pb[3])
{
    double Kp2 = KINT + 2.0;
    double cc = U * U + V * V + Kp2 / (2.0 * lam);
    double R4 = 2.0 * dw[3] - cc * dw[0];
    double R3 = dw[2] - V * dw[0];
    double R2 = dw[1] - U * dw[0];
    double X = R4 - 2.0 * U * R2 - 2.0 * V * R3;
    double a3 = 4.0 * lam * lam / Kp2 * X;
    double a2 = 2.0 * lam * R3 - V * a3;
    double a1 = 2.0 * lam * R2 - U * a3;
    double ab[4] = {abar[0], abar[1], abar[2], abar[3]};
    double Ub = 0, Vb = 0, lb = 0, ccb = 0, R2b = 0, R3b = 0, R4b = 0;
    /* a0 = dw0 - U a1 - V a2 - a3 cc / 2 */
    dwb[0] += ab[0];
    Ub -= ab[0] * a1; ab[1] -= ab[0] * U;
    Vb -= ab[0] * a2; ab[2] -= ab[0] * V;
    ab[3] -= ab[0] * 0.5 * cc; ccb -= ab[0] * 0.5 * a3;
    /* a1 = 2 lam R2 - U a3 */
    lb += ab[1] * 2.0 * R2; R2b += ab[1] * 2.0 * lam; Ub -= ab[1] * a3; ab[3] -= ab[1] * U;
    /* a2 = 2 lam R3 - V a3 */
    lb += ab[2] * 2.0 * R3; R3b += ab[2] * 2.0 * lam; Vb -= ab[2] * a3; ab[3] -= ab[2] * V;
    /* a3 = 4 lam^2 X / Kp2 */
    double Xb = ab[3] * 4.0 * lam * lam / Kp2;
    lb += ab[3] * 8.0 * lam / Kp2 * X;
    R4b += Xb; Ub -= Xb * 2.0 * R2; R2b -= Xb * 2.0 * U; Vb -= Xb * 2.0 * R3; R3b -= Xb * 2.0 * V;
    /* R2, R3, R4 */
    dwb[1] += R2b; Ub -= R2b * dw[0]; dwb[0] -= R2b * U;
    dwb[2] += R3b; Vb -= R3b * dw[0]; dwb[0] -= R3b * V;
    dwb[3] += 2.0 * R4b; ccb -= R4b * dw[0]; dwb[0] -= R4b * cc;
    /* cc */
    Ub += 2.0 * U * ccb; Vb += 2.0 * V * ccb; lb -= ccb * Kp2 / (2.0 * lam * lam);
    pb[0] += Ub; pb[1] += Vb; pb[2] += lb;
}

/* Reverse of slope_moments: (mGb, mHb) -> a, gM, hM and xi4q adjoints. */
static void slope_moments_adj(const double a[4], double u, double v, double gM, double hM, double xi4q,
                              double mGb, double mHb, double ab[4], double *gMb, double *hMb, double *xib)
{
    double b = a[0] + a[1] * u + a[2] * v + 0.5 * a[3] * (u * u + v * v);
    double bb = mGb * gM + mHb * hM;
    ab[0] += bb; ab[1] += bb * u; ab[2] += bb * v;
    ab[3] += bb * 0.5 * (u * u + v * v) + mGb * hM + mHb * xi4q * gM;
    *gMb += mGb * b + mHb * a[3] * xi4q;
    *hMb += mGb * a[3] + mHb * b;
    *xib += mHb * a[3] * gM;
}

/* Reverse of prim(): (rho, U, V, lam) adjoints -> W adjoint (accumulated). */
static void prim_adj(const double *W, double rb, double Ub, double Vb, double lb, double *Wb)
{
    double rho, U, V, lam;
    prim(W, &rho, &U, &V, &lam);
    double eint = W[3] - 0.5 * (W[1] * W[1] + W[2] * W[2]) / W[0];
    double eb = -lb * lam / eint;
    Wb[0] += rb + lb * lam / rho + eb * 0.5 * (U * U + V * V) - (Ub * U + Vb * V) / rho;
    Wb[1] += Ub / rho - eb * U;
    Wb[2] += Vb / rho - eb * V;
    Wb[3] += eb;
}

/* Reverse of a Maxwellian pair gM = rho (lam/pi) e^{-lam c^2}, hM = gM K/(4 lam)
 * at peculiar velocity (cx, cy): accumulates rho, U, V, lam adjoints. */
static void maxw_adj(double gM, double hM, double rho, double lam, double cx, double cy,
                     double gMb, double hMb, double *rb, double *Ub, double *Vb, double *lb)
{
    double c2 = cx * cx + cy * cy;
    gMb += hMb * KINT / (4.0 * lam);
    *lb -= hMb * hM / lam;
    *rb += gMb * gM / rho;
    *lb += gMb * gM * (1.0 / lam - c2);
    double c2b = -gMb * gM * lam;
    *Ub -= 2.0 * cx * c2b;
    *Vb -= 2.0 * cy * c2b;
}

#define OUTA(out, comp, c, k) ((out)[((size_t)(comp) * nc + (c)) * nv + (k)])

/* Adjoint of interior_face: nuG, nuH = dL/d(Phi_k / dt) per velocity; the
 * adjoint with respect to f of the four cells of the stencil is added to out. */
static void interior_face_adj(oracle_solver *s, int axis, int cLL, int cL, int cR, int cRR,
                              double dLLL, double dLR, double dRRR, double hL, double hR,
                              double wL, double wR, const double *nuG, const double *nuH, double *out)
{
    int nv = s->nv;
    size_t nc = s->lev[0].nc;
    const double *u = s->u, *v = s->v, *w = s->w;
    double *f0 = dalloc(2 * (size_t)nv), *sg = dalloc(2 * (size_t)nv);
    double *f0b = dalloc(2 * (size_t)nv), *sgb = dalloc(2 * (size_t)nv);
    /* ---- forward, as interior_face ---- */
    for (int k = 0; k < nv; ++k) {
        double un = axis == 0 ? u[k] : v[k];
        for (int cp = 0; cp < 2; ++cp) {
            double fL = FIX(s, cp, cL, k), fR = FIX(s, cp, cR, k);
            double sL = 0.0, sR = 0.0;
            if (cLL >= 0) sL = oracle_vanleer((fL - FIX(s, cp, cLL, k)) / dLLL, (fR - fL) / dLR);
            if (cRR >= 0) sR = oracle_vanleer((fR - fL) / dLR, (FIX(s, cp, cRR, k) - fR) / dRRR);
            double faceL = fL + sL * hL, faceR = fR - sR * hR;
            if (un > 0) { f0[cp * nv + k] = faceL; sg[cp * nv + k] = sL; }
            else if (un < 0) { f0[cp * nv + k] = faceR; sg[cp * nv + k] = sR; }
            else { f0[cp * nv + k] = 0.5 * (faceL + faceR); sg[cp * nv + k] = 0.5 * (sL + sR); }
        }
    }
    double W0[4] = {0, 0, 0, 0};
    for (int k = 0; k < nv; ++k) {
        double g = f0[k], h = f0[nv + k];
        W0[0] += w[k] * g;
        W0[1] += w[k] * u[k] * g;
        W0[2] += w[k] * v[k] * g;
        W0[3] += w[k] * (0.5 * (u[k] * u[k] + v[k] * v[k]) * g + h);
    }
    double rho0, U0, V0, lam0;
    prim(W0, &rho0, &U0, &V0, &lam0);
    double tau0 = tau_of(s, rho0, lam0);
    double dt = face_dt(s, axis, wL, wR);
    const double *WL = s->W + 4 * cL, *WR = s->W + 4 * cR;
    double dwl[4], dwr[4], aL[4], aR[4];
    for (int m = 0; m < 4; ++m) {
        dwl[m] = (W0[m] - WL[m]) / hL / rho0;
        dwr[m] = (WR[m] - W0[m]) / hR / rho0;
    }
    oracle_micro_slope(dwl, U0, V0, lam0, aL);
    oracle_micro_slope(dwr, U0, V0, lam0, aR);
    double xi4q = KINT * (KINT + 2.0) / (16.0 * lam0 * lam0);
    double q0[2] = {0, 0}, Mt[4] = {0, 0, 0, 0};
    for (int k = 0; k < nv; ++k) {
        double cx = u[k] - U0, cy = v[k] - V0, c2 = cx * cx + cy * cy;
        double g = f0[k], h = f0[nv + k];
        q0[0] += w[k] * cx * (0.5 * c2 * g + h);
        q0[1] += w[k] * cy * (0.5 * c2 * g + h);
        double un = axis == 0 ? u[k] : v[k];
        if (un == 0.0) continue;
        double gM = maxw(rho0, U0, V0, lam0, u[k], v[k]), hM = gM * KINT / (4.0 * lam0);
        double mG, mH;
        slope_moments(un > 0 ? aL : aR, u[k], v[k], gM, hM, lam0, &mG, &mH);
        Mt[0] += w[k] * un * mG;
        Mt[1] += w[k] * un * u[k] * mG;
        Mt[2] += w[k] * un * v[k] * mG;
        Mt[3] += w[k] * un * (0.5 * (u[k] * u[k] + v[k] * v[k]) * mG + mH);
    }
    double dwt[4], A[4];
    for (int m = 0; m < 4; ++m) dwt[m] = -Mt[m] / rho0;
    oracle_micro_slope(dwt, U0, V0, lam0, A);
    double qc[5], dqc[5];
    oracle_time_coeffs(dt, tau0, qc);
    oracle_time_coeffs_dtau(dt, tau0, dqc);
    double shk = (1.0 - s->pr) * 4.0 * lam0 * lam0 / (5.0 * rho0);

    /* ---- reverse of the flux assembly (last loop of interior_face) ---- */
    double qcb[5] = {0, 0, 0, 0, 0}, aLb[4] = {0, 0, 0, 0}, aRb[4] = {0, 0, 0, 0}, Ab[4] = {0, 0, 0, 0};
    double rb = 0, Ub = 0, Vb = 0, lb = 0, shkb = 0, xib = 0, q0b[2] = {0, 0};
    for (int k = 0; k < nv; ++k) {
        double un = axis == 0 ? u[k] : v[k];
        if (un == 0.0) continue; /* Phi_k = 0 identically */
        double cx = u[k] - U0, cy = v[k] - V0, c2 = cx * cx + cy * cy;
        double gM = maxw(rho0, U0, V0, lam0, u[k], v[k]), hM = gM * KINT / (4.0 * lam0);
        double Fq = shk * (cx * q0[0] + cy * q0[1]);
        double eG = 2.0 * lam0 * c2 - 4.0, eH = 2.0 * lam0 * c2 - 2.0;
        double gP = gM * (1.0 + Fq * eG), hP = hM * (1.0 + Fq * eH);
        const double *as = un > 0 ? aL : aR;
        double *asb = un > 0 ? aLb : aRb;
        double mGa, mHa, mGA, mHA;
        slope_moments(as, u[k], v[k], gM, hM, lam0, &mGa, &mHa);
        slope_moments(A, u[k], v[k], gM, hM, lam0, &mGA, &mHA);
        double PbG = nuG[k] / dt, PbH = nuH[k] / dt;
        qcb[0] += un * (PbG * gP + PbH * hP);
        qcb[1] += un * un * (PbG * mGa + PbH * mHa);
        qcb[2] += un * (PbG * mGA + PbH * mHA);
        qcb[3] += un * (PbG * f0[k] + PbH * f0[nv + k]);
        qcb[4] += un * un * (PbG * sg[k] + PbH * sg[nv + k]);
        f0b[k] += un * qc[3] * PbG;
        f0b[nv + k] += un * qc[3] * PbH;
        sgb[k] += un * un * qc[4] * PbG;
        sgb[nv + k] += un * un * qc[4] * PbH;
        double gPb = un * qc[0] * PbG, hPb = un * qc[0] * PbH;
        double gMb = 0, hMb = 0;
        slope_moments_adj(as, u[k], v[k], gM, hM, xi4q, un * un * qc[1] * PbG, un * un * qc[1] * PbH,
                          asb, &gMb, &hMb, &xib);
        slope_moments_adj(A, u[k], v[k], gM, hM, xi4q, un * qc[2] * PbG, un * qc[2] * PbH, Ab, &gMb, &hMb, &xib);
        /* Shakhov factors */
        gMb += gPb * (1.0 + Fq * eG);
        hMb += hPb * (1.0 + Fq * eH);
        double Fqb = gPb * gM * eG + hPb * hM * eH;
        double eb = (gPb * gM + hPb * hM) * Fq;          /* both e's carry 2 lam c^2 */
        lb += eb * 2.0 * c2;
        double c2b = eb * 2.0 * lam0;
        shkb += Fqb * (cx * q0[0] + cy * q0[1]);
        q0b[0] += Fqb * shk * cx;
        q0b[1] += Fqb * shk * cy;
        double cxb = Fqb * shk * q0[0] + 2.0 * cx * c2b, cyb = Fqb * shk * q0[1] + 2.0 * cy * c2b;
        Ub -= cxb; Vb -= cyb;
        maxw_adj(gM, hM, rho0, lam0, cx, cy, gMb, hMb, &rb, &Ub, &Vb, &lb);
    }
    /* shk = (1-Pr) 4 lam^2 / (5 rho) */
    lb += shkb * 2.0 * shk / lam0;
    rb -= shkb * shk / rho0;
    /* A = slope(dwt), dwt = -Mt/rho0 */
    double dwtb[4] = {0, 0, 0, 0}, pb[3] = {0, 0, 0};
    oracle_micro_slope_adj(dwt, U0, V0, lam0, Ab, dwtb, pb);
    Ub += pb[0]; Vb += pb[1]; lb += pb[2];
    double Mtb[4];
    for (int m = 0; m < 4; ++m) {
        Mtb[m] = -dwtb[m] / rho0;
        rb += dwtb[m] * Mt[m] / (rho0 * rho0);
    }
    /* time integrals through tau0 = tau(rho0, lam0) = 2 mu_ref lam^(1-omega)/rho */
    double taub = 0.0;
    for (int m = 0; m < 5; ++m) taub += qcb[m] * dqc[m];
    rb -= taub * tau0 / rho0;
    lb += taub * tau0 * (1.0 - s->omega) / lam0;
    /* ---- reverse of the heat-flux and compatibility loop ---- */
    for (int k = 0; k < nv; ++k) {
        double cx = u[k] - U0, cy = v[k] - V0, c2 = cx * cx + cy * cy;
        double g = f0[k], h = f0[nv + k], E = 0.5 * c2 * g + h;
        double un = axis == 0 ? u[k] : v[k];
        if (un != 0.0) {
            double gM = maxw(rho0, U0, V0, lam0, u[k], v[k]), hM = gM * KINT / (4.0 * lam0);
            double mGb = w[k] * un * (Mtb[0] + Mtb[1] * u[k] + Mtb[2] * v[k] + Mtb[3] * 0.5 * (u[k] * u[k] + v[k] * v[k]));
            double mHb = w[k] * un * Mtb[3];
            double gMb = 0, hMb = 0;
            slope_moments_adj(un > 0 ? aL : aR, u[k], v[k], gM, hM, xi4q, mGb, mHb, un > 0 ? aLb : aRb,
                              &gMb, &hMb, &xib);
            maxw_adj(gM, hM, rho0, lam0, cx, cy, gMb, hMb, &rb, &Ub, &Vb, &lb);
        }
        double qdc = q0b[0] * cx + q0b[1] * cy;
        f0b[k] += w[k] * qdc * 0.5 * c2;
        f0b[nv + k] += w[k] * qdc;
        double cxb = w[k] * (q0b[0] * (E + cx * cx * g) + q0b[1] * cy * cx * g);
        double cyb = w[k] * (q0b[1] * (E + cy * cy * g) + q0b[0] * cx * cy * g);
        Ub -= cxb; Vb -= cyb;
    }
    /* xi4q = K(K+2)/(16 lam^2) */
    lb += xib * (-2.0 * xi4q / lam0);
    /* equilibrium slopes */
    double dwlb[4] = {0, 0, 0, 0}, dwrb[4] = {0, 0, 0, 0};
    pb[0] = Ub; pb[1] = Vb; pb[2] = lb;
    oracle_micro_slope_adj(dwl, U0, V0, lam0, aLb, dwlb, pb);
    oracle_micro_slope_adj(dwr, U0, V0, lam0, aRb, dwrb, pb);
    Ub = pb[0]; Vb = pb[1]; lb = pb[2];
    double W0b[4] = {0, 0, 0, 0}, WLb[4], WRb[4];
    for (int m = 0; m < 4; ++m) {
        W0b[m] += dwlb[m] / (hL * rho0) - dwrb[m] / (hR * rho0);
        WLb[m] = -dwlb[m] / (hL * rho0);
        WRb[m] = dwrb[m] / (hR * rho0);
        rb -= (dwlb[m] * dwl[m] + dwrb[m] * dwr[m]) / rho0;
    }
    prim_adj(W0, rb, Ub, Vb, lb, W0b);
    /* ---- reverse of W0 and of the reconstruction ---- */
    for (int k = 0; k < nv; ++k) {
        double un = axis == 0 ? u[k] : v[k];
        double e2 = 0.5 * (u[k] * u[k] + v[k] * v[k]);
        for (int cp = 0; cp < 2; ++cp) {
            double psiW0 = cp == 0 ? W0b[0] + u[k] * W0b[1] + v[k] * W0b[2] + e2 * W0b[3] : W0b[3];
            double psiL = cp == 0 ? WLb[0] + u[k] * WLb[1] + v[k] * WLb[2] + e2 * WLb[3] : WLb[3];
            double psiR = cp == 0 ? WRb[0] + u[k] * WRb[1] + v[k] * WRb[2] + e2 * WRb[3] : WRb[3];
            double fb = f0b[cp * nv + k] + w[k] * psiW0, sb = sgb[cp * nv + k];
            double fLb = w[k] * psiL, fRb = w[k] * psiR, sLb = 0.0, sRb = 0.0;
            if (un > 0) { fLb += fb; sLb = fb * hL + sb; }
            else if (un < 0) { fRb += fb; sRb = -fb * hR + sb; }
            else { fLb += 0.5 * fb; fRb += 0.5 * fb; sLb = 0.5 * fb * hL + 0.5 * sb; sRb = -0.5 * fb * hR + 0.5 * sb; }
            double fL = FIX(s, cp, cL, k), fR = FIX(s, cp, cR, k);
            if (cLL >= 0) {
                double s1 = (fL - FIX(s, cp, cLL, k)) / dLLL, s2 = (fR - fL) / dLR;
                if (s1 * s2 > 0.0) {
                    /* derivatives of 2 s1 s2 / (s1 + s2): 2 (s2 / (s1 + s2))^2 and 2 (s1 / (s1 + s2))^2,
                       written with the quotients so that they stay finite when the slopes are near
                       the underflow threshold (the far tails of the velocity grid) */
                    double q1 = s1 / (s1 + s2), q2 = s2 / (s1 + s2);
                    double s1b = sLb * 2.0 * q2 * q2, s2b = sLb * 2.0 * q1 * q1;
                    fLb += s1b / dLLL - s2b / dLR;
                    OUTA(out, cp, cLL, k) -= s1b / dLLL;
                    fRb += s2b / dLR;
                }
            }
            if (cRR >= 0) {
                double s2 = (fR - fL) / dLR, s3 = (FIX(s, cp, cRR, k) - fR) / dRRR;
                if (s2 * s3 > 0.0) {
                    double q2 = s2 / (s2 + s3), q3 = s3 / (s2 + s3);
                    double s2b = sRb * 2.0 * q3 * q3, s3b = sRb * 2.0 * q2 * q2;
                    fRb += s2b / dLR - s3b / dRRR;
                    fLb -= s2b / dLR;
                    OUTA(out, cp, cRR, k) += s3b / dRRR;
                }
            }
            OUTA(out, cp, cL, k) += fLb;
            OUTA(out, cp, cR, k) += fRb;
        }
    }
    free(f0); free(sg); free(f0b); free(sgb);
}

/* Adjoint of boundary_face (free transport of the boundary face distribution). */
static void boundary_face_adj(const oracle_solver *s, int bcid, int axis, int outsign, int c,
                              const double *nuG, const double *nuH, double *out)
{
    int nv = s->nv;
    size_t nc = s->lev[0].nc;
    const obc_t *b = &s->bc[bcid];
    double lamw = 1.0 / b->t, rhowb = 0.0, den = 0.0;
    for (int k = 0; k < nv; ++k) {
        double un = axis == 0 ? s->u[k] : s->v[k], uo = outsign * un;
        if (uo >= 0 || b->type == ORC_BC_OUTFLOW) {
            OUTA(out, 0, c, k) += un * nuG[k];
            OUTA(out, 1, c, k) += un * nuH[k];
        } else if (b->type == ORC_BC_WALL) {
            double C = s->Cw[(size_t)bcid * nv + k];
            rhowb += un * (nuG[k] * C + nuH[k] * C * KINT / (4.0 * lamw));
            den += s->w[k] * uo * C;
        } else if (b->type == ORC_BC_SYMMETRY) {
            int km = axis == 0 ? s->mxk[k] : s->myk[k];
            OUTA(out, 0, c, km) += un * nuG[k];
            OUTA(out, 1, c, km) += un * nuH[k];
        }
    }
    if (b->type == ORC_BC_WALL)
        for (int k = 0; k < nv; ++k) {
            double uo = outsign * (axis == 0 ? s->u[k] : s->v[k]);
            if (uo > 0) OUTA(out, 0, c, k) += -s->w[k] * uo * rhowb / den;
        }
}

/* Adjoint of the collision term (g+(W, q) - f)/tau(W) of one cell, with W,
 * q the moments of f about its own velocity; mu = dL/dN of that cell. */
static void collision_adj(const oracle_solver *s, int c, const double *mu, double *out)
{
    int nv = s->nv;
    size_t nc = s->lev[0].nc;
    const double *W = s->W + 4 * c, *q = s->q + 2 * c;
    double rho, U, V, lam;
    prim(W, &rho, &U, &V, &lam);
    double itau = 1.0 / tau_of(s, rho, lam);
    double S = (1.0 - s->pr) * 4.0 / 5.0 * lam * lam / rho;
    double rb = 0, Ub = 0, Vb = 0, lb = 0, Sb = 0, itb = 0, qb[2] = {0, 0};
    for (int k = 0; k < nv; ++k) {
        double cx = s->u[k] - U, cy = s->v[k] - V, c2 = cx * cx + cy * cy;
        double gM = maxw(rho, U, V, lam, s->u[k], s->v[k]), hM = gM * KINT / (4.0 * lam);
        double Fq = S * (cx * q[0] + cy * q[1]);
        double eG = 2.0 * lam * c2 - 4.0, eH = 2.0 * lam * c2 - 2.0;
        double gP = gM * (1.0 + Fq * eG), hP = hM * (1.0 + Fq * eH);
        double mG = OUTA(mu, 0, c, k), mH = OUTA(mu, 1, c, k);
        OUTA(out, 0, c, k) -= mG * itau;
        OUTA(out, 1, c, k) -= mH * itau;
        itb += mG * (gP - FIX(s, 0, c, k)) + mH * (hP - FIX(s, 1, c, k));
        double gPb = mG * itau, hPb = mH * itau;
        double gMb = gPb * (1.0 + Fq * eG), hMb = hPb * (1.0 + Fq * eH);
        double Fqb = gPb * gM * eG + hPb * hM * eH;
        double eb = (gPb * gM + hPb * hM) * Fq;
        lb += eb * 2.0 * c2;
        double c2b = eb * 2.0 * lam;
        Sb += Fqb * (cx * q[0] + cy * q[1]);
        qb[0] += Fqb * S * cx;
        qb[1] += Fqb * S * cy;
        double cxb = Fqb * S * q[0] + 2.0 * cx * c2b, cyb = Fqb * S * q[1] + 2.0 * cy * c2b;
        Ub -= cxb; Vb -= cyb;
        maxw_adj(gM, hM, rho, lam, cx, cy, gMb, hMb, &rb, &Ub, &Vb, &lb);
    }
    lb += Sb * 2.0 * S / lam;
    rb -= Sb * S / rho;
    /* itau = rho lam^(omega-1) / (2 mu_ref) */
    rb += itb * itau / rho;
    lb += itb * itau * (s->omega - 1.0) / lam;
    /* q = sum_k w c (c^2 G/2 + H) about U(f) */
    for (int k = 0; k < nv; ++k) {
        double cx = s->u[k] - U, cy = s->v[k] - V, c2 = cx * cx + cy * cy;
        double g = FIX(s, 0, c, k), E = 0.5 * c2 * g + FIX(s, 1, c, k);
        double qdc = qb[0] * cx + qb[1] * cy;
        OUTA(out, 0, c, k) += s->w[k] * qdc * 0.5 * c2;
        OUTA(out, 1, c, k) += s->w[k] * qdc;
        Ub -= s->w[k] * (qb[0] * (E + cx * cx * g) + qb[1] * cy * cx * g);
        Vb -= s->w[k] * (qb[1] * (E + cy * cy * g) + qb[0] * cx * cy * g);
    }
    double Wb[4] = {0, 0, 0, 0};
    prim_adj(W, rb, Ub, Vb, lb, Wb);
    for (int k = 0; k < nv; ++k) {
        double e2 = 0.5 * (s->u[k] * s->u[k] + s->v[k] * s->v[k]);
        OUTA(out, 0, c, k) += s->w[k] * (Wb[0] + s->u[k] * Wb[1] + s->v[k] * Wb[2] + e2 * Wb[3]);
        OUTA(out, 1, c, k) += s->w[k] * Wb[3];
    }
}

/* N(f) of the steady equations at the current f (W, q renewed from f). */
int oracle_steady_residual(oracle_solver *s, double *N)
{
    olev_t *L0 = &s->lev[0];
    if (s->shock) return fail("adjoint: the pressure-jump collision time is not differentiated");
    int nx = L0->nx, ny = L0->ny, nv = s->nv;
    size_t nc = L0->nc;
    moments(s);
    flux_stage(s);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int c = j * nx + i;
            if (L0->solid[c]) {
                /* a cell in a body holds no state: N = -f keeps the Jacobian regular there */
                for (int cp = 0; cp < 2; ++cp)
                    for (int k = 0; k < nv; ++k) OUTA(N, cp, c, k) = -FIX(s, cp, c, k);
                continue;
            }
            double rho, U, V, lam;
            prim(s->W + 4 * c, &rho, &U, &V, &lam);
            double itau = 1.0 / tau_of(s, rho, lam);
            double Vol = L0->dx[i] * L0->dy[j];
            double qx = s->q[2 * c], qy = s->q[2 * c + 1];
            int fW = j * (nx + 1) + i, fE = fW + 1, fS = j * nx + i, fN = (j + 1) * nx + i;
            for (int k = 0; k < nv; ++k) {
                double gt[2];
                shakhov(rho, U, V, lam, qx, qy, s->pr, s->u[k], s->v[k], &gt[0], &gt[1]);
                for (int cp = 0; cp < 2; ++cp) {
                    const double *px = s->phx + (size_t)cp * L0->nfx * nv, *py = s->phy + (size_t)cp * L0->nfy * nv;
                    double div = (L0->dy[j] * (px[(size_t)fE * nv + k] - px[(size_t)fW * nv + k]) +
                                  L0->dx[i] * (py[(size_t)fN * nv + k] - py[(size_t)fS * nv + k])) / Vol;
                    OUTA(N, cp, c, k) = (gt[cp] - FIX(s, cp, c, k)) * itau - div;
                }
            }
        }
    return 0;
}

/* out = (dN/df)^T mu at the current f. */
int oracle_adjoint_residual(oracle_solver *s, const double *mu, double *out)
{
    olev_t *L0 = &s->lev[0];
    if (s->shock) return fail("adjoint: the pressure-jump collision time is not differentiated");
    int nx = L0->nx, ny = L0->ny, nv = s->nv;
    size_t nc = L0->nc;
    moments(s);
    memset(out, 0, 2 * nc * nv * sizeof(double));
    double *nuG = dalloc(nv), *nuH = dalloc(nv);
    /* x-faces: N_L gets -Phi/dx_L, N_R gets +Phi/dx_R */
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i <= nx; ++i) {
            int fi = j * (nx + 1) + i, bcid = L0->fbx[fi];
            int cL = i > 0 && !L0->solid[j * nx + i - 1] ? j * nx + i - 1 : -1;
            int cR = i < nx && !L0->solid[j * nx + i] ? j * nx + i : -1;
            if (bcid < 0 && (cL < 0 || cR < 0)) continue;        /* inside a body: no flux */
            for (int k = 0; k < nv; ++k) {
                nuG[k] = nuH[k] = 0.0;
                if (cL >= 0) { nuG[k] -= OUTA(mu, 0, cL, k) / L0->dx[i - 1]; nuH[k] -= OUTA(mu, 1, cL, k) / L0->dx[i - 1]; }
                if (cR >= 0) { nuG[k] += OUTA(mu, 0, cR, k) / L0->dx[i]; nuH[k] += OUTA(mu, 1, cR, k) / L0->dx[i]; }
            }
            if (bcid >= 0) {
                int c, os;
                face_side(L0, 0, i, j, &c, &os);
                boundary_face_adj(s, bcid, 0, os, c, nuG, nuH, out);
                continue;
            }
            int hasLL = (i - 1 > 0) && L0->fbx[fi - 1] < 0;
            int hasRR = (i + 1 < nx) && L0->fbx[fi + 1] < 0;
            interior_face_adj(s, 0, hasLL ? cL - 1 : -1, cL, cR, hasRR ? cR + 1 : -1,
                              hasLL ? L0->xc[i - 1] - L0->xc[i - 2] : 1.0, L0->xc[i] - L0->xc[i - 1],
                              hasRR ? L0->xc[i + 1] - L0->xc[i] : 1.0,
                              L0->xn[i] - L0->xc[i - 1], L0->xc[i] - L0->xn[i],
                              L0->dx[i - 1], L0->dx[i], nuG, nuH, out);
        }
    for (int j = 0; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int fi = j * nx + i, bcid = L0->fby[fi];
            int cL = j > 0 && !L0->solid[(j - 1) * nx + i] ? (j - 1) * nx + i : -1;
            int cR = j < ny && !L0->solid[j * nx + i] ? j * nx + i : -1;
            if (bcid < 0 && (cL < 0 || cR < 0)) continue;        /* inside a body: no flux */
            for (int k = 0; k < nv; ++k) {
                nuG[k] = nuH[k] = 0.0;
                if (cL >= 0) { nuG[k] -= OUTA(mu, 0, cL, k) / L0->dy[j - 1]; nuH[k] -= OUTA(mu, 1, cL, k) / L0->dy[j - 1]; }
                if (cR >= 0) { nuG[k] += OUTA(mu, 0, cR, k) / L0->dy[j]; nuH[k] += OUTA(mu, 1, cR, k) / L0->dy[j]; }
            }
            if (bcid >= 0) {
                int c, os;
                face_side(L0, 1, i, j, &c, &os);
                boundary_face_adj(s, bcid, 1, os, c, nuG, nuH, out);
                continue;
            }
            int hasLL = (j - 1 > 0) && L0->fby[fi - nx] < 0;
            int hasRR = (j + 1 < ny) && L0->fby[fi + nx] < 0;
            interior_face_adj(s, 1, hasLL ? cL - nx : -1, cL, cR, hasRR ? cR + nx : -1,
                              hasLL ? L0->yc[j - 1] - L0->yc[j - 2] : 1.0, L0->yc[j] - L0->yc[j - 1],
                              hasRR ? L0->yc[j + 1] - L0->yc[j] : 1.0,
                              L0->yn[j] - L0->yc[j - 1], L0->yc[j] - L0->yn[j],
                              L0->dy[j - 1], L0->dy[j], nuG, nuH, out);
        }
    for (size_t c = 0; c < nc; ++c) {
        if (L0->solid[c]) {                                   /* N = -f in a body */
            for (int cp = 0; cp < 2; ++cp)
                for (int k = 0; k < nv; ++k) OUTA(out, cp, c, k) -= OUTA(mu, cp, c, k);
            continue;
        }
        collision_adj(s, (int)c, mu, out);
    }
    free(nuG); free(nuH);
    return 0;
}

/* Wall objective J = sum over the faces of BC bc of S_face * Q_face, with Q
 * the wall shear (obj 0), heat flux (obj 1) or pressure (obj 2) of
 * oracle_get_wall.  Optionally returns dJ/df (2 x nc x nv, at fixed theta)
 * and dJ/dtheta (theta = T, u, v of the BC, at fixed f). */
int oracle_objective(oracle_solver *s, int obj, int bc, double *J, double *dJdf, double *dJdth)
{
    const olev_t *L0 = &s->lev[0];
    if (s->shock) return fail("adjoint: the pressure-jump collision time is not differentiated");
    int nx = L0->nx, ny = L0->ny, nv = s->nv;
    size_t nc = L0->nc;
    if (bc < 0 || bc >= s->nbc || s->bc[bc].type != ORC_BC_WALL) return fail("objective: BC %d is not a wall", bc);
    if (obj < 0 || obj > 2) return fail("objective: unknown objective %d", obj);
    const obc_t *B = &s->bc[bc];
    double T = B->t, lam = 1.0 / T, Jt = 0.0, th[3] = {0, 0, 0};
    if (dJdf) memset(dJdf, 0, 2 * nc * nv * sizeof(double));
    for (int pass = 0; pass < 2; ++pass) {
        int nfc = pass == 0 ? L0->nfx : L0->nfy;
        for (int fi = 0; fi < nfc; ++fi) {
            int b = pass == 0 ? L0->fbx[fi] : L0->fby[fi];
            if (b != bc) continue;
            int axis = pass, outsign, c;
            double S;
            if (axis == 0) {
                int i = fi % (nx + 1), j = fi / (nx + 1);
                face_side(L0, 0, i, j, &c, &outsign); S = L0->dy[j];
            } else {
                int i = fi % nx, j = fi / nx;
                face_side(L0, 1, i, j, &c, &outsign); S = L0->dx[i];
            }
            double Uwt = axis == 0 ? B->v : B->u;
            /* weights of the face distribution in Q: Q = sum_k w uo (aG fG + aH fH) */
            double num = 0.0, den = 0.0, dden[3] = {0, 0, 0};
            for (int k = 0; k < nv; ++k) {
                double uo = outsign * (axis == 0 ? s->u[k] : s->v[k]);
                if (uo > 0) num += s->w[k] * uo * FIX(s, 0, c, k);
                else if (uo < 0) {
                    double C = s->Cw[(size_t)bc * nv + k];
                    double du = s->u[k] - B->u, dv = s->v[k] - B->v, cw2 = du * du + dv * dv;
                    den += s->w[k] * uo * C;
                    dden[0] += s->w[k] * uo * C * (lam * lam * cw2 - lam);
                    dden[1] += s->w[k] * uo * C * 2.0 * lam * du;
                    dden[2] += s->w[k] * uo * C * 2.0 * lam * dv;
                }
            }
            double rhow = -num / den, rhowb = 0.0;
            double Q = 0.0;
            for (int k = 0; k < nv; ++k) {
                double uo = outsign * (axis == 0 ? s->u[k] : s->v[k]);
                double ut = axis == 0 ? s->v[k] : s->u[k];
                double du = s->u[k] - B->u, dv = s->v[k] - B->v, cw2 = du * du + dv * dv;
                double aG, aH, daG[3] = {0, 0, 0};
                if (obj == 0) { aG = ut - Uwt; aH = 0.0; daG[axis == 0 ? 2 : 1] = -1.0; }
                else if (obj == 1) { aG = 0.5 * cw2; aH = 1.0; daG[1] = -du; daG[2] = -dv; }
                else { aG = uo; aH = 0.0; }
                double wk = s->w[k] * uo;
                if (uo >= 0) {
                    double fG = FIX(s, 0, c, k), fH = FIX(s, 1, c, k);
                    Q += wk * (aG * fG + aH * fH);
                    for (int p = 0; p < 3; ++p) th[p] += S * wk * daG[p] * fG;
                    if (dJdf) {
                        OUTA(dJdf, 0, c, k) += S * wk * aG;
                        OUTA(dJdf, 1, c, k) += S * wk * aH;
                    }
                } else {
                    double C = s->Cw[(size_t)bc * nv + k];
                    double dC[3] = {C * (lam * lam * cw2 - lam), C * 2.0 * lam * du, C * 2.0 * lam * dv};
                    double hf = KINT * T / 4.0;                 /* H/G ratio of the wall Maxwellian */
                    double a = aG + aH * hf;
                    Q += wk * rhow * C * a;
                    rhowb += S * wk * C * a;
                    for (int p = 0; p < 3; ++p) {
                        double drho = -rhow / den * dden[p];
                        double da = daG[p] + (p == 0 ? aH * KINT / 4.0 : 0.0);
                        th[p] += S * wk * (drho * C * a + rhow * dC[p] * a + rhow * C * da);
                    }
                }
            }
            Jt += S * Q;
            if (dJdf)
                for (int k = 0; k < nv; ++k) {
                    double uo = outsign * (axis == 0 ? s->u[k] : s->v[k]);
                    if (uo > 0) OUTA(dJdf, 0, c, k) += -s->w[k] * uo * rhowb / den;
                }
        }
    }
    *J = Jt;
    if (dJdth) for (int p = 0; p < 3; ++p) dJdth[p] = th[p];
    return 0;
}

/* dN/dtheta at fixed f for theta = T (param 0), u (1) or v (2) of wall BC bc:
 * only the incoming velocities of the wall faces of that BC depend on it. */
int oracle_residual_dtheta(oracle_solver *s, int bc, int param, double *dN)
{
    const olev_t *L0 = &s->lev[0];
    if (s->shock) return fail("adjoint: the pressure-jump collision time is not differentiated");
    int nx = L0->nx, ny = L0->ny, nv = s->nv;
    size_t nc = L0->nc;
    if (bc < 0 || bc >= s->nbc || s->bc[bc].type != ORC_BC_WALL) return fail("dtheta: BC %d is not a wall", bc);
    if (param < 0 || param > 2) return fail("dtheta: unknown parameter %d", param);
    const obc_t *B = &s->bc[bc];
    double T = B->t, lam = 1.0 / T;
    memset(dN, 0, 2 * nc * nv * sizeof(double));
    for (int pass = 0; pass < 2; ++pass) {
        int nfc = pass == 0 ? L0->nfx : L0->nfy;
        for (int fi = 0; fi < nfc; ++fi) {
            int b = pass == 0 ? L0->fbx[fi] : L0->fby[fi];
            if (b != bc) continue;
            int axis = pass, outsign, c;
            double h;
            if (axis == 0) {
                int i = fi % (nx + 1), j = fi / (nx + 1);
                face_side(L0, 0, i, j, &c, &outsign); h = L0->dx[c % nx];
            } else {
                int i = fi % nx, j = fi / nx;
                face_side(L0, 1, i, j, &c, &outsign); h = L0->dy[c / nx];
            }
            /* N_c += outsign * (-1/h) * Phi_face: the face is the cell's upper face when outsign = +1 */
            double coef = -outsign / h;
            double num = 0.0, den = 0.0, dden = 0.0;
            for (int k = 0; k < nv; ++k) {
                double uo = outsign * (axis == 0 ? s->u[k] : s->v[k]);
                if (uo > 0) num += s->w[k] * uo * FIX(s, 0, c, k);
                else if (uo < 0) {
                    double C = s->Cw[(size_t)bc * nv + k];
                    double du = s->u[k] - B->u, dv = s->v[k] - B->v;
                    double dC = param == 0 ? C * (lam * lam * (du * du + dv * dv) - lam)
                                           : C * 2.0 * lam * (param == 1 ? du : dv);
                    den += s->w[k] * uo * C;
                    dden += s->w[k] * uo * dC;
                }
            }
            double rhow = -num / den, drho = -rhow / den * dden;
            for (int k = 0; k < nv; ++k) {
                double un = axis == 0 ? s->u[k] : s->v[k], uo = outsign * un;
                if (!(uo < 0)) continue;
                double C = s->Cw[(size_t)bc * nv + k];
                double du = s->u[k] - B->u, dv = s->v[k] - B->v;
                double dC = param == 0 ? C * (lam * lam * (du * du + dv * dv) - lam)
                                       : C * 2.0 * lam * (param == 1 ? du : dv);
                double dG = drho * C + rhow * dC;
                double dH = dG * KINT * T / 4.0 + (param == 0 ? rhow * C * KINT / 4.0 : 0.0);
                OUTA(dN, 0, c, k) += coef * un * dG;
                OUTA(dN, 1, c, k) += coef * un * dH;
            }
        }
    }
    return 0;
}

/* One CS cycle (Eq. CSCYC) as a linear map of the level-0 residual r with
 * frozen coefficients: inv_tau holds the collision frequency of every level,
 * level after level (sum of nc_l values); df = the total correction. */
int oracle_stage_cs(oracle_solver *s, const double *inv_tau, const double *r, double *df)
{
    size_t off = 0;
    for (int l = 0; l < s->L; ++l) {
        memcpy(s->lev[l].inv_tau, inv_tau + off, (size_t)s->lev[l].nc * sizeof(double));
        off += (size_t)s->lev[l].nc;
    }
    size_t n = 2 * (size_t)s->lev[0].nc * s->nv;
    memcpy(s->lev[0].r, r, n * sizeof(double));
    cs(s, 0, s->cycle);
    memcpy(df, s->lev[0].df, n * sizeof(double));
    return 0;
}

/* Multigrid cycle type of both the FAS and the CS cycle (Sec. 3.4 names V, W,
 * F and adaptive cycles): 0 V (default), 1 W, 2 F. */
/* decisions of the adaptive cycle so far (1 = a second coarse visit), the last
 * min(n, cap, ADAPT_LOG) of them in order; returns their total count */
int oracle_adapt_log(const oracle_solver *s, unsigned char *out, int cap)
{
    int n = s->adapt_n, m = n < cap ? n : cap;
    if (m > ADAPT_LOG) m = ADAPT_LOG;
    for (int q = 0; q < m; ++q) out[q] = s->adapt_log[(n - m + q) % ADAPT_LOG];
    return n;
}

int oracle_set_shock_capturing(oracle_solver *s, int on)
{
    s->shock = on != 0;
    return 0;
}

int oracle_set_adapt_ratio(oracle_solver *s, double ratio)
{
    if (!(ratio >= 0.0)) return fail("adaptive ratio %g must be >= 0", ratio);
    s->adapt_ratio = ratio;
    return 0;
}

int oracle_set_cycle(oracle_solver *s, int type)
{
    if (type < 0 || type > 3) return fail("cycle type %d: 0 V, 1 W, 2 F, 3 adaptive", type);
    s->cycle = type;
    return 0;
}

/* Full-multigrid start-up (Sec. 3.5): the state of a solver on the next
 * coarser mesh (every second grid line, same velocity grid) becomes the
 * initial state of this one by the bilinear prolongation of Eq. prolongation,
 * applied to f velocity by velocity; W and q follow from the moments. */
int oracle_init_from_coarse(oracle_solver *s, const oracle_solver *c)
{
    if (s->L < 2) return fail("init_from_coarse: the fine solver needs at least two levels");
    const olev_t *F1 = &s->lev[1], *C0 = &c->lev[0];
    if (c->nv != s->nv || C0->nx != F1->nx || C0->ny != F1->ny)
        return fail("init_from_coarse: the coarse solver is not on the next coarser mesh");
    for (int i = 0; i <= F1->nx; ++i)
        if (fabs(C0->xn[i] - F1->xn[i]) > 1e-12 * (1.0 + fabs(F1->xn[i]))) return fail("init_from_coarse: x nodes differ");
    for (int j = 0; j <= F1->ny; ++j)
        if (fabs(C0->yn[j] - F1->yn[j]) > 1e-12 * (1.0 + fabs(F1->yn[j]))) return fail("init_from_coarse: y nodes differ");
    size_t ncC = C0->nc, ncF = s->lev[0].nc;
    for (int cp = 0; cp < 2; ++cp)
        prolong_lv_s(&s->lev[0], &s->lev[1], s->nv, c->f + (size_t)cp * ncC * s->nv, s->f + (size_t)cp * ncF * s->nv, 1);
    /* a fine cell whose prolonged f has non-positive density or internal energy
     * (extrapolation next to an edge or a body across a strong gradient) takes
     * the f of its coarse cell instead (reading: the paper is silent) */
    const olev_t *L0 = &s->lev[0];
    int nv = s->nv;
    for (int j = 0; j < L0->ny; ++j)
        for (int i = 0; i < L0->nx; ++i) {
            size_t cf = (size_t)j * L0->nx + i, cc = (size_t)(j / 2) * C0->nx + i / 2;
            double W[4] = {0, 0, 0, 0};
            for (int k = 0; k < nv; ++k) {
                double g = FIX(s, 0, cf, k), h = FIX(s, 1, cf, k);
                W[0] += s->w[k] * g;
                W[1] += s->w[k] * s->u[k] * g;
                W[2] += s->w[k] * s->v[k] * g;
                W[3] += s->w[k] * (0.5 * (s->u[k] * s->u[k] + s->v[k] * s->v[k]) * g + h);
            }
            if (W[0] > 0.0 && W[3] * W[0] - 0.5 * (W[1] * W[1] + W[2] * W[2]) > 0.0) continue;
            for (int cp = 0; cp < 2; ++cp)
                for (int k = 0; k < nv; ++k)
                    FIX(s, cp, cf, k) = c->f[((size_t)cp * ncC + cc) * nv + k];
        }
    moments(s);
    s->iter = 0;
    return 0;
}
