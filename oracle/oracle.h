/*
 * oracle.h -- plain, serial, FP64 CPU oracle of the multigrid implicit unified
 * gas-kinetic scheme (MIUGKS) of Zhu, Zhong & Xu, "Unified Gas-kinetic Scheme
 * with Multigrid Convergence for Rarefied Flow Study" (arXiv 1704.03151).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA library under
 * paper_1704_03151_gb300/csrc, and the CUDA library never calls it.
 *
 * Conventions (all nondimensional): gas constant R = 1/2, reference density,
 * temperature and length 1, so lambda = 1/(2RT) = 1/T and p = rho*T/2.
 * Monatomic gas in 2-D with one internal (z-translational) degree of freedom:
 * two reduced distributions per (cell, velocity), G = int f dxi_z and
 * H = int xi_z^2/2 f dxi_z.
 *
 * Layouts: cell c = j*nx + i; f[(comp*nc + c)*nv + k] with comp 0 = G, 1 = H;
 * velocity k = a*nv_v + b with u_k = u_a, v_k = v_b.  x-faces indexed
 * j*(nx+1) + i (face between cells i-1 and i), y-faces j*nx + i (between
 * rows j-1 and j).  A face BC id of -1 marks an interior face.
 *
 * Every function returns 0 on success and a nonzero status on error, with a
 * message available from oracle_last_error().
 */
#ifndef MIUGKS_ORACLE_H
#define MIUGKS_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_BC_WALL = 0, ORC_BC_SYMMETRY = 1, ORC_BC_FARFIELD = 2, ORC_BC_OUTFLOW = 3 };

typedef struct oracle_solver oracle_solver;

/* Build the solver: mesh (rectilinear nodes), face boundary ids, BC table
 * (bc_vals = nbc x {rho, u, v, T}), velocity grid, gas and multigrid options.
 * levels = 1 is the single-grid implicit UGKS (one smoothing per step). */
oracle_solver *oracle_create(int nx, int ny, const double *xn, const double *yn,
                             const int *face_bc_x, const int *face_bc_y, const unsigned char *solid,
                             int nbc, const int *bc_type, const double *bc_vals,
                             int nu, int nv, double umin, double umax,
                             double vmin, double vmax, int rule,
                             double kn, double omega, double pr,
                             int levels, int nu1, int nu2, int nuc,
                             double cfl, double dtn_growth);
const char *oracle_last_error(void);
void oracle_destroy(oracle_solver *s);

int oracle_init_uniform(oracle_solver *s, double rho, double u, double v, double t);
int oracle_init_fields(oracle_solver *s, const double *rho, const double *u,
                       const double *v, const double *t);
/* n outer iterations (Steps 1-8); res = RMS residual of the last Step 1. */
int oracle_step(oracle_solver *s, int n, double res[4]);
/* Full-multigrid start-up: f of a solver on the next coarser mesh (every
 * second grid line, same velocity grid) prolonged bilinearly onto this one. */
int oracle_init_from_coarse(oracle_solver *s, const oracle_solver *coarse);
/* Multigrid cycle type of the FAS and CS cycles: 0 V (default), 1 W, 2 F. */
int oracle_set_cycle(oracle_solver *s, int type);
int oracle_adapt_log(const oracle_solver *s, unsigned char *out, int cap);
int oracle_set_adapt_ratio(oracle_solver *s, double ratio);
/* pressure-jump term of the interface collision time (shock capturing), 0 off (default) */
int oracle_set_shock_capturing(oracle_solver *s, int on);
int oracle_get_macro(const oracle_solver *s, double *rho, double *u, double *v,
                     double *t, double *qx, double *qy);
int oracle_get_f(const oracle_solver *s, double *f);
int oracle_set_f(oracle_solver *s, const double *f);
/* wall quantities along the faces carrying BC id bc (in face-index order:
 * x-faces first, then y-faces); *nf in: capacity, out: count. */
int oracle_get_wall(const oracle_solver *s, int bc, int *nf, double *p,
                    double *tau, double *q);
int oracle_set_bc(oracle_solver *s, int bc, double rho, double u, double v, double t);
/* Step 1 alone: the macroscopic residual R (nc x 4) of the current state. */
int oracle_residual(oracle_solver *s, double *R);
int oracle_iterations(const oracle_solver *s);

/* ---- building blocks exposed for the pins (tests/test_oracle_*.py) ---- */
int oracle_vgrid(int n, double a, double b, int rule, double *x, double *w);
void oracle_time_coeffs(double dt, double tau, double q[5]);
void oracle_micro_slope(const double dw[4], double U, double V, double lam, double a[4]);
/* Shakhov equilibrium (G+, H+) of state (rho, U, V, lambda) with heat flux (qx, qy) at n nodes (Sec. 2.1) */
void oracle_shakhov(double rho, double U, double V, double lam, double qx, double qy, double pr, int n,
                    const double *u, const double *v, double *G, double *H);
double oracle_vanleer(double s1, double s2);
double oracle_mu_ref(double kn, double omega);
void oracle_wall_jacobian(const double W[4], double Uw, double Vw, double Tw, double M[16]);
void oracle_wall_ghost(const double W[4], double Uw, double Vw, double Tw, double Wg[4]);
/* Internal stages on level 0 of an existing solver (f, W already set):
 *  flux   : Step 1 -> R (nc x 4) and the time-averaged micro face fluxes
 *           phx (2 x nfx x nv), phy (2 x nfy x nv)                            */
int oracle_stage_flux(oracle_solver *s, double *R, double *phx, double *phy);
/*  sgs_micro : one symmetric Gauss-Seidel pass on level lev for residual r
 *              (2 x nc_l x nv), collision frequency 1/tau per cell (inv_tau),
 *              order 0 = lexicographic, 1 = anti-diagonal wavefront.          */
int oracle_stage_sgs_micro(oracle_solver *s, int lev, const double *inv_tau,
                           const double *r, double *dx_out, int order);
/*  apply_micro : y = A x with the full evolution operator (all ghosts).       */
int oracle_stage_apply_micro(oracle_solver *s, int lev, const double *inv_tau,
                             const double *x, double *y);
/*  sgs_macro : one LU-SGS pass of the prediction smoother on level lev.       */
int oracle_stage_sgs_macro(oracle_solver *s, int lev, const double *W,
                           const double *Wn_gamma, const double *R, double *dW, int order);
/*  resid_macro : split-Euler residual R_E(W) on level lev (Gamma from Wg).    */
int oracle_stage_resid_macro(oracle_solver *s, int lev, const double *W,
                             const double *Wg, double *RE);
int oracle_stage_restrict(oracle_solver *s, int lev, int ncomp, const double *fine, double *coarse);
int oracle_stage_prolong(oracle_solver *s, int lev, int ncomp, const double *coarse, double *fine);
int oracle_level_size(const oracle_solver *s, int lev, int *nx, int *ny);
/*  cs : one CS cycle as a linear map of the level-0 residual r (2 x nc x nv),
 *       inv_tau of every level concatenated (sum of nc_l values) -> df.      */
int oracle_stage_cs(oracle_solver *s, const double *inv_tau, const double *r, double *df);
int oracle_nv(const oracle_solver *s);

/* ---- steady equations and their adjoint (differentiation form) ----
 * N(f; theta) = (g+(W(f), q(f)) - f)/tau(W(f)) - (1/V) sum S Phi(f; theta)/dt_p,
 * the discrete steady equations the outer iteration converges to.  theta =
 * (T, u, v) of one wall BC.  Objectives (wall bc, face order of
 * oracle_get_wall): obj 0 = sum_faces S * shear, 1 = S * heat flux,
 * 2 = S * pressure. */
int oracle_steady_residual(oracle_solver *s, double *N);
int oracle_adjoint_residual(oracle_solver *s, const double *mu, double *out);  /* (dN/df)^T mu */
int oracle_objective(oracle_solver *s, int obj, int bc, double *J, double *dJdf, double *dJdtheta);
int oracle_residual_dtheta(oracle_solver *s, int bc, int param, double *dN);
void oracle_time_coeffs_dtau(double dt, double tau, double dq[5]);
void oracle_micro_slope_adj(const double dw[4], double U, double V, double lam, const double abar[4],
                            double dwbar[4], double pbar[3]);

#ifdef __cplusplus
}
#endif
#endif
