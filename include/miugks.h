/*
 * miugks.h -- C ABI of the GB300 (sm_103a) multigrid implicit unified
 * gas-kinetic scheme (MIUGKS) library.
 *
 * Method: Zhu, Zhong & Xu, "Unified Gas-kinetic Scheme with Multigrid
 * Convergence for Rarefied Flow Study", arXiv 1704.03151.  One call of
 * miugks_step() performs Steps 1-8 of Sec. 2.4 once per iteration: explicit
 * UGKS fluxes and residuals (Sec. 2.1, Eqs. macroResidualDef,
 * macroResidualCalc, microResidualDef), the FAS prediction of the conservative
 * variables (Eq. FASCYC), the predicted equilibrium, the CS evolution of the
 * distribution function (Eq. CSCYC), its update and the moments.
 *
 * Units (nondimensional): gas constant R = 1/2, reference density,
 * temperature and length 1 -- so lambda = 1/(2RT) = 1/T, p = rho T / 2 and
 * the most probable speed is 1.  2-D monatomic gas with one internal degree
 * of freedom: two reduced distributions per (cell, velocity).
 *
 * Layouts.  Cells are row-major, c = j*nx + i.  The distribution function is
 * f[(comp*nc + c)*nv + k] (comp 0: G = int f dxi_z, comp 1: H = int xi_z^2/2
 * f dxi_z) with discrete velocity k = a*nv_v + b, u_k = u_a, v_k = v_b.
 * x-faces are indexed j*(nx+1) + i (between cells i-1 and i), y-faces
 * j*nx + i (between rows j-1 and j); a face BC id of -1 marks an interior face.
 * Boundary ids sit on the outer edges of the rectangle and on the faces of
 * bodies (solid cells, see miugks_mesh).
 *
 * Ownership and errors.  The library owns all device memory of a solver; it
 * allocates through the caller's callbacks when given (the Python binding
 * passes PyTorch's caching allocator), else with cudaMalloc, and works on the
 * caller's CUDA stream (or the legacy default stream).  Arrays passed in or
 * out are HOST arrays owned by the caller unless a name says _dev.  Every
 * call returns a status and never aborts; miugks_last_error() gives the
 * message of the last failure of that solver (valid until its next call).
 * A solver must not be used by two threads at once.
 */
#ifndef MIUGKS_H
#define MIUGKS_H
#include <stddef.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct miugks_solver miugks_solver;

typedef enum {
    MIUGKS_OK = 0,
    MIUGKS_EINVAL = 1,         /* invalid argument or unsupported configuration   */
    MIUGKS_ENOMEM = 2,         /* device or host allocation failed                */
    MIUGKS_ECUDA = 3,          /* CUDA runtime error (message has the details)    */
    MIUGKS_EDIVERGED = 4,      /* non-positive density or temperature, or NaN     */
    MIUGKS_ETIMEOUT = 5,       /* a bounded device wait gave up (sticky)          */
    MIUGKS_ENOTCONVERGED = 6,  /* miugks_run reached max_iter above tolerance    */
    MIUGKS_ESTATE = 7          /* call order (e.g. step before init)              */
} miugks_status;

typedef enum { MIUGKS_BC_WALL = 0, MIUGKS_BC_SYMMETRY = 1, MIUGKS_BC_FARFIELD = 2, MIUGKS_BC_OUTFLOW = 3 } miugks_bc_type;
/* FP64: every step in double precision.  MIXED: f, fluxes, residuals and the
 * evolution smoother in single precision (per-velocity arithmetic), with the
 * velocity sums Kahan-compensated and combined in double; the conservative
 * variables, per-face scalars, moments, the FAS prediction and the macroscopic
 * residual stay in double. */
typedef enum { MIUGKS_FP64 = 0, MIUGKS_MIXED = 1 } miugks_precision;

/* rectilinear mesh: x_nodes[nx+1], y_nodes[ny+1] increasing; face ids as above.
 * solid (nx*ny, NULL = none) marks cells inside bodies (the square cylinder of
 * Sec. 4.3): they hold no state and are never updated.  A face between two
 * fluid cells has id -1; a face between a fluid cell and a body or the domain
 * edge needs a BC id; a face with no fluid cell on either side is ignored.
 * With multigrid, bodies must fill whole cells of every coarse level. */
typedef struct {
    int nx, ny;
    const double *x_nodes, *y_nodes;
    const int *face_bc_x;      /* (nx+1)*ny */
    const int *face_bc_y;      /* nx*(ny+1) */
    const unsigned char *solid;
} miugks_mesh;

/* discrete velocities: nu x nv nodes, placed symmetrically on [umin,umax] x
 * [vmin,vmax]; rule 0 trapezoid (Sec. 4.1), 1 composite Boole, closed
 * Newton-Cotes of degree 4, needing (n-1) % 4 == 0 (Sec. 4.3) */
typedef struct { int nu, nv; double umin, umax, vmin, vmax; int rule; } miugks_vgrid;

/* Kn (VHS, alpha = 1), viscosity index omega (mu ~ T^omega), Prandtl number
 * of the Shakhov equilibrium (Sec. 2.1) */
typedef struct { double kn, omega, pr; } miugks_gas;

/* boundary condition (Sec. 3.2): wall = diffuse isothermal wall moving with
 * (u, v) at temperature t; symmetry = specular plane (needs a velocity grid
 * symmetric about 0); farfield = Maxwellian (rho, u, v, t) entering;
 * outflow = zero gradient */
typedef struct { int type; double rho, u, v, t; } miugks_bc;

/* multigrid options (Secs. 2.4, 3.4): levels (1 = single-grid implicit UGKS
 * with one smoothing per step), pre/post smoothings nu1/nu2 (2/1 in the
 * paper), smoothings on the coarsest level, CFL number of the physical time
 * step, growth factor a of the numerical time step dt_n = a^n dt_p (0 = off). */
typedef struct {
    int levels, nu1, nu2, nu_coarse;
    double cfl, dtn_growth;
    int precision;                                   /* miugks_precision */
    void *cuda_stream;                               /* cudaStream_t or NULL */
    void *(*dev_alloc)(size_t bytes, void *ctx);     /* NULL: cudaMalloc */
    void (*dev_free)(void *ptr, void *ctx);
    void *alloc_ctx;
} miugks_opts;

/* Build a solver (host mesh hierarchy by 2x2 agglomeration, Sec. 3.1; device
 * state).  nx and ny must be divisible by 2^(levels-1).  On error *out is NULL. */
miugks_status miugks_create(const miugks_mesh *mesh, const miugks_vgrid *vgrid, const miugks_gas *gas,
                            const miugks_bc *bcs, int n_bcs, const miugks_opts *opts, miugks_solver **out);
void miugks_destroy(miugks_solver *s);
const char *miugks_last_error(const miugks_solver *s);

/* Initial state: discrete Maxwellian of (rho, u, v, t), uniform or per cell (host arrays of nc). */
miugks_status miugks_init_uniform(miugks_solver *s, double rho, double u, double v, double t);
miugks_status miugks_init_fields(miugks_solver *s, const double *rho, const double *u, const double *v,
                                 const double *t);

/* n outer iterations (Steps 1-8).  res_out (may be NULL): RMS of the
 * macroscopic residual per component (rho, rho U, rho V, rho eps) over the
 * fluid cells, evaluated in Step 1 of the last iteration (Eq. Residual_Def).
 * A cell whose FAS correction, predicted state or update would have
 * non-positive density or internal energy keeps its previous value there (the
 * paper is silent; this never triggers in smooth flow).  Returns
 * MIUGKS_EDIVERGED when the state became unphysical all the same. */
miugks_status miugks_step(miugks_solver *s, int n_iter, double res_out[4]);
/* Enqueue n outer iterations on the solver's stream and return without waiting;
 * miugks_wait() then waits for them and returns the RMS residual of the last
 * one (and MIUGKS_EDIVERGED as miugks_step does).  Lets one host thread keep
 * many solvers, each on its own stream, running concurrently.  On a stream other
 * than the legacy default stream, iterations after the first are replayed from
 * a captured CUDA graph. */
miugks_status miugks_step_async(miugks_solver *s, int n_iter);
miugks_status miugks_wait(miugks_solver *s, double res_out[4]);
/* iterate until every RMS component is below tol (Sec. 4.1) or max_iter */
miugks_status miugks_run(miugks_solver *s, double tol, int max_iter, int *iters_out, double res_out[4]);
/* RMS residual of the current state (Step 1 only) */
miugks_status miugks_residual(miugks_solver *s, double res_out[4]);
int miugks_iterations(const miugks_solver *s);

/* Macroscopic fields (host, nc each; NULL skips) and the distribution function
 * (host, 2*nc*nv doubles in the layout above). */
miugks_status miugks_get_macro(miugks_solver *s, double *rho, double *u, double *v, double *t, double *qx,
                               double *qy);
miugks_status miugks_get_f(miugks_solver *s, double *f);
miugks_status miugks_set_f(miugks_solver *s, const double *f);
/* Wall pressure, shear stress and heat flux (Secs. 4.2, 4.3: momentum and
 * energy carried into the wall per unit area and time, in the wall frame)
 * for the faces with BC id bc, x-faces first, each in face-index order.
 * *n_faces: in capacity, out count (call with capacity 0 to size). */
miugks_status miugks_get_wall(miugks_solver *s, int bc, int *n_faces, double *p, double *tau, double *q);
miugks_status miugks_set_bc(miugks_solver *s, int bc, const miugks_bc *value);
/* Multigrid cycle type of both the prediction (FAS, Eq. FASCYC) and the
 * evolution (CS, Eq. CSCYC) cycles; Sec. 3.4 names V, W and F cycles and
 * evaluates only the V cycle.  type 0 V (default), 1 W (two coarse visits of
 * type W), 2 F (an F visit then a V visit), 3 adaptive (below).  A second FAS visit starts from the
 * coarse state the first left, with the same forcing function and frozen
 * Gamma; a second CS visit solves for the coarse residual the first correction
 * leaves.  W and F need two more per-velocity arrays per coarse level, taken
 * from the solver's allocator on the first selection.  The adjoint's
 * preconditioner stays the transposed V cycle.  MIUGKS_EINVAL for another type. */
miugks_status miugks_set_cycle(miugks_solver *s, int type);
/* Adaptive cycle (type 3 of miugks_set_cycle; Sec. 3.4 names adaptive cycles
 * without a rule): each level visits the next coarser level once and visits
 * it a second time when the first visit left more than `ratio` (default 0.2)
 * of the coarse residual it started from, in the L2 norm over all values: for
 * FAS the restricted residual against P + R_E(W) of the coarse state left, for
 * CS r_H against r_H - A_H df_H.  ratio 0 gives the W cycle, a ratio no visit
 * reaches the V cycle.  Each decision reads a norm back to the host, so
 * iterations of this type are launched eagerly, never from a captured graph.
 * set_adaptive_ratio: MIUGKS_EINVAL for a negative ratio.
 * adaptive_decisions: the last min(n, cap, 4096) decisions, oldest first
 * (1 = a second visit), into out (may be NULL); returns n, the number taken. */
miugks_status miugks_set_adaptive_ratio(miugks_solver *s, double ratio);
/* Launch layout of the evolution smoother's sweeps (Eq. microFinalDefect); the
 * result is the same bit for bit.  In a sweep pass a velocity whose u (or v)
 * points away from the upwind neighbour in x (or y) has a zero coefficient
 * there: velocities coupled in both directions need the anti-diagonal
 * wavefront, the others are independent along rows, along columns or per
 * cell.  mode 1 sweeps those in a separate line-parallel kernel, 2 sweeps every
 * velocity in the wavefront kernel, 0 (default) splits a level from 20 Mi
 * cell-velocity pairs on.  MIUGKS_EINVAL for another mode. */
miugks_status miugks_set_sweep_split(miugks_solver *s, int mode);
/* Shock capturing (off by default; the paper describes none, and runs its
 * Ma 5 case without): on != 0 adds the pressure-jump term of the gas-kinetic
 * schemes, dt_p |p_L - p_R| / (p_L + p_R) with p = rho / (2 lambda) of the two
 * cells, to the collision time of every interior interface in Step 1's flux
 * (Sec. 2.1), which adds numerical dissipation where the pressure jumps and
 * nothing where it is continuous.  The adjoint (which does not differentiate
 * this term) returns MIUGKS_EINVAL while it is on. */
miugks_status miugks_set_shock_capturing(miugks_solver *s, int on);
/* Bound of the prediction smoother's device waits (the cluster sweep of Eq.
 * macroFinalDefect waits for each diagonal's inputs and its neighbours'
 * values): a wait that has not completed after `seconds` (default 0.2, at
 * most 10) gives up, the kernel drains its copies in flight (waits bounded by
 * the default) and returns, and the next miugks_step / miugks_wait returns
 * MIUGKS_ETIMEOUT (sticky for the solver).  0 makes every such wait give up
 * without testing its inputs: it exercises the failure path without a fault
 * (the kernel computes one step on whatever the buffers hold, then drains and
 * returns; the state is garbage and the solver is to be destroyed), and the
 * CUDA context stays usable.  MIUGKS_EINVAL outside [0, 10]. */
miugks_status miugks_set_wait_limit(miugks_solver *s, double seconds);
int miugks_adaptive_decisions(const miugks_solver *s, unsigned char *out, int cap);
/* Full-multigrid start-up (Sec. 3.5): the state of `coarse`, a solver of the
 * same problem on the next coarser mesh (every second grid line of s's mesh,
 * same velocity grid and precision), becomes s's initial state by the bilinear
 * prolongation of Eq. prolongation applied to f velocity by velocity (a cell
 * whose prolonged f has non-positive density or internal energy, and a cell in
 * a body, takes its coarse cell's f); W and q follow from its moments and the
 * iteration count restarts at 0.  s needs at least two levels.  Waits for
 * coarse's stream.  MIUGKS_EINVAL when the meshes, bodies, velocity grids or
 * precisions do not match, MIUGKS_ESTATE when coarse has no state. */
miugks_status miugks_init_from_coarse(miugks_solver *s, const miugks_solver *coarse);
/* The state of src (f, and the iteration count that sets dt_n) becomes s's: a
 * solver of the same mesh, bodies and velocity grid, of either precision (f is
 * converted; W and q follow from its moments).  With it a run can take its
 * bulk of iterations in the mixed form and finish in FP64, where the FP32
 * rounding of the per-velocity fluxes sets a residual floor above the
 * tolerance (the paper runs FP64 throughout).  Waits for src's stream.
 * MIUGKS_EINVAL when the problems differ, MIUGKS_ESTATE when src has no state. */
miugks_status miugks_copy_state(miugks_solver *s, const miugks_solver *src);

/* Stages of one iteration on explicit host data, for kernel-level checks.
 *  flux: Step 1 at the current state -> R (nc x 4), time-averaged micro face
 *        fluxes phx (2 x nfx x nv) and phy (2 x nfy x nv); any may be NULL.
 *  sgs_micro: one LU-SGS pass of the evolution smoother on level lev with
 *        collision frequency inv_tau (nc_l) for residual r (2 x nc_l x nv).
 *  apply_micro: y = A x with the full evolution operator of level lev.
 *  sgs_macro: one LU-SGS pass of the prediction smoother at state W with
 *        Gamma frozen at Wg, residual R, and 1/dt_n of the current iteration
 *        on the diagonal (when dt_n growth is on); returns dW (all nc_l x 4).
 *  resid_macro: split-Euler residual R_E(W) with Gamma frozen at Wg.
 *  restrict / prolong: transfer of an [nc][m] array between lev and lev+1. */
miugks_status miugks_stage_flux(miugks_solver *s, double *R, double *phx, double *phy);
miugks_status miugks_stage_sgs_micro(miugks_solver *s, int lev, const double *inv_tau, const double *r, double *x);
miugks_status miugks_stage_apply_micro(miugks_solver *s, int lev, const double *inv_tau, const double *x, double *y);
miugks_status miugks_stage_sgs_macro(miugks_solver *s, int lev, const double *W, const double *Wg, const double *R,
                                     double *dW);
miugks_status miugks_stage_resid_macro(miugks_solver *s, int lev, const double *W, const double *Wg, double *RE);
miugks_status miugks_stage_restrict(miugks_solver *s, int lev, int m, const double *fine, double *coarse);
miugks_status miugks_stage_prolong(miugks_solver *s, int lev, int m, const double *coarse, double *fine);

/* ---- Differentiation form: adjoint of the steady equations ----
 * At a converged state the outer iteration solves the discrete steady
 * equations N(f; theta) = 0 of Eq. microResidualDef (Sec. 2.1) with the
 * predicted state equal to the moments of f, the UGKS interface flux of Step 1
 * and the diffuse wall of Sec. 3.2 (Eq. f_on_wall).  theta is the temperature
 * (param 0), x-velocity (1) or y-velocity (2) of one wall BC.  Objectives of a
 * wall BC: obj 0 = sum over its faces of face length x shear stress, 1 = heat
 * flux, 2 = pressure (the quantities of miugks_get_wall).  All in FP64 on an
 * FP64 copy (checkpoint) of the current f, whatever the solver's precision
 * (a state converged in the mixed form keeps its FP32 rounding there; a few
 * FP64 iterations from it, through miugks_copy_state, make the Krylov solve
 * converge several times faster).
 * On a mesh with bodies a body's faces are wall faces of the fluid cells beside
 * them and a cell in a body holds no state (N = -f there); the transposed-cycle
 * preconditioner carries the wall coupling of a body's faces as of the domain
 * edge's (a cell with two wall faces on one sweep side, at a concave body
 * corner, keeps the plain wavefront value there, which the Krylov solve
 * corrects).
 *
 *  stage_adjoint_residual: out = (dN/df)^T mu at the current f, host arrays
 *        of 2 x nc x nv ([comp][cell][k]).
 *  stage_sgs_micro_transposed: x = P^T r with P one LU-SGS pass of the
 *        evolution smoother on level 0 (collision frequency inv_tau, nc).
 *  objective: J, dJ/df (host, 2 x nc x nv, may be NULL) and dJ/dtheta at
 *        fixed f (3 values: T, u, v).
 *  adjoint: gradient dJ/dtheta = dJ/dtheta|_f + lambda . dN/dtheta|_f with
 *        (dN/df)^T lambda = -(dJ/df)^T solved by restarted GMRES (restart
 *        length `restart`, at most 32) right-preconditioned by the transposed
 *        CS cycle (stage_cs_transposed; one transposed LU-SGS pass on a single
 *        grid), to relative residual tol or max_iter iterations.  In a
 *        domain bounded only by walls and symmetry planes the steady state is
 *        fixed up to its total mass M; the total mass is then held fixed (the
 *        transposed Jacobian gets the rank-one term -m m^T/|m|^2, m = dM/df).
 *        info (may be NULL) receives {J, iterations, final relative residual}.
 *        Returns MIUGKS_ENOTCONVERGED when tol was not reached (the gradient
 *        of the last iterate is still written).  Device work memory (restart+3
 *        vectors of 2 nc nv doubles, and six per level for the transposed cycle)
 *        comes from the solver's allocator on the first call and is kept. */
miugks_status miugks_stage_adjoint_residual(miugks_solver *s, const double *mu, double *out);
miugks_status miugks_stage_sgs_micro_transposed(miugks_solver *s, const double *inv_tau, const double *r, double *x);
/*  stage_cs_transposed: out = M^T z with M one CS cycle (Eq. CSCYC, the
 *        solver's levels and smoothing counts) as a linear map of the level-0
 *        residual, frozen collision frequencies inv_tau of every level
 *        concatenated level after level (sum of nc_l values).  The adjoint
 *        solve uses this transposed cycle as its preconditioner. */
miugks_status miugks_stage_cs_transposed(miugks_solver *s, const double *inv_tau, const double *z, double *out);
/*  stage_macro_jacobian_transposed: y = J^T x with J = dR_E/dW the Jacobian of
 *        the split Euler residual of the prediction step (Eqs. macroFluxSplitting,
 *        forcingFunction; wall ghosts by Eq. boundaryWall) on level 0 at the
 *        state W, Gamma frozen at W; W, x, y host arrays of nc x 4.  The
 *        adjoint's macroscopic correction solves with this operator. */
miugks_status miugks_stage_macro_jacobian_transposed(miugks_solver *s, const double *W, const double *x, double *y);
/* Adjoint preconditioner options: macro_correction != 0 (default) adds to the
 * transposed CS cycle the transpose of the prediction step's effect (the
 * linearised forward iteration, prediction included, transposed: an inner
 * Krylov solve with the transposed Jacobian of the split Euler residual;
 * the outer solve is then flexible GMRES); 0 uses the transposed CS cycle alone. */
miugks_status miugks_set_adjoint_options(miugks_solver *s, int macro_correction);
miugks_status miugks_objective(miugks_solver *s, int obj, int bc, double *J, double *dJdf, double dJdtheta[3]);
miugks_status miugks_adjoint(miugks_solver *s, int obj, int bc, int param, double tol, int max_iter, int restart,
                             double *grad, double info[3]);

/* Checkpoint and resume: save writes the state (f in FP64, the BC table and
 * the iteration count) to a file; load reads it into a solver created with the
 * same mesh size, velocity grid and BC types, replacing its f, BC values and
 * iteration count.  Errors: MIUGKS_EINVAL for an unreadable, truncated or
 * mismatching file; the solver is unchanged unless the file was valid. */
miugks_status miugks_save(miugks_solver *s, const char *path);
miugks_status miugks_load(miugks_solver *s, const char *path);

/* Sizes and the CUDA events bracketing the last Step-1 flux launch (for
 * roofline timing): elapsed milliseconds of the flux kernels of the last
 * iteration, or -1 when timing is off.  miugks_set_timing(s, 1) enables it. */
miugks_status miugks_sizes(const miugks_solver *s, int *nx, int *ny, int *nv, int *levels);
miugks_status miugks_set_timing(miugks_solver *s, int on);
miugks_status miugks_kernel_times(miugks_solver *s, double *flux_ms, double *sweep_ms, double *total_ms);
/* With timing on, every launch of the prediction smoother's LU-SGS kernel on
 * the finest level (Eq. macroFinalDefect, Sec. 2.1.1) is bracketed by its own
 * pair of CUDA events: total milliseconds and launch count since the last
 * call (-1 and 0 when timing is off); the counters are reset. */
miugks_status miugks_macro_sweep_times(miugks_solver *s, double *ms, int *launches);
/* With timing on, every launch of the evolution smoother's sweep kernels on the
 * finest level (Eq. microFinalDefect; see miugks_set_sweep_split) is bracketed
 * by CUDA events.  out[0..2]: total milliseconds, launches and cell-velocity
 * pairs swept by the wavefront kernel; out[3..5]: the same for the line-class
 * kernel; since the last call (then reset).  -1 ms when timing is off. */
miugks_status miugks_sweep_kernel_times(miugks_solver *s, double out[6]);

/* Residual norm of caller-owned device arrays without allocating anything.
 * The paper has no counterpart.  It serves callers that cannot allocate device
 * memory at the point where they need the convergence measure: host frameworks
 * that lend only their own pre-sized pools and forbid the CUDA allocator, and
 * latency-critical loops that must not enter any allocator.
 *   R_dev:     nc x 4 residuals (device, [cell][component]);
 *   W_dev:     nc x 4 conservative variables (device), used for a health count;
 *   solid_dev: nc bytes (device), nonzero for a cell inside a body, or NULL
 *              when there is no body; such cells are skipped;
 *   out_dev:   5 doubles (device): the root mean square of each residual
 *              component over the fluid cells (the norm miugks_residual
 *              reports), then the number of fluid cells with non-positive
 *              density or internal energy (or NaN);
 *   cuda_stream: cudaStream_t or NULL (legacy default stream).
 * The partial sums live in a fixed scratch array inside the library (one
 * __device__ array of 4096 rows of 6 doubles per GPU that loads it, kept until
 * process exit): nc is limited to 1,048,576 cells, and larger nc returns
 * MIUGKS_EINVAL without launching anything.  The first call on a device
 * resolves the scratch address with that device current and keeps it for the
 * life of the process (so no cudaDeviceReset in between); make that first call
 * before any stream capture.  Every call overwrites the rows it reads, so
 * nothing needs clearing, but all calls share the one array: calls whose
 * kernels overlap on the GPU race and must be serialised by the caller.
 * Asynchronous on cuda_stream; the error message of a failed call is returned
 * by miugks_last_error(NULL). */
miugks_status miugks_residual_rms_noalloc(const double *R_dev, const double *W_dev, const unsigned char *solid_dev,
                                          int nc, double *out_dev, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
