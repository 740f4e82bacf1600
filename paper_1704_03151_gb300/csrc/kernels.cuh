// kernels.cuh -- argument structs and launchers of the MIUGKS kernels.
#pragma once
#include "common.cuh"
#include <vector>

namespace miugks {

template <typename F>
struct FaceFluxArgs {
    LevelDev L; VelDev V; GasDev gas;
    const BcDev* bc; const double* Cw;     // Cw[b * nv + k]: unit-density Maxwellian of BC b
    const F* f;                            // [2][nc][nv]
    const double* W;                       // [nc][4]
    F* ph;                                 // [2][nf][nv] time-averaged micro flux, along +axis
    double* Fm;                            // [nf][4] macro flux
    int axis; double cfl;
    int shock;                             // add the pressure-jump term to the interface collision time
    const double* geo;                     // [nf][kFluxGeo] constants of each interior face of this axis
};
// Per interior face: 1/(x_{i-1} - x_{i-2}), 1/(x_i - x_{i-1}), 1/(x_{i+1} - x_i)
// (1 where the outer cell does not exist), the face-to-centre distances h_L,
// h_R, the time step dt = CFL min(dx_L, dx_R) / max|u|, 1/dt, 1/h_L, 1/h_R.
// They depend only on the mesh, so they are computed once on the host.
constexpr int kFluxGeo = 10;

void upload_series_coefficients();
template <typename F> cudaError_t launch_face_flux(const FaceFluxArgs<F>& a, cudaStream_t st);
cudaError_t launch_cell_residual(const LevelDev& L, const double* Fx, const double* Fy, double* R, cudaStream_t st);
cudaError_t launch_rms(const double* R, const double* W, int nc, int nfluid, double* part, double* out, cudaStream_t st);

// ---- prediction step (macroscopic state in FP64) ----
struct MacroArgs {
    LevelDev L; GasDev gas; const BcDev* bc;
    double dtn_inv;                        // 1/dt_n (0 when off)
    double* flag;                          // set to 1 when a bounded device wait gave up
    unsigned long long wait_ns;            // bound of the sweep's waits for its inputs (ns of global time)
};
// Gamma of every face from the frozen state Wg
// (and the inverse diagonal of the smoother per cell)
cudaError_t launch_macro_gamma(const MacroArgs& a, const double* Wg, double* gx, double* gy, double* idiag,
                               cudaStream_t st);
// mode 0: out = Rin - R_E(W)  (forcing);  mode 1: out = Rin + R_E(W)  (renewal P + R_E)
cudaError_t launch_macro_resid(const MacroArgs& a, const double* W, const double* gx, const double* gy,
                               const double* Rin, double* out, int mode, cudaStream_t st);
// y = J^T x, J = dR_E/dW at W with Gamma frozen (gx, gy); x may be null (no product);
// binv (16 per cell, may be null) receives the inverses of the transposed diagonal blocks
cudaError_t launch_macro_jacT(const MacroArgs& a, const double* W, const double* gx, const double* gy,
                              const double* x, double* y, double* binv, cudaStream_t st);
// one LU-SGS pass: dW from R at state W; then W += dW.  F: arithmetic of the sweep
// (double, or float with increments); rec: macro_rec_bytes(nx, ny, F == float) of scratch
template <typename F>
cudaError_t launch_macro_sgs(const MacroArgs& a, double* W, const double* gx, const double* gy, const double* idiag,
                             void* rec, const double* R, double* dW, cudaStream_t st);
size_t macro_rec_bytes(int nx, int ny, bool mixed);
template <typename T>
cudaError_t launch_restrict(const LevelDev& F, const LevelDev& C, int m, int nblk, const T* fine, T* coarse,
                            cudaStream_t st);
// fine += prolong(coarse) (m components per cell, nblk blocks of [nc][m]); also writes the
// prolongated values into out_pro when it is not null
// idx4/w4: per fine cell the four coarse stencil cells and their bilinear weights
template <typename T>
cudaError_t launch_prolong_add(const LevelDev& F, const LevelDev& C, int m, int nblk, const int* idx4,
                               const double* w4, const T* coarse, T* fine, T* out_pro, cudaStream_t st);
cudaError_t launch_axpy(double* y, const double* x, double a, size_t n, cudaStream_t st);
// Wt = Wc, or Wn in a cell where Wc has non-positive density or internal energy
cudaError_t launch_predicted_state(int nc, const double* Wn, const double* Wc, double* Wt, cudaStream_t st);
// FAS correction W += P dWc of the [nc][4] state, dropped in a cell where it would
// leave the density or the internal energy non-positive
cudaError_t launch_prolong_state(const LevelDev& F, const int* idx4, const double* w4, const double* dWc, double* W,
                                 cudaStream_t st);
cudaError_t launch_sub(double* out, const double* a, const double* b, size_t n, cudaStream_t st);

// ---- evolution step (microscopic) ----
// The sweep order of one level (device tables, per pass 0 forward / 1 backward).
// A boundary-line cell is a fluid cell with a boundary face on the sweep side:
// the domain edge's column and row (a corner cell first), and the lines along
// bodies.  Each such cell has a fold entry e (its ghost-folded inputs).
struct SweepPlanDev {
    const int* code[2];     // per cell: -1 ordinary, -2 in a body, else e << 2 | x-face line << 1 | y-face line
    const int4* lcell[2];   // per fold entry: {cell, line axis (0 x-face, 1 y-face), wall-density slot, final}
    const int* lines[2];    // lines along bodies: [q][8] = {i0, j0, di, dj, len, line axis, density slot, 0}
    int nl[2];              // fold entries of the edge lines (the rest belong to body lines)
    int nl_max;             // fold-entry stride of the layout
    int bodies;             // the level has solid cells
};
constexpr int kMaxBodyLines = 64;   // lines along bodies per pass and level
struct MicroArgs {
    LevelDev L; VelDev V; const BcDev* bc; const double* Cw;
    const double* inv_tau;                 // [nc] collision frequency (+ 1/dt_n)
    SweepPlanDev P;
};
// Host schedule of the body lines of one pass: after wave step dd - 1, the lines
// q0 .. q0 + nq - 1 (fold entries e0 .. e0 + ne - 1) are walked and folded.
struct SweepBreak { int dd, q0, nq, e0, ne; };
// Timing mode: event pairs around the launches of the wavefront and line-class
// sweep kernels, with the cell-velocity pairs each launch sweeps.
struct SweepTimer {
    std::vector<cudaEvent_t> ev;  // two per launch
    std::vector<int> kind;        // 0 wavefront, 1 line class
    std::vector<double> units;
    int used = 0;
};
// split: 0 by the level's size, 1 always split the velocities by coupling class, 2 never;
// timer: null unless the launches are to be timed
struct SweepPlanHost { const SweepBreak* brk[2]; int nbrk[2]; int split; SweepTimer* timer; };
// Step 3-4: r = (g~ - f)/tau~ - div(ph) on level 0; also inv_tau (with dtn_inv) and invD
template <typename F>
cudaError_t launch_micro_residual(const MicroArgs& m, GasDev gas, const double* Wt, const double* q,
                                  const F* f, const F* phx, const F* phy, double dtn_inv,
                                  double* inv_tau, F* invD, F* r, cudaStream_t st);
// inv_tau and invD of a coarse level from its restricted predicted state
template <typename F>
cudaError_t launch_coarse_coeffs(const MicroArgs& m, GasDev gas, const double* Wt, double dtn_inv,
                                 double* inv_tau, F* invD, cudaStream_t st);
// one symmetric Gauss-Seidel pass: x = SGS(r).  Zw[b*4 + axis*2 + (outsign>0)] = sum over the
// incoming velocities of w u_n C_k of wall BC b; xcorner: scratch of
// micro_scratch_elems(nv, nl_max, body lines) values (the largest over the levels)
size_t micro_scratch_elems(int nv, int nl, int nlines);
// *out = sum of a[q]^2 over n values; part: scratch of 128 doubles
template <typename T>
cudaError_t launch_sumsq(const T* a, size_t n, double* part, double* out, cudaStream_t st);
// coupling classes of the evolution sweep for one pass (VelDev::wblk, lk, nrow, ncol, nelem)
void sweep_classes(const double* u, const double* v, int nv, int pass, std::vector<int>& wblk, std::vector<int>& lk,
                   int& nrow, int& ncol, int& nelem);
template <typename F>
cudaError_t launch_micro_sgs(const MicroArgs& m, const SweepPlanHost& plan, const double* Zw, const F* invD,
                             const F* r, F* x, F* xcorner, cudaStream_t st);
// r -= A x (when renew) and acc += x (when acc != null)
template <typename F>
cudaError_t launch_micro_renew(const MicroArgs& m, const double* Zw, const F* x, F* r, F* acc, int renew,
                               cudaStream_t st);
// Steps 6-7: f += df; W, q from moments
template <typename F>
cudaError_t launch_update_moments(const LevelDev& L, const VelDev& V, F* f, const F* df, double* W, double* q,
                                  cudaStream_t st);
template <typename F>
cudaError_t launch_moments(const LevelDev& L, const VelDev& V, const F* f, double* W, double* q, cudaStream_t st);
// full-multigrid start-up: cells whose prolonged f is unphysical take their coarse cell's f
template <typename F>
cudaError_t launch_state_fallback(const LevelDev& L, const VelDev& V, int ncx, size_t ncc, const F* fc, F* f,
                                  cudaStream_t st);
template <typename F>
cudaError_t launch_init_maxwell(const LevelDev& L, const VelDev& V, const double* prim, F* f, cudaStream_t st);
// per wall face p, tau, q (one block per face of BC bc, in face order)
template <typename F>
cudaError_t launch_wall_quantities(const LevelDev& L, const VelDev& V, const BcDev* bc, const double* Cw,
                                   const F* f, int bcid, const int* faces, int nfaces, double* out,
                                   cudaStream_t st);

// ---- differentiation form: adjoint of the steady equations (FP64) ----
constexpr int kFaceRec = 28;              // doubles per face record of the adjoint residual
constexpr int kCellRec = 9;               // doubles per cell record
constexpr int kMaxAdjNv = 12288;          // velocities per cell of the transposed sweep (2 x 8 B each in shared memory)
struct AdjDev {
    LevelDev L; VelDev V; GasDev gas;
    const BcDev* bc; const double* Cw;
    const double* f;                       // [2][nc][nv] linearisation point (FP64 copy of f)
    const double* W;                       // [nc][4] its moments
    const double* q;                       // [nc][2] its heat flux
    double cfl;
};
struct AdjSweepArgs {
    LevelDev L; VelDev V; const BcDev* bc; const double* Cw; const double* Zw;
    const double* inv_tau;                 // [nc]
    const double* invD;                    // [nc][nv] 1 / (1/tau + |u|/dx + |v|/dy)
    const double* r;                       // [2][nc][nv] right-hand side
    double* y;                             // [2][nc][nv] result of the ascending pass
    double* x;                             // [2][nc][nv] result
};
// out = (dN/df)^T mu (+ pen * dM/df, M the total mass); rec*: per-face / per-cell scratch
cudaError_t launch_adjoint_residual(const AdjDev& A, const double* mu, double* recx, double* recy, double* crec,
                                    double pen, double* out, cudaStream_t st);
// Cells of a level with one wall face of a body on a transposed pass's side
// (pass 0 east or north, pass 1 west or south), grouped by the wavefront step
// of the transposed sweep that reaches them.  The sweep stops after each such
// step and adds the within-cell wall coupling of those cells (the outgoing
// rows take the transposed reflection of the incoming ones) before it goes on.
struct AdjBodyPlan {
    const int* cells[2];      // device, per pass: entries cell * 4 + face (0 west, 1 east, 2 south, 3 north)
    const int* step[2];       // host, per pass: the wavefront step of each group, ascending
    const int* off[2];        // host, per pass: first entry of group g is off[g], its end off[g + 1]
    int ngroups[2];
};
// x = P^T r, P one LU-SGS pass of the evolution smoother of the level
cudaError_t launch_adjoint_sgs(const AdjSweepArgs& S, const AdjBodyPlan& P, cudaStream_t st);
// y = A^T x with the evolution operator of one level (all neighbours and ghosts)
cudaError_t launch_adjoint_apply(const AdjSweepArgs& S, const double* x, double* y, cudaStream_t st);
// fine = R^T coarse (volume-weighted restriction transposed), coarse = P^T fine (bilinear
// prolongation transposed, inverse stencil in CSR form); 2 x nv values per cell
cudaError_t launch_adjoint_restrict_t(const LevelDev& F, const LevelDev& C, int nv, const double* coarse,
                                      double* fine, cudaStream_t st);
cudaError_t launch_adjoint_prolong_t(const LevelDev& F, const LevelDev& C, int nv, const int* ptr, const int* cell,
                                     const double* wgt, const double* fine, double* coarse, cudaStream_t st);
// per wall face: part[4 m ..] = (S Q, S dQ/dT, S dQ/du, S dQ/dv); dJdf += dJ/df (may be null)
cudaError_t launch_adjoint_objective(const AdjDev& A, int obj, int bcid, const int* faces, int nfaces, double* part,
                                     double* dJdf, cudaStream_t st);
// per wall face: part[3 m + p] = lambda . dN/dtheta_p
cudaError_t launch_adjoint_dtheta(const AdjDev& A, int bcid, const int* faces, int nfaces, const double* lam,
                                  double* part, cudaStream_t st);
cudaError_t launch_multi_dot(const double* Vb, int m, size_t n, const double* w, double* part, int nblk,
                             cudaStream_t st);
cudaError_t launch_multi_axpy(const double* Vb, int m, size_t n, const double* h, double a, double* w,
                              cudaStream_t st);
cudaError_t launch_mass_dot(const LevelDev& L, const VelDev& V, const double* x, double* part, cudaStream_t st);
template <typename F> cudaError_t launch_to_double(const F* a, double* b, size_t n, cudaStream_t st);
cudaError_t launch_to_float(const double* a, float* b, size_t n, cudaStream_t st);
// zero the entries of cells in bodies of a 2 x nc x nv vector
cudaError_t launch_zero_solid(const LevelDev& L, int nv, double* x, cudaStream_t st);
cudaError_t launch_inv_tau(const GasDev& gas, const double* W, int nc, double* it, cudaStream_t st);
cudaError_t launch_adjoint_invD(const LevelDev& L, const VelDev& V, const double* it, double* invD, cudaStream_t st);
// m_c = (dr_c/dW~_c)^T y_c (micro residual w.r.t. the predicted state, heat flux held)
cudaError_t launch_adjoint_macro_m(const AdjDev& A, const double* y, double* m, cudaStream_t st);
// out -= Pi^T w (moment weights times the cell 4-vectors)
cudaError_t launch_adjoint_macro_spread(const LevelDev& L, const VelDev& V, const double* w, double* out,
                                        cudaStream_t st);
cudaError_t launch_block_apply(int nc, const double* binv, const double* r, double* z, cudaStream_t st);
// closed domains: partial sums of sum_c V_c w_c[0], and w_c[0] -= coef V_c
cudaError_t launch_macro_null_dot(const LevelDev& L, const double* w, double* part, int nblk, cudaStream_t st);
cudaError_t launch_macro_null_sub(const LevelDev& L, double coef, double* w, cudaStream_t st);

} // namespace miugks
