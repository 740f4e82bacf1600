// macro.cu -- prediction step of MIUGKS (arXiv 1704.03151, Secs. 2.1.1, 2.3,
// 2.4, 3.2): the Euler split flux (Eq. macroFluxSplitting) with the spectral
// radius Gamma (Eq. predictionSpectralRadius), the residual R_E used by the FAS
// forcing function and renewal (Eqs. forcingFunction, renewResiduals), the
// LU-SGS smoother of Eq. macroFinalDefect, and the grid-transfer kernels
// (Eqs. macroRestriction, microRestriction, prolongation).
//
// The LU-SGS sweep runs as an anti-diagonal wavefront inside one thread-block
// cluster: the cells of a diagonal are spread over the cluster's CTAs and a
// hardware cluster barrier separates consecutive diagonals, so the serial
// sweep order is kept without grid-wide synchronisation.
#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace miugks {

constexpr int kMacroCluster = 8;
constexpr int kMacroThreads = 128;

__device__ __forceinline__ void euler_flux(const double* W, int axis, double sgn, double T[4])
{
    double rho, U, V, lam;
    prim4(W, rho, U, V, lam);
    double p = rho / (2.0 * lam);
    double nx = axis == 0 ? sgn : 0.0, ny = axis == 1 ? sgn : 0.0;
    double Un = U * nx + V * ny;
    T[0] = rho * Un;
    T[1] = W[1] * Un + p * nx;
    T[2] = W[2] * Un + p * ny;
    T[3] = (W[3] + p) * Un;
}

// Euler flux along +e_axis: (m_a, m_x U_a + p d_xa, m_y U_a + p d_ya, (E + p) U_a),
// with p = 2 e_int / (K + 2)
__device__ __forceinline__ void euler_axis(const double* W, int axis, double T[4])
{
    double ir = rcp64(W[0]);
    double U = W[1] * ir, V = W[2] * ir;
    double p = (2.0 / (kKint + 2)) * (W[3] - 0.5 * (W[1] * U + W[2] * V));
    double Ua = axis == 0 ? U : V;
    T[0] = W[1 + axis];
    T[1] = W[1] * Ua + (axis == 0 ? p : 0.0);
    T[2] = W[2] * Ua + (axis == 1 ? p : 0.0);
    T[3] = (W[3] + p) * Ua;
}

// ghost state of a boundary face (Eqs. boundaryRelation, boundaryWall) and, when
// M != null, its Jacobian dB/dW (Eq. example_results, with the wall velocity
// in place of U_0, V_0)
__device__ void macro_ghost(const BcDev& b, int axis, const double* Wi, double Wg[4], double* M)
{
    if (b.type == BC_WALL) {
        double rho, U, V, lam;
        prim4(Wi, rho, U, V, lam);
        double lamw = 1.0 / b.t;
        double lamg = 2.0 * lamw - lam, Ug = 2.0 * b.u - U, Vg = 2.0 * b.v - V;
        Wg[0] = rho; Wg[1] = rho * Ug; Wg[2] = rho * Vg;
        Wg[3] = 0.5 * rho * (Ug * Ug + Vg * Vg) + (kKint + 2) * rho / (4.0 * lamg);
        if (M) {
            double Y = lam / (lam - 2.0 * lamw), K = kKint + 2.0;
            for (int q = 0; q < 16; ++q) M[q] = 0.0;
            M[0] = 1.0;
            M[4] = 2.0 * b.u; M[5] = -1.0;
            M[8] = 2.0 * b.v; M[10] = -1.0;
            M[12] = 2.0 * (b.u * b.u + b.v * b.v) - 0.5 * (U * U + V * V) * (1.0 + Y * Y) + K / (4.0 * lam) * (Y * Y - Y);
            M[13] = U - 2.0 * b.u + U * Y * Y;
            M[14] = V - 2.0 * b.v + V * Y * Y;
            M[15] = -Y * Y;
        }
    } else if (b.type == BC_SYMMETRY) {
        for (int m = 0; m < 4; ++m) Wg[m] = Wi[m];
        Wg[1 + axis] = -Wi[1 + axis];
        if (M) {
            for (int q = 0; q < 16; ++q) M[q] = 0.0;
            M[0] = M[5] = M[10] = M[15] = 1.0;
            M[5 * (1 + axis)] = -1.0;
        }
    } else if (b.type == BC_FARFIELD) {
        double lam = 1.0 / b.t;
        Wg[0] = b.rho; Wg[1] = b.rho * b.u; Wg[2] = b.rho * b.v;
        Wg[3] = 0.5 * b.rho * (b.u * b.u + b.v * b.v) + (kKint + 2) * b.rho / (4.0 * lam);
        if (M) for (int q = 0; q < 16; ++q) M[q] = 0.0;
    } else {
        for (int m = 0; m < 4; ++m) Wg[m] = Wi[m];
        if (M) {
            for (int q = 0; q < 16; ++q) M[q] = 0.0;
            M[0] = M[5] = M[10] = M[15] = 1.0;
        }
    }
}

__device__ __forceinline__ double gamma_of(const GasDev& g, const double* Wa, const double* Wb, int axis, double dist)
{
    double Wm[4], rho, U, V, lam;
    for (int m = 0; m < 4; ++m) Wm[m] = 0.5 * (Wa[m] + Wb[m]);
    prim4(Wm, rho, U, V, lam);
    double gam = (kKint + 4.0) / (kKint + 2.0);
    double as = sqrt(gam / (2.0 * lam));
    double nu = g.mu_ref * pow(1.0 / lam, g.omega) / rho;
    return fabs(axis == 0 ? U : V) + as + 2.0 * nu / dist;
}

__global__ void k_macro_gamma(MacroArgs a, const double* __restrict__ Wg, double* __restrict__ gx, double* __restrict__ gy)
{
    const LevelDev& L = a.L;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    int nx = L.nx, ny = L.ny;
    if (t < L.nfx) {
        int i = t % (nx + 1), j = t / (nx + 1);
        int bcid = L.fbx[t];
        if (bcid >= 0) {
            int c = j * nx + (i == 0 ? 0 : nx - 1);
            double G[4];
            macro_ghost(a.bc[bcid], 0, Wg + 4 * (size_t)c, G, nullptr);
            gx[t] = gamma_of(a.gas, Wg + 4 * (size_t)c, G, 0, L.dx[i == 0 ? 0 : nx - 1]);
        } else {
            int c = j * nx + i;
            gx[t] = gamma_of(a.gas, Wg + 4 * (size_t)c, Wg + 4 * (size_t)(c - 1), 0, L.xc[i] - L.xc[i - 1]);
        }
        return;
    }
    t -= L.nfx;
    if (t < L.nfy) {
        int i = t % nx, j = t / nx;
        int bcid = L.fby[t];
        if (bcid >= 0) {
            int c = (j == 0 ? 0 : ny - 1) * nx + i;
            double G[4];
            macro_ghost(a.bc[bcid], 1, Wg + 4 * (size_t)c, G, nullptr);
            gy[t] = gamma_of(a.gas, Wg + 4 * (size_t)c, G, 1, L.dy[j == 0 ? 0 : ny - 1]);
        } else {
            int c = j * nx + i;
            gy[t] = gamma_of(a.gas, Wg + 4 * (size_t)c, Wg + 4 * (size_t)(c - nx), 1, L.yc[j] - L.yc[j - 1]);
        }
    }
}

// 1 / ((1/2V) sum_faces S Gamma + 1/dt_n): the inverse diagonal of the smoother
__global__ void k_macro_idiag(MacroArgs a, const double* __restrict__ gx, const double* __restrict__ gy,
                              double* __restrict__ idiag)
{
    const LevelDev& L = a.L;
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= L.nc) return;
    int i = c % L.nx, j = c / L.nx;
    double sx = gx[j * (L.nx + 1) + i] + gx[j * (L.nx + 1) + i + 1];
    double sy = gy[j * L.nx + i] + gy[(j + 1) * L.nx + i];
    double V = L.dx[i] * L.dy[j];
    idiag[c] = 1.0 / ((L.dy[j] * sx + L.dx[i] * sy) / (2.0 * V) + a.dtn_inv);
}

cudaError_t launch_macro_gamma(const MacroArgs& a, const double* Wg, double* gx, double* gy, double* idiag,
                               cudaStream_t st)
{
    int n = a.L.nfx + a.L.nfy;
    k_macro_gamma<<<(n + 127) / 128, 128, 0, st>>>(a, Wg, gx, gy);
    k_macro_idiag<<<(a.L.nc + 127) / 128, 128, 0, st>>>(a, gx, gy, idiag);
    return cudaGetLastError();
}

// Euler fluxes of every cell along +x and +y, [nc][8]
__global__ void k_macro_prep(LevelDev L, const double* __restrict__ W, double* __restrict__ T)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= L.nc) return;
    euler_axis(W + 4 * (size_t)c, 0, T + 8 * (size_t)c);
    euler_axis(W + 4 * (size_t)c, 1, T + 8 * (size_t)c + 4);
}

// face f of cell (i, j): 0 west, 1 east, 2 south, 3 north
__device__ __forceinline__ void face_of(const LevelDev& L, int i, int j, int f, int& bcid, int& nb, double& gidx_dummy)
{
    (void)gidx_dummy;
    int nx = L.nx;
    int axis = f >> 1, up = f & 1;
    if (axis == 0) {
        bcid = L.fbx[j * (nx + 1) + i + up];
        nb = j * nx + i + (up ? 1 : -1);
    } else {
        bcid = L.fby[(j + up) * nx + i];
        nb = (j + (up ? 1 : -1)) * nx + i;
    }
}

__device__ __forceinline__ double face_gamma(const LevelDev& L, const double* gx, const double* gy, int i, int j, int f)
{
    int axis = f >> 1, up = f & 1;
    return axis == 0 ? gx[j * (L.nx + 1) + i + up] : gy[(j + up) * L.nx + i];
}

// R_E of one cell: -(1/V) sum_faces S F_split(W_i, W_j)
__device__ void macro_resid_cell(const MacroArgs& a, const double* W, const double* gx, const double* gy,
                                 int i, int j, double RE[4])
{
    const LevelDev& L = a.L;
    int c = j * L.nx + i;
    double V = L.dx[i] * L.dy[j], acc[4] = {0, 0, 0, 0};
    const double* Wi = W + 4 * (size_t)c;
    double Ti[4][4];
    #pragma unroll
    for (int f = 0; f < 4; ++f) {
        int axis = f >> 1, up = f & 1;
        double sgn = up ? 1.0 : -1.0, S = axis == 0 ? L.dy[j] : L.dx[i];
        int bcid, nb; double dum = 0;
        face_of(L, i, j, f, bcid, nb, dum);
        double G[4], Tj[4];
        const double* Wj;
        if (bcid >= 0) { macro_ghost(a.bc[bcid], axis, Wi, G, nullptr); Wj = G; }
        else Wj = W + 4 * (size_t)nb;
        euler_flux(Wi, axis, sgn, Ti[f]);
        euler_flux(Wj, axis, sgn, Tj);
        double gm = face_gamma(L, gx, gy, i, j, f);
        for (int m = 0; m < 4; ++m) acc[m] += S * (0.5 * (Ti[f][m] + Tj[m] + gm * (Wi[m] - Wj[m])));
    }
    for (int m = 0; m < 4; ++m) RE[m] = -acc[m] / V;
}

__global__ void k_macro_resid(MacroArgs a, const double* __restrict__ W, const double* __restrict__ gx,
                              const double* __restrict__ gy, const double* __restrict__ Rin, double* __restrict__ out,
                              int mode)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.L.nc) return;
    double RE[4];
    macro_resid_cell(a, W, gx, gy, c % a.L.nx, c / a.L.nx, RE);
    for (int m = 0; m < 4; ++m)
        out[4 * (size_t)c + m] = mode == 0 ? Rin[4 * (size_t)c + m] - RE[m] : Rin[4 * (size_t)c + m] + RE[m];
}

cudaError_t launch_macro_resid(const MacroArgs& a, const double* W, const double* gx, const double* gy,
                               const double* Rin, double* out, int mode, cudaStream_t st)
{
    k_macro_resid<<<(a.L.nc + 127) / 128, 128, 0, st>>>(a, W, gx, gy, Rin, out, mode);
    return cudaGetLastError();
}

// LU-SGS pass of Eq. macroFinalDefect, one lane per (cell, component).
//
// On GB300 an FP64 warp instruction occupies its SM sub-partition for 64 cycles
// however many lanes are active, so the sweep minimises FP64 instructions per
// lane rather than lanes: each lane updates one component of one cell of the
// current diagonal (about eight FP64 instructions), and the four lanes of a
// cell then evaluate the Euler fluxes of the new state W + dW along x and y,
// which the cell's successors on the next diagonal need.  Boundary ghosts
// enter only the backward sweep (they use dW_i of the forward sweep), so their
// contribution is computed for all boundary cells in parallel between the two
// half sweeps.  Arrays: T0 = T(W) [nc][8] (from k_macro_prep), T1 = T(W + dW)
// [nc][8], G = upper-side ghost terms [nc][4].

// Euler flux component m of W along +e_axis, given 1/rho, U_a and p
__device__ __forceinline__ double euler_comp(const double* W, int m, int axis, double Ua, double p)
{
    if (m == 0) return W[1 + axis];
    if (m == 3) return (W[3] + p) * Ua;
    double v = W[m] * Ua;
    return (m == 1 + axis) ? v + p : v;
}

__device__ __forceinline__ void producer_fluxes(const double wp, int m, int g0, double* T1c)
{
    // gather the four components of W + dW of this cell (lanes g0..g0+3)
    double Wp[4];
    #pragma unroll
    for (int q = 0; q < 4; ++q) Wp[q] = __shfl_sync(0xffffffffu, wp, g0 + q);
    double ir = rcp64(Wp[0]);
    double U = Wp[1] * ir, V = Wp[2] * ir;
    double p = (2.0 / (kKint + 2)) * fma(-0.5, fma(Wp[2], V, Wp[1] * U), Wp[3]);
    T1c[m] = euler_comp(Wp, m, 0, U, p);
    T1c[4 + m] = euler_comp(Wp, m, 1, V, p);
}

// ghost term of the upper-side boundary faces of cell (i, j) for the backward sweep
__device__ void macro_ghost_terms(const MacroArgs& a, const double* W, const double* gx, const double* gy,
                                  const double* dW, int i, int j, double Gc[4])
{
    const LevelDev& L = a.L;
    const int c = j * L.nx + i;
    for (int m = 0; m < 4; ++m) Gc[m] = 0.0;
    for (int axis = 0; axis < 2; ++axis) {
        int bcid = axis == 0 ? (i == L.nx - 1 ? L.fbx[j * (L.nx + 1) + L.nx] : -1)
                             : (j == L.ny - 1 ? L.fby[L.ny * L.nx + i] : -1);
        if (bcid < 0) continue;
        double Wn[4], dWn[4], Wp[4], T1[4], T0[4], M[16];
        macro_ghost(a.bc[bcid], axis, W + 4 * (size_t)c, Wn, M);
        for (int m = 0; m < 4; ++m) {
            double s2 = 0.0;
            for (int q = 0; q < 4; ++q) s2 += M[4 * m + q] * dW[4 * (size_t)c + q];
            dWn[m] = s2;
            Wp[m] = Wn[m] + dWn[m];
        }
        euler_axis(Wp, axis, T1);
        euler_axis(Wn, axis, T0);
        double S = axis == 0 ? L.dy[j] : L.dx[i];
        double gm = axis == 0 ? gx[j * (L.nx + 1) + i + 1] : gy[(j + 1) * L.nx + i];
        for (int m = 0; m < 4; ++m) Gc[m] += S * ((T1[m] - T0[m]) - gm * dWn[m]);
    }
}

// inputs of one lane for one diagonal that do not depend on the previous diagonal
struct MacroLane {
    int c, nb[2];
    bool on, inter[2];
    double gm[2], S[2], T0[2], own, id, hv, W, G;
};

__global__ void __cluster_dims__(kMacroCluster, 1, 1) __launch_bounds__(kMacroThreads)
k_macro_sgs(MacroArgs a, double* __restrict__ W, const double* __restrict__ T0, double* __restrict__ T1,
            double* __restrict__ Gt, const double* __restrict__ gx, const double* __restrict__ gy,
            const double* __restrict__ idiag, const double* __restrict__ R, double* __restrict__ dW)
{
    cg::cluster_group cl = cg::this_cluster();
    const LevelDev& L = a.L;
    const int nx = L.nx, ny = L.ny, nd = nx + ny - 1;
    const int t = cl.block_rank() * blockDim.x + threadIdx.x;
    const int m = t & 3, g0 = threadIdx.x & 28;        // component; first lane of the cell's group
    const int slot = t >> 2;                            // one cell of a diagonal per four lanes
    auto prepare = [&](int pass, int d, MacroLane& p) {
        int ilo = d - (ny - 1) > 0 ? d - (ny - 1) : 0, ihi = d < nx - 1 ? d : nx - 1;
        p.on = slot <= ihi - ilo;
        if (!p.on) return;
        int i = ilo + slot, j = d - i, c = j * nx + i;
        p.c = c;
        #pragma unroll
        for (int axis = 0; axis < 2; ++axis) {
            int fidx = axis == 0 ? j * (nx + 1) + i + pass : (j + pass) * nx + i;
            p.inter[axis] = (axis == 0 ? L.fbx[fidx] : L.fby[fidx]) < 0;
            p.nb[axis] = axis == 0 ? c + (pass ? 1 : -1) : c + (pass ? nx : -nx);
            p.gm[axis] = axis == 0 ? gx[fidx] : gy[fidx];
            p.S[axis] = axis == 0 ? L.dy[j] : L.dx[i];
            p.T0[axis] = p.inter[axis] ? T0[8 * (size_t)p.nb[axis] + 4 * axis + m] : 0.0;
        }
        p.own = pass == 0 ? R[4 * (size_t)c + m] : dW[4 * (size_t)c + m];
        p.id = idiag[c];
        p.hv = 0.5 * L.rdx[i] * L.rdy[j];
        p.W = W[4 * (size_t)c + m];
        p.G = (pass == 1 && (i == nx - 1 || j == ny - 1)) ? Gt[4 * (size_t)c + m] : 0.0;
    };
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            // upper-side ghost terms of the last column and row, from the forward dW (one thread per cell)
            for (int b = t; b < nx + ny - 1; b += kMacroCluster * blockDim.x) {
                int i = b < ny ? nx - 1 : b - ny, j = b < ny ? b : ny - 1;
                macro_ghost_terms(a, W, gx, gy, dW, i, j, Gt + 4 * (size_t)(j * nx + i));
            }
            cl.sync();
        }
        const double sgn = pass ? 1.0 : -1.0;
        MacroLane cur, nxt;
        prepare(pass, pass == 0 ? 0 : nd - 1, cur);
        for (int d0 = 0; d0 < nd; ++d0) {
            double wp = 0.0;
            if (cur.on) {
                double acc = cur.G;
                #pragma unroll
                for (int axis = 0; axis < 2; ++axis) {
                    if (!cur.inter[axis]) continue;
                    const size_t nb = cur.nb[axis];
                    double dT = T1[8 * nb + 4 * axis + m] - cur.T0[axis];
                    acc = fma(cur.S[axis], fma(-cur.gm[axis], dW[4 * nb + m], sgn * dT), acc);
                }
                double dw = pass == 0 ? fma(-acc, cur.hv, cur.own) * cur.id : fma(-acc * cur.hv, cur.id, cur.own);
                dW[4 * (size_t)cur.c + m] = dw;
                wp = cur.W + dw;
            }
            double T1c[8];
            producer_fluxes(wp, m, g0, T1c);
            if (cur.on) {
                T1[8 * (size_t)cur.c + m] = T1c[m];
                T1[8 * (size_t)cur.c + 4 + m] = T1c[4 + m];
            }
            if (d0 + 1 < nd) prepare(pass, pass == 0 ? d0 + 1 : nd - 2 - d0, nxt);
            cl.sync();   // release/acquire at cluster scope: the diagonal is visible to the next one
            cur = nxt;
        }
    }
    for (int c = t; c < 4 * L.nc; c += kMacroCluster * blockDim.x) W[c] += dW[c];
}

cudaError_t launch_macro_sgs(const MacroArgs& a, double* W, const double* gx, const double* gy, const double* idiag,
                             double* T, const double* R, double* dW, cudaStream_t st)
{
    // T: [nc][8] T(W), then [nc][8] T(W + dW), then [nc][4] ghost terms
    double* T0 = T;
    double* T1 = T + 8 * (size_t)a.L.nc;
    double* Gt = T + 16 * (size_t)a.L.nc;
    // one cell of a diagonal per four lanes of the cluster
    const int maxdiag = a.L.nx < a.L.ny ? a.L.nx : a.L.ny;
    if (4 * maxdiag > kMacroCluster * kMacroThreads) return cudaErrorInvalidValue;
    k_macro_prep<<<(a.L.nc + 127) / 128, 128, 0, st>>>(a.L, W, T0);
    k_macro_sgs<<<kMacroCluster, kMacroThreads, 0, st>>>(a, W, T0, T1, Gt, gx, gy, idiag, R, dW);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// volume-weighted restriction (nblk blocks of [nc][m])
template <typename T>
__global__ void k_restrict(LevelDev F, LevelDev C, int m, int nblk, const T* __restrict__ fine,
                           T* __restrict__ coarse)
{
    size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    size_t per = (size_t)C.nc * m;
    if (t >= per * nblk) return;
    int blk = (int)(t / per);
    size_t rem = t - blk * per;
    int cc = (int)(rem / m), q = (int)(rem - (size_t)cc * m);
    int I = cc % C.nx, J = cc / C.nx;
    const T* fb = fine + (size_t)blk * F.nc * m;
    double s = 0.0, vs = 0.0;
    #pragma unroll
    for (int b = 0; b < 2; ++b)
        #pragma unroll
        for (int a2 = 0; a2 < 2; ++a2) {
            int i = 2 * I + a2, j = 2 * J + b;
            double V = F.dx[i] * F.dy[j];
            s += (double)fb[(size_t)(j * F.nx + i) * m + q] * V;
            vs += V;
        }
    coarse[(size_t)blk * per + rem] = (T)(s / vs);
}

template <typename T>
cudaError_t launch_restrict(const LevelDev& F, const LevelDev& C, int m, int nblk, const T* fine, T* coarse,
                            cudaStream_t st)
{
    size_t n = (size_t)C.nc * m * nblk;
    k_restrict<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(F, C, m, nblk, fine, coarse);
    return cudaGetLastError();
}
template cudaError_t launch_restrict<double>(const LevelDev&, const LevelDev&, int, int, const double*, double*,
                                             cudaStream_t);
template cudaError_t launch_restrict<float>(const LevelDev&, const LevelDev&, int, int, const float*, float*,
                                            cudaStream_t);

template <typename T>
__global__ void k_prolong_add(LevelDev F, LevelDev C, int m, int nblk, const int* __restrict__ idx4,
                              const double* __restrict__ w4, const T* __restrict__ coarse,
                              T* __restrict__ fine, T* __restrict__ out_pro)
{
    size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    size_t per = (size_t)F.nc * m;
    if (t >= per * nblk) return;
    int blk = (int)(t / per);
    size_t rem = t - blk * per;
    int c = (int)(rem / m), q = (int)(rem - (size_t)c * m);
    const T* cb = coarse + (size_t)blk * C.nc * m;
    double v = 0.0;
    #pragma unroll
    for (int s = 0; s < 4; ++s) v += w4[4 * c + s] * (double)cb[(size_t)idx4[4 * c + s] * m + q];
    fine[t] = (T)((double)fine[t] + v);
    if (out_pro) out_pro[t] = (T)v;
}

template <typename T>
cudaError_t launch_prolong_add(const LevelDev& F, const LevelDev& C, int m, int nblk, const int* idx4,
                               const double* w4, const T* coarse, T* fine, T* out_pro, cudaStream_t st)
{
    size_t n = (size_t)F.nc * m * nblk;
    k_prolong_add<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(F, C, m, nblk, idx4, w4, coarse, fine, out_pro);
    return cudaGetLastError();
}
template cudaError_t launch_prolong_add<double>(const LevelDev&, const LevelDev&, int, int, const int*,
                                                const double*, const double*, double*, double*, cudaStream_t);
template cudaError_t launch_prolong_add<float>(const LevelDev&, const LevelDev&, int, int, const int*,
                                               const double*, const float*, float*, float*, cudaStream_t);

__global__ void k_axpy(double* __restrict__ y, const double* __restrict__ x, double a, size_t n)
{
    size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t < n) y[t] += a * x[t];
}
__global__ void k_sub(double* __restrict__ out, const double* __restrict__ a, const double* __restrict__ b, size_t n)
{
    size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t < n) out[t] = a[t] - b[t];
}
cudaError_t launch_axpy(double* y, const double* x, double a, size_t n, cudaStream_t st)
{
    k_axpy<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(y, x, a, n);
    return cudaGetLastError();
}
cudaError_t launch_sub(double* out, const double* a, const double* b, size_t n, cudaStream_t st)
{
    k_sub<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, a, b, n);
    return cudaGetLastError();
}

} // namespace miugks
