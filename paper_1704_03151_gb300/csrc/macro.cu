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

cudaError_t launch_macro_gamma(const MacroArgs& a, const double* Wg, double* gx, double* gy, cudaStream_t st)
{
    int n = a.L.nfx + a.L.nfy;
    k_macro_gamma<<<(n + 127) / 128, 128, 0, st>>>(a, Wg, gx, gy);
    return cudaGetLastError();
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

// one cell of the LU-SGS pass (pass 0 forward with west/south, pass 1 backward with east/north)
__device__ void macro_sgs_cell(const MacroArgs& a, const double* W, const double* gx, const double* gy,
                               const double* R, double* dW, int i, int j, int pass)
{
    const LevelDev& L = a.L;
    int c = j * L.nx + i;
    double V = L.dx[i] * L.dy[j];
    double diag = 0.0;
    #pragma unroll
    for (int f = 0; f < 4; ++f) diag += ((f >> 1) == 0 ? L.dy[j] : L.dx[i]) * face_gamma(L, gx, gy, i, j, f);
    diag = diag / (2.0 * V) + a.dtn_inv;
    double acc[4] = {0, 0, 0, 0};
    const double* Wi = W + 4 * (size_t)c;
    for (int f = pass; f < 4; f += 2) {
        int axis = f >> 1;
        double sgn = pass ? 1.0 : -1.0, S = axis == 0 ? L.dy[j] : L.dx[i];
        int bcid, nb; double dum = 0;
        face_of(L, i, j, f, bcid, nb, dum);
        double Wn[4], dWn[4], Wp[4], T1[4], T0[4];
        if (bcid >= 0) {
            double M[16];
            macro_ghost(a.bc[bcid], axis, Wi, Wn, M);
            for (int m = 0; m < 4; ++m) {
                double s = 0.0;
                if (pass == 1)
                    for (int q = 0; q < 4; ++q) s += M[4 * m + q] * dW[4 * (size_t)c + q];
                dWn[m] = s;
            }
        } else {
            for (int m = 0; m < 4; ++m) { Wn[m] = W[4 * (size_t)nb + m]; dWn[m] = dW[4 * (size_t)nb + m]; }
        }
        for (int m = 0; m < 4; ++m) Wp[m] = Wn[m] + dWn[m];
        euler_flux(Wp, axis, sgn, T1);
        euler_flux(Wn, axis, sgn, T0);
        double gm = face_gamma(L, gx, gy, i, j, f);
        for (int m = 0; m < 4; ++m) acc[m] += S * ((T1[m] - T0[m]) - gm * dWn[m]);
    }
    if (pass == 0)
        for (int m = 0; m < 4; ++m) dW[4 * (size_t)c + m] = (R[4 * (size_t)c + m] - acc[m] / (2.0 * V)) / diag;
    else
        for (int m = 0; m < 4; ++m) dW[4 * (size_t)c + m] = dW[4 * (size_t)c + m] - acc[m] / (2.0 * V * diag);
}

__global__ void __cluster_dims__(kMacroCluster, 1, 1) __launch_bounds__(kMacroThreads)
k_macro_sgs(MacroArgs a, double* __restrict__ W, const double* __restrict__ gx, const double* __restrict__ gy,
            const double* __restrict__ R, double* __restrict__ dW)
{
    cg::cluster_group cl = cg::this_cluster();
    const LevelDev& L = a.L;
    const int nx = L.nx, ny = L.ny, nd = nx + ny - 1;
    const int g = cl.block_rank() * blockDim.x + threadIdx.x, G = kMacroCluster * blockDim.x;
    for (int pass = 0; pass < 2; ++pass) {
        for (int d0 = 0; d0 < nd; ++d0) {
            int d = pass == 0 ? d0 : nd - 1 - d0;
            int ilo = d - (ny - 1) > 0 ? d - (ny - 1) : 0, ihi = d < nx - 1 ? d : nx - 1;
            for (int t = g; t <= ihi - ilo; t += G) {
                int i = ilo + t;
                macro_sgs_cell(a, W, gx, gy, R, dW, i, d - i, pass);
            }
            cl.sync();   // release/acquire at cluster scope: the diagonal is visible to the next one
        }
    }
    for (int c = g; c < L.nc; c += G)
        for (int m = 0; m < 4; ++m) W[4 * (size_t)c + m] += dW[4 * (size_t)c + m];
}

cudaError_t launch_macro_sgs(const MacroArgs& a, double* W, const double* gx, const double* gy, const double* R,
                             double* dW, int* err, cudaStream_t st)
{
    (void)err;
    k_macro_sgs<<<kMacroCluster, kMacroThreads, 0, st>>>(a, W, gx, gy, R, dW);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// volume-weighted restriction (nblk blocks of [nc][m])
__global__ void k_restrict(LevelDev F, LevelDev C, int m, int nblk, const double* __restrict__ fine,
                           double* __restrict__ coarse)
{
    size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    size_t per = (size_t)C.nc * m;
    if (t >= per * nblk) return;
    int blk = (int)(t / per);
    size_t rem = t - blk * per;
    int cc = (int)(rem / m), q = (int)(rem - (size_t)cc * m);
    int I = cc % C.nx, J = cc / C.nx;
    const double* fb = fine + (size_t)blk * F.nc * m;
    double s = 0.0, vs = 0.0;
    #pragma unroll
    for (int b = 0; b < 2; ++b)
        #pragma unroll
        for (int a2 = 0; a2 < 2; ++a2) {
            int i = 2 * I + a2, j = 2 * J + b;
            double V = F.dx[i] * F.dy[j];
            s += fb[(size_t)(j * F.nx + i) * m + q] * V;
            vs += V;
        }
    coarse[(size_t)blk * per + rem] = s / vs;
}

cudaError_t launch_restrict(const LevelDev& F, const LevelDev& C, int m, int nblk, const double* fine, double* coarse,
                            cudaStream_t st)
{
    size_t n = (size_t)C.nc * m * nblk;
    k_restrict<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(F, C, m, nblk, fine, coarse);
    return cudaGetLastError();
}

__global__ void k_prolong_add(LevelDev F, LevelDev C, int m, int nblk, const int* __restrict__ idx4,
                              const double* __restrict__ w4, const double* __restrict__ coarse,
                              double* __restrict__ fine, double* __restrict__ out_pro)
{
    size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    size_t per = (size_t)F.nc * m;
    if (t >= per * nblk) return;
    int blk = (int)(t / per);
    size_t rem = t - blk * per;
    int c = (int)(rem / m), q = (int)(rem - (size_t)c * m);
    const double* cb = coarse + (size_t)blk * C.nc * m;
    double v = 0.0;
    #pragma unroll
    for (int s = 0; s < 4; ++s) v += w4[4 * c + s] * cb[(size_t)idx4[4 * c + s] * m + q];
    fine[t] += v;
    if (out_pro) out_pro[t] = v;
}

cudaError_t launch_prolong_add(const LevelDev& F, const LevelDev& C, int m, int nblk, const int* idx4,
                               const double* w4, const double* coarse, double* fine, double* out_pro,
                               cudaStream_t st)
{
    size_t n = (size_t)F.nc * m * nblk;
    k_prolong_add<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(F, C, m, nblk, idx4, w4, coarse, fine, out_pro);
    return cudaGetLastError();
}

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
