// adjoint.cu -- differentiation form of the MIUGKS path (arXiv 1704.03151):
// the transposed Jacobian of the discrete steady equations
//   N(f; theta)_i,k = (g+_k(W_i, q_i) - f_i,k) / tau(W_i)
//                     - (1/V_i) sum_j S_ij Phi_ij,k(f; theta) / dt_p
// (Eq. microResidualDef with the predicted state equal to the moments of f,
// the UGKS interface flux of Step 1 and the diffuse wall of Sec. 3.2), the
// transposed LU-SGS preconditioner, and the wall objectives whose gradient
// with respect to a wall temperature or velocity the adjoint delivers.
//
// (dN/df)^T mu is assembled in three launches:
//   k_adj_face   one CTA per face: recomputes the face's forward scalars and
//                reduces the reverse sweep over the velocities into a small
//                per-face record (adjoints of the interface state, heat flux
//                and neighbour cell states);
//   k_adj_cell   one CTA per cell: the same for the collision term;
//   k_adj_gather one thread per (cell, velocity): sums, without atomics, what
//                the (up to eight) faces whose stencil holds the cell and the
//                cell's own collision term contribute to that entry.
// Everything runs in FP64 on an FP64 copy (checkpoint) of f.
#include "kernels.cuh"
#include <climits>

namespace miugks {

namespace {

constexpr int kRed = 32;   // shared reduction slots per value (one per warp)
constexpr size_t kAdjCacheBytes = 160 * 1024;   // dynamic shared memory of the cached face kernel (at most)
constexpr int kAdjKc = 4;                         // velocities per CTA of the transposed wavefront

// time integrals q_m(dt, tau) of the UGKS integral solution and their tau
// derivatives: closed form for x = dt/tau >= 1, power series below
__device__ void adj_time_coeffs(double dt, double tau, double q[5], double dq[5])
{
    double x = dt / tau;
    if (x < 1.0) {
        // q_m = dt^p_m s_m(x), s_m = sum_n c_mn x^n; dq_m/dtau = -(dt^p_m/tau) sum_n n c_mn x^n
        double s[5] = {0, 0, 0, 0, 0}, ds[5] = {0, 0, 0, 0, 0};
        double xn = 1.0, fact = 1.0;                  // x^n, n!
        for (int n = 0; n < 28; ++n) {
            if (n > 0) { xn *= x; fact *= n; }
            double sg = (n & 1) ? -1.0 : 1.0;           // (-1)^n
            double f1 = fact * (n + 1), f2 = f1 * (n + 2);   // (n+1)!, (n+2)!
            double c[5];
            c[0] = n >= 1 ? -sg / f1 : 0.0;             // (-1)^{n+1} x^n/(n+1)!
            c[1] = n >= 1 ? sg * n / f2 : 0.0;          // (-1)^n n x^n/(n+2)!
            c[2] = n >= 1 ? -sg / f2 : 0.0;             // (-1)^{n+1} x^n/(n+2)!
            c[3] = sg / f1;                             // (-1)^n x^n/(n+1)!
            c[4] = -sg * (n + 1) / f2;                  // (-1)^{n+1} (n+1) x^n/(n+2)!
            for (int m = 0; m < 5; ++m) { s[m] += c[m] * xn; ds[m] += n * c[m] * xn; }
        }
        const double p1 = dt, p2 = dt * dt;
        q[0] = p1 * s[0]; q[1] = p2 * s[1]; q[2] = p2 * s[2]; q[3] = p1 * s[3]; q[4] = p2 * s[4];
        dq[0] = -p1 / tau * ds[0]; dq[1] = -p2 / tau * ds[1]; dq[2] = -p2 / tau * ds[2];
        dq[3] = -p1 / tau * ds[3]; dq[4] = -p2 / tau * ds[4];
    } else {
        double e = exp(-x), E1 = -expm1(-x);
        q[0] = dt - tau * E1;
        q[1] = -tau * dt * (1.0 + e) + 2.0 * tau * tau * E1;
        q[2] = 0.5 * dt * dt - tau * dt + tau * tau * E1;
        q[3] = tau * E1;
        q[4] = tau * dt * e - tau * tau * E1;
        // d e / d tau = e x / tau
        dq[0] = -E1 + x * e;
        dq[1] = -dt * (1.0 + e) - dt * x * e + 4.0 * tau * E1 - 2.0 * tau * x * e;
        dq[2] = -dt + 2.0 * tau * E1 - tau * x * e;
        dq[3] = E1 - x * e;
        dq[4] = dt * e + dt * x * e - 2.0 * tau * E1 + tau * x * e;
    }
}

// conservative -> primitive (rho, U, V, lambda), plain divisions
__device__ __forceinline__ void adj_prim(const double* W, double& rho, double& U, double& V, double& lam)
{
    rho = W[0];
    U = W[1] / W[0];
    V = W[2] / W[0];
    double eint = W[3] - 0.5 * (W[1] * W[1] + W[2] * W[2]) / W[0];
    lam = (kKint + 2) * W[0] / (4.0 * eint);
}

// reverse of adj_prim: (rho, U, V, lam) adjoints -> W adjoint (added)
__device__ __forceinline__ void adj_prim_rev(const double* W, double rb, double Ub, double Vb, double lb, double* Wb)
{
    double rho, U, V, lam;
    adj_prim(W, rho, U, V, lam);
    double eint = W[3] - 0.5 * (W[1] * W[1] + W[2] * W[2]) / W[0];
    double eb = -lb * lam / eint;
    Wb[0] += rb + lb * lam / rho + eb * 0.5 * (U * U + V * V) - (Ub * U + Vb * V) / rho;
    Wb[1] += Ub / rho - eb * U;
    Wb[2] += Vb / rho - eb * V;
    Wb[3] += eb;
}

// equilibrium-slope inversion a = slope(dw; U, V, lam) and its reverse
__device__ __forceinline__ void adj_slope(const double dw[4], double U, double V, double lam, double a[4])
{
    const double Kp2 = kKint + 2.0;
    double cc = U * U + V * V + Kp2 / (2.0 * lam);
    double R4 = 2.0 * dw[3] - cc * dw[0], R3 = dw[2] - V * dw[0], R2 = dw[1] - U * dw[0];
    a[3] = 4.0 * lam * lam / Kp2 * (R4 - 2.0 * U * R2 - 2.0 * V * R3);
    a[2] = 2.0 * lam * R3 - V * a[3];
    a[1] = 2.0 * lam * R2 - U * a[3];
    a[0] = dw[0] - U * a[1] - V * a[2] - 0.5 * a[3] * cc;
}

__device__ void adj_slope_rev(const double dw[4], double U, double V, double lam, const double abar[4],
                              double dwb[4], double& Ub, double& Vb, double& lb)
{
    const double Kp2 = kKint + 2.0;
    double cc = U * U + V * V + Kp2 / (2.0 * lam);
    double R4 = 2.0 * dw[3] - cc * dw[0], R3 = dw[2] - V * dw[0], R2 = dw[1] - U * dw[0];
    double X = R4 - 2.0 * U * R2 - 2.0 * V * R3;
    double a3 = 4.0 * lam * lam / Kp2 * X, a2 = 2.0 * lam * R3 - V * a3, a1 = 2.0 * lam * R2 - U * a3;
    double ab0 = abar[0], ab1 = abar[1], ab2 = abar[2], ab3 = abar[3];
    double ccb = 0, R2b = 0, R3b = 0, R4b = 0;
    dwb[0] += ab0; Ub -= ab0 * a1; ab1 -= ab0 * U; Vb -= ab0 * a2; ab2 -= ab0 * V;
    ab3 -= ab0 * 0.5 * cc; ccb -= ab0 * 0.5 * a3;
    lb += ab1 * 2.0 * R2; R2b += ab1 * 2.0 * lam; Ub -= ab1 * a3; ab3 -= ab1 * U;
    lb += ab2 * 2.0 * R3; R3b += ab2 * 2.0 * lam; Vb -= ab2 * a3; ab3 -= ab2 * V;
    double Xb = ab3 * 4.0 * lam * lam / Kp2;
    lb += ab3 * 8.0 * lam / Kp2 * X;
    R4b += Xb; Ub -= Xb * 2.0 * R2; R2b -= Xb * 2.0 * U; Vb -= Xb * 2.0 * R3; R3b -= Xb * 2.0 * V;
    dwb[1] += R2b; Ub -= R2b * dw[0]; dwb[0] -= R2b * U;
    dwb[2] += R3b; Vb -= R3b * dw[0]; dwb[0] -= R3b * V;
    dwb[3] += 2.0 * R4b; ccb -= R4b * dw[0]; dwb[0] -= R4b * cc;
    Ub += 2.0 * U * ccb; Vb += 2.0 * V * ccb; lb -= ccb * Kp2 / (2.0 * lam * lam);
}

// (a . psi) g in the reduced components and its reverse
__device__ __forceinline__ void adj_smom(const double* a, double u, double v, double gM, double hM, double xi,
                                         double& mG, double& mH)
{
    double b = a[0] + a[1] * u + a[2] * v + 0.5 * a[3] * (u * u + v * v);
    mG = b * gM + a[3] * hM;
    mH = b * hM + a[3] * xi * gM;
}
__device__ __forceinline__ void adj_smom_rev(const double* a, double u, double v, double gM, double hM, double xi,
                                             double mGb, double mHb, double* ab, double& gMb, double& hMb,
                                             double& xib)
{
    double b = a[0] + a[1] * u + a[2] * v + 0.5 * a[3] * (u * u + v * v);
    double bb = mGb * gM + mHb * hM;
    ab[0] += bb; ab[1] += bb * u; ab[2] += bb * v;
    ab[3] += bb * 0.5 * (u * u + v * v) + mGb * hM + mHb * xi * gM;
    gMb += mGb * b + mHb * a[3] * xi;
    hMb += mGb * a[3] + mHb * b;
    xib += mHb * a[3] * gM;
}

// reverse of gM = rho (lam/pi) e^{-lam c^2}, hM = gM K / (4 lam)
__device__ __forceinline__ void adj_maxw_rev(double gM, double hM, double rho, double lam, double cx, double cy,
                                             double gMb, double hMb, double& rb, double& Ub, double& Vb, double& lb)
{
    double c2 = cx * cx + cy * cy;
    gMb += hMb * kKint / (4.0 * lam);
    lb -= hMb * hM / lam;
    rb += gMb * gM / rho;
    lb += gMb * gM * (1.0 / lam - c2);
    double c2b = -gMb * gM * lam;
    Ub -= 2.0 * cx * c2b;
    Vb -= 2.0 * cy * c2b;
}

__device__ __forceinline__ double adj_maxw(double rho, double U, double V, double lam, double u, double v)
{
    return rho * (lam / kPi) * exp(-lam * ((u - U) * (u - U) + (v - V) * (v - V)));
}

__device__ __forceinline__ double adj_vl(double s1, double s2)
{
    double p = s1 * s2;
    return p > 0.0 ? 2.0 * p / (s1 + s2) : 0.0;
}

// geometry of interior face fi along axis: stencil cells and distances
struct FaceGeo {
    int cLL, cL, cR, cRR;
    double dLLL, dLR, dRRR, hL, hR, wL, wR;
    double rLLL, rLR, rRRR;                 // reciprocals of the centre distances
};

__device__ __forceinline__ FaceGeo face_geo(const LevelDev& L, int axis, int fi)
{
    FaceGeo g;
    const int nx = L.nx, ny = L.ny;
    if (axis == 0) {
        int i = fi % (nx + 1), j = fi / (nx + 1);
        g.cL = j * nx + i - 1; g.cR = g.cL + 1;
        g.cLL = (i - 1 > 0 && L.fbx[fi - 1] < 0) ? g.cL - 1 : -1;
        g.cRR = (i + 1 < nx && L.fbx[fi + 1] < 0) ? g.cR + 1 : -1;
        g.dLLL = g.cLL >= 0 ? L.xc[i - 1] - L.xc[i - 2] : 1.0;
        g.dRRR = g.cRR >= 0 ? L.xc[i + 1] - L.xc[i] : 1.0;
        g.dLR = L.xc[i] - L.xc[i - 1];
        g.hL = L.xn[i] - L.xc[i - 1]; g.hR = L.xc[i] - L.xn[i];
        g.wL = L.dx[i - 1]; g.wR = L.dx[i];
    } else {
        int i = fi % nx, j = fi / nx;
        g.cL = (j - 1) * nx + i; g.cR = g.cL + nx;
        g.cLL = (j - 1 > 0 && L.fby[fi - nx] < 0) ? g.cL - nx : -1;
        g.cRR = (j + 1 < ny && L.fby[fi + nx] < 0) ? g.cR + nx : -1;
        g.dLLL = g.cLL >= 0 ? L.yc[j - 1] - L.yc[j - 2] : 1.0;
        g.dRRR = g.cRR >= 0 ? L.yc[j + 1] - L.yc[j] : 1.0;
        g.dLR = L.yc[j] - L.yc[j - 1];
        g.hL = L.yn[j] - L.yc[j - 1]; g.hR = L.yc[j] - L.yn[j];
        g.wL = L.dy[j - 1]; g.wR = L.dy[j];
    }
    g.rLLL = 1.0 / g.dLLL; g.rLR = 1.0 / g.dLR; g.rRRR = 1.0 / g.dRRR;
    return g;
}

// upwinded reconstructed face value and slope of one (velocity, component)
__device__ __forceinline__ void face_recon(const double* fc, size_t nv, int k, const FaceGeo& g, double un,
                                           double& f0, double& sg)
{
    double fL = fc[g.cL * nv + k], fR = fc[g.cR * nv + k];
    double sL = g.cLL >= 0 ? adj_vl((fL - fc[g.cLL * nv + k]) * g.rLLL, (fR - fL) * g.rLR) : 0.0;
    double sR = g.cRR >= 0 ? adj_vl((fR - fL) * g.rLR, (fc[g.cRR * nv + k] - fR) * g.rRRR) : 0.0;
    double faceL = fL + sL * g.hL, faceR = fR - sR * g.hR;
    if (un > 0) { f0 = faceL; sg = sL; }
    else if (un < 0) { f0 = faceR; sg = sR; }
    else { f0 = 0.5 * (faceL + faceR); sg = 0.5 * (sL + sR); }
}

template <int N>
__device__ __forceinline__ void red_sum(double (&v)[N], double* scratch)
{
    block_sum<N>(v, scratch);
}

} // namespace

// ---------------------------------------------------------------------------
// per-face record: [0..3] W0 adjoint, [4..5] q0 adjoint, [6] U0, [7] V0,
// [8] q4/dt, [9] q5/dt, [10..13] W_L adjoint, [14..17] W_R adjoint,
// [18] wall faces: rho_w adjoint / sum_in w u_o C, [20..22] reciprocal centre
// distances LL-L, L-R, R-RR, [23..24] face-centre distances h_L, h_R,
// [25..26] dN/dPhi coefficients of mu_L, mu_R, [27] 1 (LL exists) + 2 (RR exists).
// CACHE: the upwinded face values and slopes of every velocity are kept in
// shared memory after the first pass instead of being reconstructed again.
template <bool CACHE>
__global__ void __launch_bounds__(256) k_adj_face(AdjDev A, int axis, const double* __restrict__ mu,
                                                   double* __restrict__ rec)
{
    __shared__ double red[kRed * 25];
    extern __shared__ double etab[];           // e^{-lam0 (u_a - U0)^2} [nu], then e^{-lam0 (v_b - V0)^2} [nvv]
    double* fcache = etab + (A.V.nu + A.V.nvv);   // CACHE: [4][nv] f0 G, f0 H, slope G, slope H
    const LevelDev& L = A.L;
    const VelDev& Vg = A.V;
    const int nv = Vg.nv, tid = threadIdx.x, bs = blockDim.x, fi = blockIdx.x;
    const int nx = L.nx;
    const size_t nc = L.nc, snv = nv;
    const double* fG = A.f;
    const double* fH = A.f + nc * snv;
    const double* muG = mu;
    const double* muH = mu + nc * snv;
    double* out = rec + (size_t)fi * kFaceRec;
    const int i = axis == 0 ? fi % (nx + 1) : fi % nx;
    const int j = axis == 0 ? fi / (nx + 1) : fi / nx;
    const int bcid = (axis == 0 ? L.fbx : L.fby)[fi];

    if (bcid >= 0) {
        const BcDev B = A.bc[bcid];
        if (tid < kFaceRec) out[tid] = 0.0;
        if (B.type != BC_WALL) return;
        int outsign, c;                          // the face's fluid cell (domain edge or body face)
        bface_side(L, axis, i, j, c, outsign);
        const double d = axis == 0 ? L.dx[c % nx] : L.dy[c / nx];
        const double coef = (outsign < 0 ? 1.0 : -1.0) / d;     // nu = coef * mu_c
        const double* Cb = A.Cw + (size_t)bcid * nv;
        const double hf = kKint * B.t / 4.0;
        double s[2] = {0.0, 0.0};
        for (int k = tid; k < nv; k += bs) {
            double un = axis == 0 ? Vg.u[k] : Vg.v[k], uo = outsign * un;
            if (uo < 0) {
                double C = Cb[k];
                s[0] += un * coef * (muG[c * snv + k] * C + muH[c * snv + k] * C * hf);
                s[1] += Vg.w[k] * uo * C;
            }
        }
        red_sum<2>(s, red);
        if (tid == 0) out[18] = s[0] / s[1];
        return;
    }

    if (inactive_face(L, axis, i, j)) {          // inside a body: no flux, an empty record
        if (tid < kFaceRec) out[tid] = 0.0;
        return;
    }
    const FaceGeo g = face_geo(L, axis, fi);
    const double nuL = -1.0 / g.wL, nuR = 1.0 / g.wR;      // nu = nuL mu_L + nuR mu_R
    // upwinded reconstructed values and slopes of velocity k (both components)
    auto recon = [&](int k, double un, double& f0g, double& f0h, double& sgg, double& sgh) {
        if (CACHE) {
            f0g = fcache[k]; f0h = fcache[nv + k]; sgg = fcache[2 * nv + k]; sgh = fcache[3 * nv + k];
        } else {
            face_recon(fG, snv, k, g, un, f0g, sgg);
            face_recon(fH, snv, k, g, un, f0h, sgh);
        }
    };
    // ---- forward pass A: interface conservative variables
    double W0[4] = {0, 0, 0, 0};
    for (int k = tid; k < nv; k += bs) {
        double un = axis == 0 ? Vg.u[k] : Vg.v[k];
        double f0g, f0h, sg, sgh;
        face_recon(fG, snv, k, g, un, f0g, sg);
        face_recon(fH, snv, k, g, un, f0h, sgh);
        if (CACHE) { fcache[k] = f0g; fcache[nv + k] = f0h; fcache[2 * nv + k] = sg; fcache[3 * nv + k] = sgh; }
        double u = Vg.u[k], v = Vg.v[k], w = Vg.w[k];
        W0[0] += w * f0g; W0[1] += w * u * f0g; W0[2] += w * v * f0g;
        W0[3] += w * (0.5 * (u * u + v * v) * f0g + f0h);
    }
    red_sum<4>(W0, red);
    // Face scalars are computed by thread 0 and broadcast through shared memory
    // (an FP64 division or series costs the SM as much for one lane as for 32).
    __shared__ double sc[32];
    double rho0, U0, V0, lam0, tau0 = 0, dt = 0, xi;
    double dwl[4], dwr[4], aL[4], aR[4];
    if (tid == 0) {
        adj_prim(W0, rho0, U0, V0, lam0);
        const double T0 = 1.0 / lam0;
        tau0 = A.gas.mu_ref * pow(T0, A.gas.omega) / (0.5 * rho0 * T0);
        dt = A.cfl * fmin(g.wL, g.wR) / (axis == 0 ? Vg.umax : Vg.vmax);
        const double* WL = A.W + 4 * (size_t)g.cL;
        const double* WR = A.W + 4 * (size_t)g.cR;
        for (int m = 0; m < 4; ++m) {
            dwl[m] = (W0[m] - WL[m]) / g.hL / rho0;
            dwr[m] = (WR[m] - W0[m]) / g.hR / rho0;
        }
        adj_slope(dwl, U0, V0, lam0, aL);
        adj_slope(dwr, U0, V0, lam0, aR);
        sc[0] = rho0; sc[1] = U0; sc[2] = V0; sc[3] = lam0; sc[4] = tau0; sc[5] = dt;
        for (int m = 0; m < 4; ++m) { sc[6 + m] = aL[m]; sc[10 + m] = aR[m]; }
        sc[14] = kKint * (kKint + 2.0) / (16.0 * lam0 * lam0);
        sc[15] = rho0 * lam0 / kPi; sc[16] = kKint / (4.0 * lam0); sc[17] = 1.0 / dt;
    }
    __syncthreads();
    rho0 = sc[0]; U0 = sc[1]; V0 = sc[2]; lam0 = sc[3];
    for (int m = 0; m < 4; ++m) { aL[m] = sc[6 + m]; aR[m] = sc[10 + m]; }
    xi = sc[14];
    // separable equilibrium: gM(k) = rho0 lam0/pi Eu[a] Ev[b] (nu + nvv exponentials per face)
    for (int e = tid; e < Vg.nu + Vg.nvv; e += bs) {
        double dlt = e < Vg.nu ? Vg.ua[e] - U0 : Vg.vb[e - Vg.nu] - V0;
        etab[e] = exp(-lam0 * dlt * dlt);
    }
    __syncthreads();
    const double gnorm = sc[15], hfac = sc[16], idt = sc[17];
    auto gM_of = [&](int k) -> double { int a = k / Vg.nvv; return gnorm * etab[a] * etab[Vg.nu + k - a * Vg.nvv]; };
    // ---- forward pass B: heat flux of f0 and compatibility moments
    double s6[6] = {0, 0, 0, 0, 0, 0};
    for (int k = tid; k < nv; k += bs) {
        double un = axis == 0 ? Vg.u[k] : Vg.v[k];
        double f0g, f0h, sg, sgh;
        recon(k, un, f0g, f0h, sg, sgh);
        double u = Vg.u[k], v = Vg.v[k], w = Vg.w[k];
        double cx = u - U0, cy = v - V0, c2 = cx * cx + cy * cy, e = 0.5 * c2 * f0g + f0h;
        s6[0] += w * cx * e;
        s6[1] += w * cy * e;
        if (un != 0.0) {
            double gM = gM_of(k), hM = gM * hfac, mG, mH;
            adj_smom(un > 0 ? aL : aR, u, v, gM, hM, xi, mG, mH);
            s6[2] += w * un * mG; s6[3] += w * un * u * mG; s6[4] += w * un * v * mG;
            s6[5] += w * un * (0.5 * (u * u + v * v) * mG + mH);
        }
    }
    red_sum<6>(s6, red);
    const double q0[2] = {s6[0], s6[1]};
    const double Mt[4] = {s6[2], s6[3], s6[4], s6[5]};
    double dwt[4], At[4], qc[5], dqc[5];
    if (tid == 0) {
        for (int m = 0; m < 4; ++m) dwt[m] = -Mt[m] / rho0;
        adj_slope(dwt, U0, V0, lam0, At);
        adj_time_coeffs(dt, tau0, qc, dqc);
        for (int m = 0; m < 4; ++m) sc[18 + m] = At[m];
        for (int m = 0; m < 5; ++m) sc[22 + m] = qc[m];
        sc[27] = (1.0 - A.gas.pr) * 4.0 * lam0 * lam0 / (5.0 * rho0);
    }
    __syncthreads();
    for (int m = 0; m < 4; ++m) At[m] = sc[18 + m];
    for (int m = 0; m < 5; ++m) qc[m] = sc[22 + m];
    const double shk = sc[27];

    // ---- reverse pass C: the flux assembly
    // r[0..4] qc adjoint, [5..8] aL, [9..12] aR, [13..16] A, [17] rho, [18] U, [19] V, [20] lam,
    // [21] shk, [22] xi, [23..24] q0
    double r[25];
    for (int m = 0; m < 25; ++m) r[m] = 0.0;
    for (int k = tid; k < nv; k += bs) {
        double un = axis == 0 ? Vg.u[k] : Vg.v[k];
        if (un == 0.0) continue;
        double f0g, f0h, sgg, sgh;
        recon(k, un, f0g, f0h, sgg, sgh);
        double u = Vg.u[k], v = Vg.v[k];
        double cx = u - U0, cy = v - V0, c2 = cx * cx + cy * cy;
        double gM = gM_of(k), hM = gM * hfac;
        double Fq = shk * (cx * q0[0] + cy * q0[1]);
        double eG = 2.0 * lam0 * c2 - 4.0, eH = 2.0 * lam0 * c2 - 2.0;
        double gP = gM * (1.0 + Fq * eG), hP = hM * (1.0 + Fq * eH);
        const double* as = un > 0 ? aL : aR;
        double* asb = r + (un > 0 ? 5 : 9);
        double mGa, mHa, mGA, mHA;
        adj_smom(as, u, v, gM, hM, xi, mGa, mHa);
        adj_smom(At, u, v, gM, hM, xi, mGA, mHA);
        double PbG = (nuL * muG[g.cL * snv + k] + nuR * muG[g.cR * snv + k]) * idt;
        double PbH = (nuL * muH[g.cL * snv + k] + nuR * muH[g.cR * snv + k]) * idt;
        r[0] += un * (PbG * gP + PbH * hP);
        r[1] += un * un * (PbG * mGa + PbH * mHa);
        r[2] += un * (PbG * mGA + PbH * mHA);
        r[3] += un * (PbG * f0g + PbH * f0h);
        r[4] += un * un * (PbG * sgg + PbH * sgh);
        double gPb = un * qc[0] * PbG, hPb = un * qc[0] * PbH;
        double gMb = 0.0, hMb = 0.0;
        adj_smom_rev(as, u, v, gM, hM, xi, un * un * qc[1] * PbG, un * un * qc[1] * PbH, asb, gMb, hMb, r[22]);
        adj_smom_rev(At, u, v, gM, hM, xi, un * qc[2] * PbG, un * qc[2] * PbH, r + 13, gMb, hMb, r[22]);
        gMb += gPb * (1.0 + Fq * eG);
        hMb += hPb * (1.0 + Fq * eH);
        double Fqb = gPb * gM * eG + hPb * hM * eH;
        double eb = (gPb * gM + hPb * hM) * Fq;
        r[20] += eb * 2.0 * c2;
        double c2b = eb * 2.0 * lam0;
        r[21] += Fqb * (cx * q0[0] + cy * q0[1]);
        r[23] += Fqb * shk * cx;
        r[24] += Fqb * shk * cy;
        double cxb = Fqb * shk * q0[0] + 2.0 * cx * c2b, cyb = Fqb * shk * q0[1] + 2.0 * cy * c2b;
        r[18] -= cxb; r[19] -= cyb;
        adj_maxw_rev(gM, hM, rho0, lam0, cx, cy, gMb, hMb, r[17], r[18], r[19], r[20]);
    }
    red_sum<25>(r, red);
    double aLb[4] = {r[5], r[6], r[7], r[8]}, aRb[4] = {r[9], r[10], r[11], r[12]};
    double rb = r[17], Ub = r[18], Vb = r[19], lb = r[20], xib = r[22];
    const double q0b[2] = {r[23], r[24]};
    double Mtb[4];
    __shared__ double sM[4];
    if (tid == 0) {
        lb += r[21] * 2.0 * shk / lam0;
        rb -= r[21] * shk / rho0;
        double dwtb[4] = {0, 0, 0, 0};
        adj_slope_rev(dwt, U0, V0, lam0, r + 13, dwtb, Ub, Vb, lb);
        for (int m = 0; m < 4; ++m) {
            Mtb[m] = -dwtb[m] / rho0;
            rb += dwtb[m] * Mt[m] / (rho0 * rho0);
            sM[m] = Mtb[m];
        }
        double taub = 0.0;
        for (int m = 0; m < 5; ++m) taub += r[m] * dqc[m];
        rb -= taub * tau0 / rho0;
        lb += taub * tau0 * (1.0 - A.gas.omega) / lam0;
    }
    __syncthreads();
    for (int m = 0; m < 4; ++m) Mtb[m] = sM[m];

    // ---- reverse pass D: heat flux and compatibility moments
    double t[13];
    for (int m = 0; m < 13; ++m) t[m] = 0.0;      // [0..3] aL, [4..7] aR, [8] rho, [9] U, [10] V, [11] lam, [12] xi
    for (int k = tid; k < nv; k += bs) {
        double un = axis == 0 ? Vg.u[k] : Vg.v[k];
        double f0g, f0h, sg, sgh;
        recon(k, un, f0g, f0h, sg, sgh);
        double u = Vg.u[k], v = Vg.v[k], w = Vg.w[k];
        double cx = u - U0, cy = v - V0, c2 = cx * cx + cy * cy, E = 0.5 * c2 * f0g + f0h;
        if (un != 0.0) {
            double gM = gM_of(k), hM = gM * hfac;
            double mGb = w * un * (Mtb[0] + Mtb[1] * u + Mtb[2] * v + Mtb[3] * 0.5 * (u * u + v * v));
            double mHb = w * un * Mtb[3];
            double gMb = 0.0, hMb = 0.0;
            adj_smom_rev(un > 0 ? aL : aR, u, v, gM, hM, xi, mGb, mHb, t + (un > 0 ? 0 : 4), gMb, hMb, t[12]);
            adj_maxw_rev(gM, hM, rho0, lam0, cx, cy, gMb, hMb, t[8], t[9], t[10], t[11]);
        }
        t[9] -= w * (q0b[0] * (E + cx * cx * f0g) + q0b[1] * cy * cx * f0g);
        t[10] -= w * (q0b[1] * (E + cy * cy * f0g) + q0b[0] * cx * cy * f0g);
    }
    red_sum<13>(t, red);
    if (tid == 0) {
        for (int m = 0; m < 4; ++m) { aLb[m] += t[m]; aRb[m] += t[4 + m]; }
        rb += t[8]; Ub += t[9]; Vb += t[10]; lb += t[11]; xib += t[12];
        lb += xib * (-2.0 * xi / lam0);
        double dwlb[4] = {0, 0, 0, 0}, dwrb[4] = {0, 0, 0, 0};
        adj_slope_rev(dwl, U0, V0, lam0, aLb, dwlb, Ub, Vb, lb);
        adj_slope_rev(dwr, U0, V0, lam0, aRb, dwrb, Ub, Vb, lb);
        double W0b[4] = {0, 0, 0, 0};
        for (int m = 0; m < 4; ++m) {
            W0b[m] += dwlb[m] / (g.hL * rho0) - dwrb[m] / (g.hR * rho0);
            out[10 + m] = -dwlb[m] / (g.hL * rho0);
            out[14 + m] = dwrb[m] / (g.hR * rho0);
            rb -= (dwlb[m] * dwl[m] + dwrb[m] * dwr[m]) / rho0;
        }
        adj_prim_rev(W0, rb, Ub, Vb, lb, W0b);
        for (int m = 0; m < 4; ++m) out[m] = W0b[m];
        out[4] = q0b[0]; out[5] = q0b[1];
        out[6] = U0; out[7] = V0;
        out[8] = qc[3] / dt; out[9] = qc[4] / dt;
        out[18] = 0.0; out[19] = 0.0;
        out[20] = g.rLLL; out[21] = g.rLR; out[22] = g.rRRR; out[23] = g.hL; out[24] = g.hR;
        out[25] = nuL; out[26] = nuR; out[27] = (g.cLL >= 0 ? 1.0 : 0.0) + (g.cRR >= 0 ? 2.0 : 0.0);
    }
}

// per-cell record: [0..3] W adjoint, [4..5] q adjoint, [6] U, [7] V, [8] 1/tau
__global__ void __launch_bounds__(256) k_adj_cell(AdjDev A, const double* __restrict__ mu, double* __restrict__ crec)
{
    __shared__ double red[kRed * 8];
    const VelDev& Vg = A.V;
    const int nv = Vg.nv, tid = threadIdx.x, bs = blockDim.x, c = blockIdx.x;
    const size_t nc = A.L.nc, snv = nv;
    const double* fG = A.f + c * snv;
    const double* fH = A.f + (nc + c) * snv;
    const double* mG = mu + c * snv;
    const double* mH = mu + (nc + c) * snv;
    const double* W = A.W + 4 * (size_t)c;
    const double* q = A.q + 2 * (size_t)c;
    double rho, U, V, lam;
    adj_prim(W, rho, U, V, lam);
    const double T = 1.0 / lam;
    const double itau = 1.0 / (A.gas.mu_ref * pow(T, A.gas.omega) / (0.5 * rho * T));
    const double S = (1.0 - A.gas.pr) * 4.0 / 5.0 * lam * lam / rho;
    // [0] rho, [1] U, [2] V, [3] lam, [4] S, [5] itau, [6..7] q
    double r[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = tid; k < nv; k += bs) {
        double u = Vg.u[k], v = Vg.v[k];
        double cx = u - U, cy = v - V, c2 = cx * cx + cy * cy;
        double gM = adj_maxw(rho, U, V, lam, u, v), hM = gM * kKint / (4.0 * lam);
        double Fq = S * (cx * q[0] + cy * q[1]);
        double eG = 2.0 * lam * c2 - 4.0, eH = 2.0 * lam * c2 - 2.0;
        double gP = gM * (1.0 + Fq * eG), hP = hM * (1.0 + Fq * eH);
        double a = mG[k], b = mH[k];
        r[5] += a * (gP - fG[k]) + b * (hP - fH[k]);
        double gPb = a * itau, hPb = b * itau;
        double gMb = gPb * (1.0 + Fq * eG), hMb = hPb * (1.0 + Fq * eH);
        double Fqb = gPb * gM * eG + hPb * hM * eH;
        double eb = (gPb * gM + hPb * hM) * Fq;
        r[3] += eb * 2.0 * c2;
        double c2b = eb * 2.0 * lam;
        r[4] += Fqb * (cx * q[0] + cy * q[1]);
        r[6] += Fqb * S * cx;
        r[7] += Fqb * S * cy;
        r[1] -= Fqb * S * q[0] + 2.0 * cx * c2b;
        r[2] -= Fqb * S * q[1] + 2.0 * cy * c2b;
        adj_maxw_rev(gM, hM, rho, lam, cx, cy, gMb, hMb, r[0], r[1], r[2], r[3]);
    }
    red_sum<8>(r, red);
    double rb = r[0], Ub = r[1], Vb = r[2], lb = r[3];
    const double qb[2] = {r[6], r[7]};
    lb += r[4] * 2.0 * S / lam;
    rb -= r[4] * S / rho;
    rb += r[5] * itau / rho;
    lb += r[5] * itau * (A.gas.omega - 1.0) / lam;
    double t[2] = {0, 0};
    for (int k = tid; k < nv; k += bs) {
        double cx = Vg.u[k] - U, cy = Vg.v[k] - V, c2 = cx * cx + cy * cy;
        double gk = fG[k], E = 0.5 * c2 * gk + fH[k], w = Vg.w[k];
        t[0] -= w * (qb[0] * (E + cx * cx * gk) + qb[1] * cy * cx * gk);
        t[1] -= w * (qb[1] * (E + cy * cy * gk) + qb[0] * cx * cy * gk);
    }
    red_sum<2>(t, red);
    Ub += t[0]; Vb += t[1];
    if (tid == 0) {
        double Wb[4] = {0, 0, 0, 0};
        adj_prim_rev(W, rb, Ub, Vb, lb, Wb);
        double* o = crec + (size_t)kCellRec * c;
        for (int m = 0; m < 4; ++m) o[m] = Wb[m];
        o[4] = qb[0]; o[5] = qb[1]; o[6] = U; o[7] = V; o[8] = itau;
    }
}

namespace {
// what interior face (axis, fi) contributes to entry (cell at position pos of
// the face's stencil: 0 LL, 1 L, 2 R, 3 RR, velocity k) of (dN/df)^T mu
__device__ __forceinline__ void face_contrib(const AdjDev& A, const double* mu, const double* rec, int axis, int fi,
                                             int pos, int k, double out[2])
{
    const LevelDev& L = A.L;
    const VelDev& Vg = A.V;
    const size_t nc = L.nc, snv = Vg.nv;
    const double* R = rec + (size_t)fi * kFaceRec;
    const int flags = (int)R[27];
    if ((pos == 0 && !(flags & 1)) || (pos == 3 && !(flags & 2))) return;
    // stencil and geometry of the face (computed once per face by k_adj_face)
    FaceGeo g;
    const int nx = L.nx;
    if (axis == 0) {
        int i = fi % (nx + 1), j = fi / (nx + 1);
        g.cL = j * nx + i - 1; g.cR = g.cL + 1;
        g.cLL = (flags & 1) ? g.cL - 1 : -1; g.cRR = (flags & 2) ? g.cR + 1 : -1;
    } else {
        int i = fi % nx, j = fi / nx;
        g.cL = (j - 1) * nx + i; g.cR = g.cL + nx;
        g.cLL = (flags & 1) ? g.cL - nx : -1; g.cRR = (flags & 2) ? g.cR + nx : -1;
    }
    g.rLLL = R[20]; g.rLR = R[21]; g.rRRR = R[22]; g.hL = R[23]; g.hR = R[24];
    const double u = Vg.u[k], v = Vg.v[k], w = Vg.w[k];
    const double un = axis == 0 ? u : v;
    const double e2 = 0.5 * (u * u + v * v);
    const double cx = u - R[6], cy = v - R[7], qdc = R[4] * cx + R[5] * cy;
    const double nuL = R[25], nuR = R[26];
    for (int cp = 0; cp < 2; ++cp) {
        const double* fc = A.f + cp * nc * snv;
        const double* mc = mu + cp * nc * snv;
        double nu = nuL * mc[g.cL * snv + k] + nuR * mc[g.cR * snv + k];
        double psi0 = cp == 0 ? R[0] + u * R[1] + v * R[2] + e2 * R[3] : R[3];
        double fb = un * R[8] * nu + w * psi0 + (cp == 0 ? w * qdc * 0.5 * (cx * cx + cy * cy) : w * qdc);
        double sb = un * un * R[9] * nu;
        double fLb = 0.0, fRb = 0.0, sLb = 0.0, sRb = 0.0;
        if (pos == 1) fLb = w * (cp == 0 ? R[10] + u * R[11] + v * R[12] + e2 * R[13] : R[13]);
        if (pos == 2) fRb = w * (cp == 0 ? R[14] + u * R[15] + v * R[16] + e2 * R[17] : R[17]);
        if (un > 0) { fLb += fb; sLb = fb * g.hL + sb; }
        else if (un < 0) { fRb += fb; sRb = -fb * g.hR + sb; }
        else { fLb += 0.5 * fb; fRb += 0.5 * fb; sLb = 0.5 * fb * g.hL + 0.5 * sb; sRb = -0.5 * fb * g.hR + 0.5 * sb; }
        double fL = fc[g.cL * snv + k], fR = fc[g.cR * snv + k];
        double res = pos == 1 ? fLb : pos == 2 ? fRb : 0.0;
        if (g.cLL >= 0 && sLb != 0.0) {
            double s1 = (fL - fc[g.cLL * snv + k]) * g.rLLL, s2 = (fR - fL) * g.rLR;
            if (s1 * s2 > 0.0) {
                // d/ds1 of 2 s1 s2/(s1 + s2) is 2 (s2/(s1 + s2))^2: quotients in (0, 1), so the
                // derivative stays finite for slopes near the underflow threshold (far velocity tails)
                const double q1 = s1 / (s1 + s2), q2 = s2 / (s1 + s2);
                double s1b = 2.0 * sLb * q2 * q2, s2b = 2.0 * sLb * q1 * q1;
                if (pos == 0) res -= s1b * g.rLLL;
                else if (pos == 1) res += s1b * g.rLLL - s2b * g.rLR;
                else if (pos == 2) res += s2b * g.rLR;
            }
        }
        if (g.cRR >= 0 && sRb != 0.0) {
            double s2 = (fR - fL) * g.rLR, s3 = (fc[g.cRR * snv + k] - fR) * g.rRRR;
            if (s2 * s3 > 0.0) {
                const double q2 = s2 / (s2 + s3), q3 = s3 / (s2 + s3);
                double s2b = 2.0 * sRb * q3 * q3, s3b = 2.0 * sRb * q2 * q2;
                if (pos == 1) res -= s2b * g.rLR;
                else if (pos == 2) res += s2b * g.rLR - s3b * g.rRRR;
                else if (pos == 3) res += s3b * g.rRRR;
            }
        }
        out[cp] += res;
    }
}

// what boundary face (axis, fi) of cell c contributes to entry (c, k)
__device__ __forceinline__ void boundary_contrib(const AdjDev& A, const double* mu, const double* rec, int axis,
                                                 int fi, int c, int outsign, double d, int k, double out[2])
{
    const VelDev& Vg = A.V;
    const size_t nc = A.L.nc, snv = Vg.nv;
    const int bcid = (axis == 0 ? A.L.fbx : A.L.fby)[fi];
    const int type = A.bc[bcid].type;
    const double coef = (outsign < 0 ? 1.0 : -1.0) / d;
    const double un = axis == 0 ? Vg.u[k] : Vg.v[k], uo = outsign * un;
    if (uo >= 0 || type == BC_OUTFLOW) {
        out[0] += un * coef * mu[c * snv + k];
        out[1] += un * coef * mu[(nc + c) * snv + k];
    }
    if (type == BC_WALL && uo > 0) out[0] += -Vg.w[k] * uo * rec[(size_t)fi * kFaceRec + 18];
    if (type == BC_SYMMETRY && uo > 0) {
        int a = k / Vg.nvv, b = k - a * Vg.nvv;
        int km = axis == 0 ? (Vg.nu - 1 - a) * Vg.nvv + b : a * Vg.nvv + (Vg.nvv - 1 - b);
        double unm = axis == 0 ? Vg.u[km] : Vg.v[km];
        out[0] += unm * coef * mu[c * snv + km];
        out[1] += unm * coef * mu[(nc + c) * snv + km];
    }
}
} // namespace

// out = (dN/df)^T mu (+ pen * dM/df when pen != 0): one thread per (cell, velocity)
__global__ void __launch_bounds__(128) k_adj_gather(AdjDev A, const double* __restrict__ mu,
                                                     const double* __restrict__ recx, const double* __restrict__ recy,
                                                     const double* __restrict__ crec, double pen,
                                                     double* __restrict__ out)
{
    const LevelDev& L = A.L;
    const VelDev& Vg = A.V;
    const int nv = Vg.nv, c = blockIdx.x, k = blockIdx.y * blockDim.x + threadIdx.x;
    if (k >= nv) return;
    const int nx = L.nx, ny = L.ny, i = c % nx, j = c / nx;
    const size_t nc = L.nc, snv = nv;
    if (L.solid[c]) {                              // N = -f in a body
        out[c * snv + k] = -mu[c * snv + k];
        out[(nc + c) * snv + k] = -mu[(nc + c) * snv + k];
        return;
    }
    double acc[2] = {0.0, 0.0};
    // collision term of the cell itself
    {
        const double* C = crec + (size_t)kCellRec * c;
        const double u = Vg.u[k], v = Vg.v[k], w = Vg.w[k];
        const double cx = u - C[6], cy = v - C[7], c2 = cx * cx + cy * cy, qdc = C[4] * cx + C[5] * cy;
        acc[0] = -mu[c * snv + k] * C[8] + w * qdc * 0.5 * c2 + w * (C[0] + u * C[1] + v * C[2] + 0.5 * (u * u + v * v) * C[3]);
        acc[1] = -mu[(nc + c) * snv + k] * C[8] + w * qdc + w * C[3];
    }
    // x-faces ii = i-1 .. i+2 (face ii between cells ii-1 and ii)
    for (int ii = i - 1; ii <= i + 2; ++ii) {
        if (ii < 0 || ii > nx) continue;
        const int fi = j * (nx + 1) + ii;
        if (L.fbx[fi] >= 0) {
            if (ii == i || ii == i + 1) {              // a boundary face of this cell (domain edge or body)
                int cc, os;
                bface_side(L, 0, ii, j, cc, os);
                if (cc == c) boundary_contrib(A, mu, recx, 0, fi, c, os, L.dx[i], k, acc);
            }
            continue;
        }
        if (inactive_face(L, 0, ii, j)) continue;
        face_contrib(A, mu, recx, 0, fi, ii - i + 1 == 0 ? 3 : ii - i + 1 == 1 ? 2 : ii - i + 1 == 2 ? 1 : 0, k, acc);
    }
    for (int jj = j - 1; jj <= j + 2; ++jj) {
        if (jj < 0 || jj > ny) continue;
        const int fi = jj * nx + i;
        if (L.fby[fi] >= 0) {
            if (jj == j || jj == j + 1) {
                int cc, os;
                bface_side(L, 1, i, jj, cc, os);
                if (cc == c) boundary_contrib(A, mu, recy, 1, fi, c, os, L.dy[j], k, acc);
            }
            continue;
        }
        if (inactive_face(L, 1, i, jj)) continue;
        face_contrib(A, mu, recy, 1, fi, jj - j + 1 == 0 ? 3 : jj - j + 1 == 1 ? 2 : jj - j + 1 == 2 ? 1 : 0, k, acc);
    }
    if (pen != 0.0) acc[0] += pen * L.dx[i] * L.dy[j] * Vg.w[k];
    out[c * snv + k] = acc[0];
    out[(nc + c) * snv + k] = acc[1];
}

// ---------------------------------------------------------------------------
// Transposed LU-SGS pass.  The evolution smoother solves (D + L') x* = r then
// (D + U') x = D x* (L' / U': lower / upper neighbours and the within-cell
// ghost couplings of the lower / upper boundary faces), i.e. x = P r with
// P = (D + U')^{-1} D (D + L')^{-1}.  Its transpose is
//   P^T = (D + L'^T)^{-1} D (D + U'^T)^{-1}:
// pass 0 solves (D + U'^T) y = r in ascending anti-diagonal order (the upper
// neighbours' coefficients, read from the lower neighbours' rows, and the
// transposed couplings of the cell's upper boundary faces); pass 1 solves
// (D + L'^T) x = D y in descending order.  One CTA per cell of one
// anti-diagonal; one launch per diagonal.
// one cell (i, j) of a transposed pass, all velocities, by the whole CTA
// (ys: 2 nv doubles of shared memory, red: 4 kRed doubles)
__device__ void adjT_cell(const AdjSweepArgs& S, int pass, int i, int j, double* ys, double* red)
{
    const LevelDev& L = S.L;
    const VelDev& Vg = S.V;
    const int nx = L.nx, ny = L.ny, nv = Vg.nv, tid = threadIdx.x, bs = blockDim.x;
    const size_t nc = L.nc, snv = nv;
    const int c = j * nx + i;
    const double rdx = L.rdx[i], rdy = L.rdy[j];
    const double it = S.inv_tau[c];
    double* dst = pass == 0 ? S.y : S.x;
    // neighbours: pass 0 lower (west, south), pass 1 upper (east, north)
    const bool nW = pass == 0 && i > 0 && L.fbx[j * (nx + 1) + i] < 0;
    const bool nS = pass == 0 && j > 0 && L.fby[j * nx + i] < 0;
    const bool nE = pass == 1 && i < nx - 1 && L.fbx[j * (nx + 1) + i + 1] < 0;
    const bool nN = pass == 1 && j < ny - 1 && L.fby[(j + 1) * nx + i] < 0;
    const double cW = nW ? L.rdx[i - 1] : 0.0, cS = nS ? L.rdy[j - 1] : 0.0;
    const double cE = nE ? L.rdx[i + 1] : 0.0, cN = nN ? L.rdy[j + 1] : 0.0;
    // boundary faces on this pass's side: pass 0 upper (east, north), pass 1 lower (west, south)
    int nb = 0, bax[2], bos[2], bid[2];
    double bS[2];
    if (pass == 1 && i == 0) { bax[nb] = 0; bos[nb] = -1; bid[nb] = L.fbx[j * (nx + 1)]; bS[nb] = rdx; ++nb; }
    if (pass == 1 && j == 0) { bax[nb] = 1; bos[nb] = -1; bid[nb] = L.fby[i]; bS[nb] = rdy; ++nb; }
    if (pass == 0 && i == nx - 1) { bax[nb] = 0; bos[nb] = 1; bid[nb] = L.fbx[j * (nx + 1) + nx]; bS[nb] = rdx; ++nb; }
    if (pass == 0 && j == ny - 1) { bax[nb] = 1; bos[nb] = 1; bid[nb] = L.fby[ny * nx + i]; bS[nb] = rdy; ++nb; }
    int btype[2] = {-1, -1};
    double Z[2] = {0.0, 0.0}, Hf[2] = {0.0, 0.0};
    int nwall = 0, nsym = 0;
    for (int b = 0; b < nb; ++b) {
        btype[b] = S.bc[bid[b]].type;
        Hf[b] = kKint * S.bc[bid[b]].t / 4.0;
        if (btype[b] == BC_WALL) { ++nwall; Z[b] = S.Zw[bid[b] * 4 + bax[b] * 2 + (bos[b] > 0)]; }
        if (btype[b] == BC_SYMMETRY) ++nsym;
    }
    // Db(k): (1/V) u_o S through face b for an incoming velocity (u_o < 0), else 0
    auto Db = [&](int b, int k) -> double {
        double uo = bos[b] * (bax[b] == 0 ? Vg.u[k] : Vg.v[k]);
        return uo < 0 ? uo * bS[b] : 0.0;
    };
    auto Dk = [&](int k) -> double { return it + fabs(Vg.u[k]) * rdx + fabs(Vg.v[k]) * rdy; };
    bool outflow = false;
    for (int b = 0; b < nb; ++b) outflow = outflow || btype[b] == BC_OUTFLOW;
    // reciprocal of the diagonal (with the outflow ghost, which is the cell itself)
    auto rden_of = [&](int k) -> double {
        if (!outflow) return S.invD[(size_t)c * snv + k];
        double dd = Dk(k);
        for (int b = 0; b < nb; ++b) if (btype[b] == BC_OUTFLOW) dd += Db(b, k);
        return 1.0 / dd;
    };
    auto base_of = [&](int cp, int k) -> double {
        size_t e = (cp * nc + c) * snv + k;
        double u = Vg.u[k], v = Vg.v[k], bsum;
        if (pass == 0) {
            bsum = S.r[e];
            if (nW && u < 0) bsum -= u * cW * S.y[e - snv];
            if (nS && v < 0) bsum -= v * cS * S.y[e - (size_t)nx * snv];
        } else {
            bsum = Dk(k) * S.y[e];
            if (nE && u > 0) bsum += u * cE * S.x[e + snv];
            if (nN && v > 0) bsum += v * cN * S.x[e + (size_t)nx * snv];
        }
        return bsum;
    };
    auto mirror = [&](int b, int k) -> int {
        int a = k / Vg.nvv, bb = k - a * Vg.nvv;
        return bax[b] == 0 ? (Vg.nu - 1 - a) * Vg.nvv + bb : a * Vg.nvv + (Vg.nvv - 1 - bb);
    };

    if (nwall + nsym == 0) {
        for (int k = tid; k < nv; k += bs) {
            double rd = rden_of(k);
            dst[(size_t)c * snv + k] = base_of(0, k) * rd;
            dst[(nc + c) * snv + k] = base_of(1, k) * rd;
        }
        return;
    }
    if (nwall == 2 && nb == 2) {
        // s_b = sum over velocities incoming at wall b of Db (C y_G + C Hf y_H);
        // s_b = a_b + m_b s_o with o the other wall.  The right-hand sides stay
        // in shared memory between the two loops (each thread its own entries).
        double acc[4] = {0, 0, 0, 0};
        for (int k = tid; k < nv; k += bs) {
            double rd = rden_of(k), b0 = base_of(0, k), b1 = base_of(1, k);
            ys[k] = b0;
            ys[nv + k] = b1;
            for (int b = 0; b < 2; ++b) {
                double Dbk = Db(b, k);
                if (Dbk == 0.0) continue;
                int o = 1 - b;
                double C = S.Cw[(size_t)bid[b] * nv + k];
                acc[b] += Dbk * C * (b0 + Hf[b] * b1) * rd;
                double uoo = bos[o] * (bax[o] == 0 ? Vg.u[k] : Vg.v[k]);
                if (uoo > 0) acc[2 + b] += Dbk * C * Vg.w[k] * uoo / Z[o] * rd;
            }
        }
        red_sum<4>(acc, red);
        double s0 = (acc[0] + acc[2] * acc[1]) / (1.0 - acc[2] * acc[3]);
        double s1 = acc[1] + acc[3] * s0;
        double sb[2] = {s0, s1};
        for (int k = tid; k < nv; k += bs) {
            double rd = rden_of(k), g0 = ys[k];
            for (int b = 0; b < 2; ++b) {
                double uo = bos[b] * (bax[b] == 0 ? Vg.u[k] : Vg.v[k]);
                if (uo > 0) g0 += Vg.w[k] * uo / Z[b] * sb[b];
            }
            dst[(size_t)c * snv + k] = g0 * rd;
            dst[(nc + c) * snv + k] = ys[nv + k] * rd;
        }
        __syncthreads();
        return;
    }
    if (nb == 1 && nwall == 1) {
        // incoming rows have no coupling; the outgoing G rows need their sum
        double acc[1] = {0};
        for (int k = tid; k < nv; k += bs) {
            double b0 = base_of(0, k), b1 = base_of(1, k);
            ys[k] = b0;
            ys[nv + k] = b1;
            double Dbk = Db(0, k);
            if (Dbk != 0.0) acc[0] += Dbk * S.Cw[(size_t)bid[0] * nv + k] * (b0 + Hf[0] * b1) * rden_of(k);
        }
        red_sum<1>(acc, red);
        const double sZ = acc[0] / Z[0];
        for (int k = tid; k < nv; k += bs) {
            double rd = rden_of(k), g0 = ys[k];
            double uo = bos[0] * (bax[0] == 0 ? Vg.u[k] : Vg.v[k]);
            if (uo > 0) g0 += Vg.w[k] * uo * sZ;
            dst[(size_t)c * snv + k] = g0 * rd;
            dst[(nc + c) * snv + k] = ys[nv + k] * rd;
        }
        __syncthreads();
        return;
    }
    if (nb == 1 && nsym == 1) {
        // the outgoing rows take the mirrored incoming values, which have no coupling
        for (int k = tid; k < nv; k += bs) {
            ys[k] = base_of(0, k);
            ys[nv + k] = base_of(1, k);
        }
        __syncthreads();
        for (int k = tid; k < nv; k += bs) {
            double rd = rden_of(k), g0 = ys[k], g1 = ys[nv + k];
            double uo = bos[0] * (bax[0] == 0 ? Vg.u[k] : Vg.v[k]);
            if (uo > 0) {
                int km = mirror(0, k);
                double Dm = Db(0, km), rm = rden_of(km);
                g0 -= Dm * ys[km] * rm;
                g1 -= Dm * ys[nv + km] * rm;
            }
            dst[(size_t)c * snv + k] = g0 * rd;
            dst[(nc + c) * snv + k] = g1 * rd;
        }
        __syncthreads();
        return;
    }
    // three substitution rounds (exact: the coupling is nilpotent of the same
    // degree as in the untransposed block)
    for (int k = tid; k < nv; k += bs) {
        double rd = rden_of(k);
        ys[k] = base_of(0, k) * rd;
        ys[nv + k] = base_of(1, k) * rd;
    }
    __syncthreads();
    for (int round = 0; round < 3; ++round) {
        double sb[2] = {0.0, 0.0};
        for (int k = tid; k < nv; k += bs)
            for (int b = 0; b < nb; ++b) {
                if (btype[b] != BC_WALL) continue;
                double Dbk = Db(b, k);
                if (Dbk != 0.0) sb[b] += Dbk * S.Cw[(size_t)bid[b] * nv + k] * (ys[k] + Hf[b] * ys[nv + k]);
            }
        red_sum<2>(sb, red);     // ends with a barrier: ys is read by all before it changes
        for (int k = tid; k < nv; k += bs) {
            double rd = rden_of(k), g0 = base_of(0, k), g1 = base_of(1, k);
            for (int b = 0; b < nb; ++b) {
                double uo = bos[b] * (bax[b] == 0 ? Vg.u[k] : Vg.v[k]);
                if (!(uo > 0)) continue;
                if (btype[b] == BC_WALL) g0 += Vg.w[k] * uo / Z[b] * sb[b];
                else if (btype[b] == BC_SYMMETRY) {
                    int km = mirror(b, k);
                    double Dm = Db(b, km);
                    g0 -= Dm * ys[km];
                    g1 -= Dm * ys[nv + km];
                }
            }
            dst[(size_t)c * snv + k] = g0 * rd;
            dst[(nc + c) * snv + k] = g1 * rd;
        }
        __syncthreads();
        for (int k = tid; k < nv; k += bs) {
            ys[k] = dst[(size_t)c * snv + k];
            ys[nv + k] = dst[(nc + c) * snv + k];
        }
        __syncthreads();
    }
}

// The boundary lines on the side of a pass are sinks of its order: pass 0
// (ascending, upper boundary blocks) the last row and the last column, pass 1
// (descending, lower blocks) the first row and the first column.  They depend
// on each other only through the corner cell they share: CTA 0 walks the row,
// CTA 1 the column without the corner, one cell at a time; the corner follows
// in a launch of its own (corner = 1).
__global__ void __launch_bounds__(512) k_adjT_chain(AdjSweepArgs S, int pass, int corner)
{
    extern __shared__ double ys[];
    __shared__ double red[kRed * 4];
    const int nx = S.L.nx, ny = S.L.ny;
    if (corner) {
        if (pass == 0) adjT_cell(S, 0, nx - 1, ny - 1, ys, red);
        else adjT_cell(S, 1, 0, 0, ys, red);
        return;
    }
    if (pass == 0) {
        if (blockIdx.x == 0) for (int i = 0; i < nx - 1; ++i) { adjT_cell(S, 0, i, ny - 1, ys, red); __syncthreads(); }
        else for (int j = 0; j < ny - 1; ++j) { adjT_cell(S, 0, nx - 1, j, ys, red); __syncthreads(); }
    } else {
        if (blockIdx.x == 0) for (int i = nx - 1; i >= 1; --i) { adjT_cell(S, 1, i, 0, ys, red); __syncthreads(); }
        else for (int j = ny - 1; j >= 1; --j) { adjT_cell(S, 1, 0, j, ys, red); __syncthreads(); }
    }
}

// Every other cell of a pass has no domain-edge face on its side: a plain
// triangular solve along anti-diagonals, independent per velocity.  Each CTA
// owns kAdjKc consecutive velocities and sweeps the cells of wavefront steps
// [t0, t1) diagonal by diagonal with only block barriers between diagonals.
// A body's faces carry no neighbour term here; their within-cell wall
// coupling is added by k_adjT_body between the steps.
__global__ void __launch_bounds__(256) k_adjT_wave(AdjSweepArgs S, int pass, int t0, int t1)
{
    const LevelDev& L = S.L;
    const VelDev& Vg = S.V;
    const int nx = L.nx, ny = L.ny, nv = Vg.nv;
    const size_t nc = L.nc, snv = nv;
    const int k0 = blockIdx.x * kAdjKc;
    // interior block: pass 0 i <= nx-2, j <= ny-2; pass 1 i >= 1, j >= 1
    const int mx = nx - 1, my = ny - 1;                 // its extent
    if (mx <= 0 || my <= 0) return;
    const int nd = mx + my - 1;
    for (int t = t0; t < min(t1, nd); ++t) {
        const int dd = pass == 0 ? t : nd - 1 - t;      // diagonal within the block
        const int ilo = dd - (my - 1) > 0 ? dd - (my - 1) : 0, ihi = dd < mx - 1 ? dd : mx - 1;
        const int m = ihi - ilo + 1;
        for (int q = threadIdx.x; q < m * kAdjKc; q += blockDim.x) {
            const int kk = q % kAdjKc, k = k0 + kk;
            if (k >= nv) continue;
            const int bi = ilo + q / kAdjKc, bj = dd - bi;
            const int i = pass == 0 ? bi : bi + 1, j = pass == 0 ? bj : bj + 1, c = j * nx + i;
            const double u = Vg.u[k], v = Vg.v[k], rD = S.invD[(size_t)c * snv + k];
            for (int cp = 0; cp < 2; ++cp) {
                const size_t e = (cp * nc + c) * snv + k;
                if (pass == 0) {
                    double b = S.r[e];
                    if (u < 0 && i > 0 && L.fbx[j * (nx + 1) + i] < 0) b -= u * L.rdx[i - 1] * S.y[e - snv];
                    if (v < 0 && j > 0 && L.fby[j * nx + i] < 0) b -= v * L.rdy[j - 1] * S.y[e - (size_t)nx * snv];
                    S.y[e] = b * rD;
                } else {
                    double b = 0.0;
                    if (u > 0 && L.fbx[j * (nx + 1) + i + 1] < 0) b += u * L.rdx[i + 1] * S.x[e + snv];
                    if (v > 0 && L.fby[(j + 1) * nx + i] < 0) b += v * L.rdy[j + 1] * S.x[e + (size_t)nx * snv];
                    S.x[e] = S.y[e] + b * rD;
                }
            }
        }
        __syncthreads();
    }
}

// The wall coupling of a body face in a transposed pass, for one cell per CTA
// (entries cell * 4 + face), after the wavefront has computed the cell's rows
// without it: the incoming rows (u_o < 0 at the face) are final, and each
// outgoing G row gains w u_o s / Z times its inverse diagonal, with
// s = sum over incoming velocities of Db C (y_G + K T_w / 4 y_H) the
// transposed wall-density sum (as in adjT_cell with one wall face).
__global__ void __launch_bounds__(256) k_adjT_body(AdjSweepArgs S, int pass, const int* __restrict__ ent)
{
    __shared__ double red[kRed];
    const LevelDev& L = S.L;
    const VelDev& Vg = S.V;
    const int e = ent[blockIdx.x], c = e >> 2, face = e & 3, nx = L.nx, nv = Vg.nv, i = c % nx, j = c / nx;
    const size_t nc = L.nc, snv = nv;
    const int axis = face >> 1, os = (face & 1) ? 1 : -1;
    const int bid = axis == 0 ? L.fbx[j * (nx + 1) + i + (os > 0)] : L.fby[(j + (os > 0)) * nx + i];
    const double bS = axis == 0 ? L.rdx[i] : L.rdy[j];
    const double Z = S.Zw[bid * 4 + axis * 2 + (os > 0)];
    const double Hf = kKint * S.bc[bid].t / 4.0;
    double* dst = pass == 0 ? S.y : S.x;
    double acc[1] = {0.0};
    for (int k = threadIdx.x; k < nv; k += blockDim.x) {
        const double uo = os * (axis == 0 ? Vg.u[k] : Vg.v[k]);
        if (uo < 0) acc[0] += uo * bS * S.Cw[(size_t)bid * nv + k] * (dst[c * snv + k] + Hf * dst[(nc + c) * snv + k]);
    }
    red_sum<1>(acc, red);                    // ends with a barrier: the incoming rows are read before any write
    const double sZ = acc[0] / Z;
    for (int k = threadIdx.x; k < nv; k += blockDim.x) {
        const double uo = os * (axis == 0 ? Vg.u[k] : Vg.v[k]);
        if (uo > 0) dst[c * snv + k] += Vg.w[k] * uo * sZ * S.invD[c * snv + k];
    }
}

// ---------------------------------------------------------------------------
// y = A^T x on one level: A is the evolution operator of Eq. microFinalDefect
// with every neighbour and every boundary ghost (the operator of the residual
// renewal, Eq. renewResidualMicro).  Row c of A^T collects the coefficient that
// each neighbour's row holds for c, and the transposed within-cell ghost block.
// One CTA per cell.
__global__ void __launch_bounds__(256) k_adjT_apply(AdjSweepArgs S, const double* __restrict__ x,
                                                     double* __restrict__ y)
{
    __shared__ double red[kRed * 4];
    const LevelDev& L = S.L;
    const VelDev& Vg = S.V;
    const int nx = L.nx, ny = L.ny, nv = Vg.nv, tid = threadIdx.x, bs = blockDim.x;
    const size_t nc = L.nc, snv = nv;
    const int c = blockIdx.x, i = c % nx, j = c / nx;
    const double rdx = 1.0 / L.dx[i], rdy = 1.0 / L.dy[j], it = S.inv_tau[c];
    const bool nW = i > 0 && L.fbx[j * (nx + 1) + i] < 0, nE = i < nx - 1 && L.fbx[j * (nx + 1) + i + 1] < 0;
    const bool nS = j > 0 && L.fby[j * nx + i] < 0, nN = j < ny - 1 && L.fby[(j + 1) * nx + i] < 0;
    const double cW = nW ? 1.0 / L.dx[i - 1] : 0.0, cE = nE ? 1.0 / L.dx[i + 1] : 0.0;
    const double cS = nS ? 1.0 / L.dy[j - 1] : 0.0, cN = nN ? 1.0 / L.dy[j + 1] : 0.0;
    int nb = 0, bax[4], bos[4], btype[4], bid[4];
    double bS[4], Z[4], Hf[4];
    auto addb = [&](int ax, int os, int id, double rS) {
        bax[nb] = ax; bos[nb] = os; bid[nb] = id; bS[nb] = rS; btype[nb] = S.bc[id].type;
        Hf[nb] = kKint * S.bc[id].t / 4.0;
        Z[nb] = btype[nb] == BC_WALL ? S.Zw[id * 4 + ax * 2 + (os > 0)] : 0.0;
        ++nb;
    };
    if (i == 0) addb(0, -1, L.fbx[j * (nx + 1)], rdx);
    if (j == 0) addb(1, -1, L.fby[i], rdy);
    if (i == nx - 1) addb(0, 1, L.fbx[j * (nx + 1) + nx], rdx);
    if (j == ny - 1) addb(1, 1, L.fby[ny * nx + i], rdy);
    if (!L.solid[c]) {                          // a body's faces (BC ids inside the domain)
        if (i > 0 && L.fbx[j * (nx + 1) + i] >= 0) addb(0, -1, L.fbx[j * (nx + 1) + i], rdx);
        if (j > 0 && L.fby[j * nx + i] >= 0) addb(1, -1, L.fby[j * nx + i], rdy);
        if (i < nx - 1 && L.fbx[j * (nx + 1) + i + 1] >= 0) addb(0, 1, L.fbx[j * (nx + 1) + i + 1], rdx);
        if (j < ny - 1 && L.fby[(j + 1) * nx + i] >= 0) addb(1, 1, L.fby[(j + 1) * nx + i], rdy);
    }
    auto Db = [&](int b, int k) -> double {
        double uo = bos[b] * (bax[b] == 0 ? Vg.u[k] : Vg.v[k]);
        return uo < 0 ? uo * bS[b] : 0.0;
    };
    // wall sums s_b = sum over velocities incoming at b of Db (C x_G + C Hf x_H)
    double sb[4] = {0, 0, 0, 0};
    for (int k = tid; k < nv; k += bs)
        for (int b = 0; b < nb; ++b) {
            if (btype[b] != BC_WALL) continue;
            double Dbk = Db(b, k);
            if (Dbk != 0.0)
                sb[b] += Dbk * S.Cw[(size_t)bid[b] * nv + k] * (x[c * snv + k] + Hf[b] * x[(nc + c) * snv + k]);
        }
    red_sum<4>(sb, red);
    for (int k = tid; k < nv; k += bs) {
        const double u = Vg.u[k], v = Vg.v[k];
        const double D = it + fabs(u) * rdx + fabs(v) * rdy;
        for (int cp = 0; cp < 2; ++cp) {
            const size_t e = (cp * nc + c) * snv + k;
            double acc = D * x[e];
            if (nW && u < 0) acc += u * cW * x[e - snv];
            if (nE && u > 0) acc -= u * cE * x[e + snv];
            if (nS && v < 0) acc += v * cS * x[e - (size_t)nx * snv];
            if (nN && v > 0) acc -= v * cN * x[e + (size_t)nx * snv];
            for (int b = 0; b < nb; ++b) {
                if (btype[b] == BC_OUTFLOW) { acc += Db(b, k) * x[e]; continue; }
                double uo = bos[b] * (bax[b] == 0 ? u : v);
                if (!(uo > 0)) continue;
                if (btype[b] == BC_WALL) {
                    if (cp == 0) acc += -Vg.w[k] * uo / Z[b] * sb[b];
                } else if (btype[b] == BC_SYMMETRY) {
                    int a = k / Vg.nvv, bb = k - a * Vg.nvv;
                    int km = bax[b] == 0 ? (Vg.nu - 1 - a) * Vg.nvv + bb : a * Vg.nvv + (Vg.nvv - 1 - bb);
                    acc += Db(b, km) * x[(cp * nc + c) * snv + km];
                }
            }
            y[e] = acc;
        }
    }
}

// fine = R^T coarse: R is the volume-weighted restriction of Eq. microRestriction,
// so fine cell j of coarse cell I receives V_j / V_I times coarse_I (2 x nv values per cell)
__global__ void k_adjT_restrict(LevelDev F, LevelDev C, int nv, const double* __restrict__ coarse,
                                double* __restrict__ fine)
{
    const int c = blockIdx.x, i = c % F.nx, j = c / F.nx, I = i / 2, J = j / 2, cc = J * C.nx + I;
    double VI = 0.0;          // sum of the four fine volumes, as the restriction divides by it
    for (int q = 0; q < 4; ++q) VI += F.dx[2 * I + (q & 1)] * F.dy[2 * J + (q >> 1)];
    const double wgt = F.dx[i] * F.dy[j] / VI;
    for (int q = threadIdx.x; q < 2 * nv; q += blockDim.x) {
        const int cp = q / nv, k = q - cp * nv;
        fine[((size_t)cp * F.nc + c) * nv + k] = wgt * coarse[((size_t)cp * C.nc + cc) * nv + k];
    }
}

// coarse = P^T fine: P is the bilinear prolongation (Eq. prolongation); rows of P^T
// are gathered through the inverse stencil (CSR: ptr[I] .. ptr[I+1] of (fine cell, weight))
__global__ void k_adjT_prolong(LevelDev F, LevelDev C, int nv, const int* __restrict__ ptr,
                               const int* __restrict__ cell, const double* __restrict__ wgt,
                               const double* __restrict__ fine, double* __restrict__ coarse)
{
    const int I = blockIdx.x, p0 = ptr[I], p1 = ptr[I + 1];
    for (int q = threadIdx.x; q < 2 * nv; q += blockDim.x) {
        const int cp = q / nv, k = q - cp * nv;
        double acc = 0.0;
        for (int p = p0; p < p1; ++p) acc += wgt[p] * fine[((size_t)cp * F.nc + cell[p]) * nv + k];
        coarse[((size_t)cp * C.nc + I) * nv + k] = acc;
    }
}

// ---------------------------------------------------------------------------
// Wall objective of one face of wall BC bcid: out[4 * m ..] = S Q, S dQ/d(T, u, v)
// at fixed f; dJdf (when not null) += S dQ/df of the face's cell.  Q = shear
// (obj 0), heat flux (1) or pressure (2) of the face distribution (diffuse wall
// with rho_w from zero mass flux).
__global__ void __launch_bounds__(256) k_adj_objective(AdjDev A, int obj, int bcid, const int* __restrict__ faces,
                                                        double* __restrict__ part, double* __restrict__ dJdf)
{
    __shared__ double red[kRed * 8];
    const LevelDev& L = A.L;
    const VelDev& Vg = A.V;
    const int nv = Vg.nv, tid = threadIdx.x, bs = blockDim.x, nx = L.nx;
    const size_t nc = L.nc, snv = nv;
    const int code = faces[blockIdx.x], axis = code >> 30, fi = code & ((1 << 30) - 1);
    int outsign, c;
    double S;
    if (axis == 0) {
        int i = fi % (nx + 1), j = fi / (nx + 1);
        bface_side(L, 0, i, j, c, outsign); S = L.dy[j];
    } else {
        int i = fi % nx, j = fi / nx;
        bface_side(L, 1, i, j, c, outsign); S = L.dx[i];
    }
    const BcDev B = A.bc[bcid];
    const double T = B.t, lam = 1.0 / T, hf = kKint * T / 4.0, Uwt = axis == 0 ? B.v : B.u;
    const double* Cb = A.Cw + (size_t)bcid * nv;
    const double* fG = A.f + c * snv;
    const double* fH = A.f + (nc + c) * snv;
    double s[5] = {0, 0, 0, 0, 0};      // num, den, d den / d(T, u, v)
    for (int k = tid; k < nv; k += bs) {
        double uo = outsign * (axis == 0 ? Vg.u[k] : Vg.v[k]), w = Vg.w[k];
        if (uo > 0) s[0] += w * uo * fG[k];
        else if (uo < 0) {
            double C = Cb[k], du = Vg.u[k] - B.u, dv = Vg.v[k] - B.v;
            s[1] += w * uo * C;
            s[2] += w * uo * C * (lam * lam * (du * du + dv * dv) - lam);
            s[3] += w * uo * C * 2.0 * lam * du;
            s[4] += w * uo * C * 2.0 * lam * dv;
        }
    }
    red_sum<5>(s, red);
    const double rhow = -s[0] / s[1];
    double t[5] = {0, 0, 0, 0, 0};      // Q, dQ/d(T, u, v), rho_w adjoint
    for (int k = tid; k < nv; k += bs) {
        double u = Vg.u[k], v = Vg.v[k], w = Vg.w[k];
        double uo = outsign * (axis == 0 ? u : v), ut = axis == 0 ? v : u;
        double du = u - B.u, dv = v - B.v, cw2 = du * du + dv * dv;
        double aG, aH, da[3] = {0, 0, 0};
        if (obj == 0) { aG = ut - Uwt; aH = 0.0; da[axis == 0 ? 2 : 1] = -1.0; }
        else if (obj == 1) { aG = 0.5 * cw2; aH = 1.0; da[1] = -du; da[2] = -dv; }
        else { aG = uo; aH = 0.0; }
        double wk = w * uo;
        if (uo >= 0) {
            t[0] += wk * (aG * fG[k] + aH * fH[k]);
            for (int p = 0; p < 3; ++p) t[1 + p] += wk * da[p] * fG[k];
            if (dJdf) {
                atomicAdd(dJdf + c * snv + k, S * wk * aG);
                atomicAdd(dJdf + (nc + c) * snv + k, S * wk * aH);
            }
        } else {
            double C = Cb[k];
            double dC[3] = {C * (lam * lam * cw2 - lam), C * 2.0 * lam * du, C * 2.0 * lam * dv};
            double a = aG + aH * hf;
            t[0] += wk * rhow * C * a;
            t[4] += wk * C * a;
            for (int p = 0; p < 3; ++p) {
                double drho = -rhow / s[1] * s[2 + p];
                double dap = da[p] + (p == 0 ? aH * kKint / 4.0 : 0.0);
                t[1 + p] += wk * (drho * C * a + rhow * dC[p] * a + rhow * C * dap);
            }
        }
    }
    red_sum<5>(t, red);
    if (dJdf)
        for (int k = tid; k < nv; k += bs) {
            double uo = outsign * (axis == 0 ? Vg.u[k] : Vg.v[k]);
            if (uo > 0) atomicAdd(dJdf + c * snv + k, -S * Vg.w[k] * uo * t[4] / s[1]);
        }
    if (tid == 0)
        for (int p = 0; p < 4; ++p) part[4 * (size_t)blockIdx.x + p] = S * t[p];
}

// lambda . dN/dtheta of one face of wall BC bcid, theta = (T, u, v): out[3 * m + p]
__global__ void __launch_bounds__(256) k_adj_dtheta(AdjDev A, int bcid, const int* __restrict__ faces,
                                                     const double* __restrict__ lam_, double* __restrict__ part)
{
    __shared__ double red[kRed * 4];
    const LevelDev& L = A.L;
    const VelDev& Vg = A.V;
    const int nv = Vg.nv, tid = threadIdx.x, bs = blockDim.x, nx = L.nx;
    const size_t nc = L.nc, snv = nv;
    const int code = faces[blockIdx.x], axis = code >> 30, fi = code & ((1 << 30) - 1);
    int outsign, c;
    double h;
    if (axis == 0) {
        int i = fi % (nx + 1), j = fi / (nx + 1);
        bface_side(L, 0, i, j, c, outsign); h = L.dx[c % nx];
    } else {
        int i = fi % nx, j = fi / nx;
        bface_side(L, 1, i, j, c, outsign); h = L.dy[c / nx];
    }
    const BcDev B = A.bc[bcid];
    const double T = B.t, lam = 1.0 / T, coef = -outsign / h;
    const double* Cb = A.Cw + (size_t)bcid * nv;
    double s[5] = {0, 0, 0, 0, 0};
    for (int k = tid; k < nv; k += bs) {
        double uo = outsign * (axis == 0 ? Vg.u[k] : Vg.v[k]), w = Vg.w[k];
        if (uo > 0) s[0] += w * uo * A.f[c * snv + k];
        else if (uo < 0) {
            double C = Cb[k], du = Vg.u[k] - B.u, dv = Vg.v[k] - B.v;
            s[1] += w * uo * C;
            s[2] += w * uo * C * (lam * lam * (du * du + dv * dv) - lam);
            s[3] += w * uo * C * 2.0 * lam * du;
            s[4] += w * uo * C * 2.0 * lam * dv;
        }
    }
    red_sum<5>(s, red);
    const double rhow = -s[0] / s[1];
    double t[4] = {0, 0, 0, 0};
    for (int k = tid; k < nv; k += bs) {
        double un = axis == 0 ? Vg.u[k] : Vg.v[k], uo = outsign * un;
        if (!(uo < 0)) continue;
        double C = Cb[k], du = Vg.u[k] - B.u, dv = Vg.v[k] - B.v;
        double dC[3] = {C * (lam * lam * (du * du + dv * dv) - lam), C * 2.0 * lam * du, C * 2.0 * lam * dv};
        double lG = lam_[c * snv + k], lH = lam_[(nc + c) * snv + k];
        for (int p = 0; p < 3; ++p) {
            double drho = -rhow / s[1] * s[2 + p];
            double dG = drho * C + rhow * dC[p];
            double dH = dG * kKint * T / 4.0 + (p == 0 ? rhow * C * kKint / 4.0 : 0.0);
            t[p] += coef * un * (lG * dG + lH * dH);
        }
    }
    red_sum<4>(t, red);
    if (tid == 0)
        for (int p = 0; p < 3; ++p) part[3 * (size_t)blockIdx.x + p] = t[p];
}

// ---------------------------------------------------------------------------
// vector kernels of the Krylov solve (fixed reduction order: deterministic)

// part[b * m + q] = partial dot products of w with the m basis vectors V_q over block b's range
__global__ void __launch_bounds__(256) k_multi_dot(const double* __restrict__ Vb, int m, size_t n,
                                                    const double* __restrict__ w, double* __restrict__ part)
{
    __shared__ double red[kRed];
    const size_t per = (n + gridDim.x - 1) / gridDim.x;
    const size_t lo = blockIdx.x * per, hi = lo + per < n ? lo + per : n;
    for (int q = 0; q < m; ++q) {
        double s[1] = {0.0};
        const double* v = Vb + (size_t)q * n;
        for (size_t e = lo + threadIdx.x; e < hi; e += blockDim.x) s[0] += v[e] * w[e];
        red_sum<1>(s, red);
        if (threadIdx.x == 0) part[(size_t)blockIdx.x * m + q] = s[0];
    }
}

// w = a * w + sum_q h[q] V_q  (h in constant-size argument array)
struct Coef32 { double h[33]; };
__global__ void k_multi_axpy(const double* __restrict__ Vb, int m, size_t n, Coef32 h, double a,
                             double* __restrict__ w)
{
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        double acc = a * w[e];
        for (int q = 0; q < m; ++q) acc += h.h[q] * Vb[(size_t)q * n + e];
        w[e] = acc;
    }
}

// mass weights dot product: part[b] = sum over block b's cells of V_c sum_k w_k x_G
__global__ void __launch_bounds__(256) k_mass_dot(LevelDev L, VelDev Vg, const double* __restrict__ x,
                                                   double* __restrict__ part)
{
    __shared__ double red[kRed];
    const int c = blockIdx.x, i = c % L.nx, j = c / L.nx;
    double s[1] = {0.0};
    for (int k = threadIdx.x; k < Vg.nv; k += blockDim.x) s[0] += Vg.w[k] * x[(size_t)c * Vg.nv + k];
    red_sum<1>(s, red);
    if (threadIdx.x == 0) part[c] = L.dx[i] * L.dy[j] * s[0];
}

// m_c = (dr_c / dW~_c)^T y_c: how the micro residual r = (g~(W~, q) - f) / tau(W~) of a cell
// moves with its predicted state W~ (q held), contracted with y.  One CTA per cell.
__global__ void __launch_bounds__(256) k_adj_macro_m(AdjDev A, const double* __restrict__ y, double* __restrict__ m)
{
    __shared__ double red[kRed * 6];
    const VelDev& Vg = A.V;
    const int nv = Vg.nv, tid = threadIdx.x, bs = blockDim.x, c = blockIdx.x;
    const size_t nc = A.L.nc, snv = nv;
    if (A.L.solid[c]) {                          // no equation in a body
        if (tid < 4) m[4 * (size_t)c + tid] = 0.0;
        return;
    }
    const double* fG = A.f + c * snv;
    const double* fH = A.f + (nc + c) * snv;
    const double* yG = y + c * snv;
    const double* yH = y + (nc + c) * snv;
    const double* W = A.W + 4 * (size_t)c;
    const double* q = A.q + 2 * (size_t)c;
    double rho, U, V, lam;
    adj_prim(W, rho, U, V, lam);
    const double T = 1.0 / lam;
    const double itau = 1.0 / (A.gas.mu_ref * pow(T, A.gas.omega) / (0.5 * rho * T));
    const double S = (1.0 - A.gas.pr) * 4.0 / 5.0 * lam * lam / rho;
    double r[6] = {0, 0, 0, 0, 0, 0};       // rho, U, V, lam, S, itau adjoints
    for (int k = tid; k < nv; k += bs) {
        double u = Vg.u[k], v = Vg.v[k];
        double cx = u - U, cy = v - V, c2 = cx * cx + cy * cy;
        double gM = adj_maxw(rho, U, V, lam, u, v), hM = gM * kKint / (4.0 * lam);
        double Fq = S * (cx * q[0] + cy * q[1]);
        double eG = 2.0 * lam * c2 - 4.0, eH = 2.0 * lam * c2 - 2.0;
        double gP = gM * (1.0 + Fq * eG), hP = hM * (1.0 + Fq * eH);
        double a = yG[k], b = yH[k];
        r[5] += a * (gP - fG[k]) + b * (hP - fH[k]);
        double gPb = a * itau, hPb = b * itau;
        double gMb = gPb * (1.0 + Fq * eG), hMb = hPb * (1.0 + Fq * eH);
        double Fqb = gPb * gM * eG + hPb * hM * eH;
        double eb = (gPb * gM + hPb * hM) * Fq;
        r[3] += eb * 2.0 * c2;
        double c2b = eb * 2.0 * lam;
        r[4] += Fqb * (cx * q[0] + cy * q[1]);
        r[1] -= Fqb * S * q[0] + 2.0 * cx * c2b;
        r[2] -= Fqb * S * q[1] + 2.0 * cy * c2b;
        adj_maxw_rev(gM, hM, rho, lam, cx, cy, gMb, hMb, r[0], r[1], r[2], r[3]);
    }
    red_sum<6>(r, red);
    if (tid == 0) {
        double rb = r[0], lb = r[3];
        lb += r[4] * 2.0 * S / lam;
        rb -= r[4] * S / rho;
        rb += r[5] * itau / rho;
        lb += r[5] * itau * (A.gas.omega - 1.0) / lam;
        double Wb[4] = {0, 0, 0, 0};
        adj_prim_rev(W, rb, r[1], r[2], lb, Wb);
        for (int q2 = 0; q2 < 4; ++q2) m[4 * (size_t)c + q2] = Wb[q2];
    }
}

// out -= Pi^T w: the moment weights of every velocity times the cell's 4-vector w
__global__ void k_adj_macro_spread(LevelDev L, VelDev Vg, const double* __restrict__ w, double* __restrict__ out)
{
    const int c = blockIdx.x;
    const size_t nc = L.nc, snv = Vg.nv;
    const double w0 = w[4 * (size_t)c], w1 = w[4 * (size_t)c + 1], w2 = w[4 * (size_t)c + 2], w3 = w[4 * (size_t)c + 3];
    for (int k = threadIdx.x; k < Vg.nv; k += blockDim.x) {
        const double u = Vg.u[k], v = Vg.v[k], wk = Vg.w[k];
        out[c * snv + k] -= wk * (w0 + u * w1 + v * w2 + 0.5 * (u * u + v * v) * w3);
        out[(nc + c) * snv + k] -= wk * w3;
    }
}

// partial sums of sum_c V_c w_c[0] (the closed-domain null direction of the transposed
// split Euler Jacobian: total mass is conserved by every state)
__global__ void __launch_bounds__(256) k_macro_null_dot(LevelDev L, const double* __restrict__ w, double* __restrict__ part)
{
    __shared__ double red[kRed];
    double s[1] = {0.0};
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < L.nc; c += gridDim.x * blockDim.x) {
        const int i = c % L.nx, j = c / L.nx;
        s[0] += L.dx[i] * L.dy[j] * w[4 * (size_t)c];
    }
    red_sum<1>(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

// w_c[0] -= coef V_c
__global__ void k_macro_null_sub(LevelDev L, double coef, double* __restrict__ w)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= L.nc) return;
    w[4 * (size_t)c] -= coef * L.dx[c % L.nx] * L.dy[c / L.nx];
}

// z_c = binv_c r_c (4x4 blocks)
__global__ void k_block_apply(int nc, const double* __restrict__ binv, const double* __restrict__ r,
                              double* __restrict__ z)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    const double* B = binv + 16 * (size_t)c;
    const double* x = r + 4 * (size_t)c;
    for (int a = 0; a < 4; ++a) z[4 * (size_t)c + a] = B[a * 4] * x[0] + B[a * 4 + 1] * x[1] + B[a * 4 + 2] * x[2] + B[a * 4 + 3] * x[3];
}

// x = 0 in the cells of bodies (2 x nc x nv values)
__global__ void k_zero_solid(LevelDev L, int nv, double* __restrict__ x)
{
    const size_t n = 2 * (size_t)L.nc * nv;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const size_t c = (e / nv) % L.nc;
        if (L.solid[c]) x[e] = 0.0;
    }
}
cudaError_t launch_zero_solid(const LevelDev& L, int nv, double* x, cudaStream_t st)
{
    k_zero_solid<<<1216, 256, 0, st>>>(L, nv, x);
    return cudaGetLastError();
}

template <typename F>
__global__ void k_to_double(const F* __restrict__ a, double* __restrict__ b, size_t n)
{
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        b[e] = (double)a[e];
}

// 1 / (1/tau_c + |u_k|/dx + |v_k|/dy) per (cell, velocity) of one level
__global__ void k_adj_invD(LevelDev L, VelDev Vg, const double* __restrict__ it, double* __restrict__ invD)
{
    const int c = blockIdx.x, i = c % L.nx, j = c / L.nx;
    const double rdx = 1.0 / L.dx[i], rdy = 1.0 / L.dy[j];
    for (int k = threadIdx.x; k < Vg.nv; k += blockDim.x)
        invD[(size_t)c * Vg.nv + k] = 1.0 / (it[c] + fabs(Vg.u[k]) * rdx + fabs(Vg.v[k]) * rdy);
}

__global__ void k_inv_tau_of(GasDev gas, const double* __restrict__ W, int nc, double* __restrict__ it)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    double rho, U, V, lam;
    adj_prim(W + 4 * (size_t)c, rho, U, V, lam);
    double T = 1.0 / lam;
    it[c] = 1.0 / (gas.mu_ref * pow(T, gas.omega) / (0.5 * rho * T));
}

// ---------------------------------------------------------------------------
// launchers

cudaError_t launch_adjoint_residual(const AdjDev& A, const double* mu, double* recx, double* recy, double* crec,
                                    double pen, double* out, cudaStream_t st)
{
    const size_t etab = (size_t)(A.V.nu + A.V.nvv) * sizeof(double);
    const size_t cache = etab + 4 * (size_t)A.V.nv * sizeof(double);
    if (cache <= kAdjCacheBytes) {
        cudaError_t e = cudaFuncSetAttribute(k_adj_face<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kAdjCacheBytes);
        if (e != cudaSuccess) return e;
        k_adj_face<true><<<A.L.nfx, 256, cache, st>>>(A, 0, mu, recx);
        k_adj_face<true><<<A.L.nfy, 256, cache, st>>>(A, 1, mu, recy);
    } else {
        k_adj_face<false><<<A.L.nfx, 256, etab, st>>>(A, 0, mu, recx);
        k_adj_face<false><<<A.L.nfy, 256, etab, st>>>(A, 1, mu, recy);
    }
    k_adj_cell<<<A.L.nc, 256, 0, st>>>(A, mu, crec);
    dim3 grid(A.L.nc, (A.V.nv + 127) / 128);
    k_adj_gather<<<grid, 128, 0, st>>>(A, mu, recx, recy, crec, pen, out);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_sgs(const AdjSweepArgs& S, const AdjBodyPlan& P, cudaStream_t st)
{
    const size_t smem = 2 * (size_t)S.V.nv * sizeof(double);
    if (S.V.nv > kMaxAdjNv) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_adjT_chain, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         2 * kMaxAdjNv * (int)sizeof(double));
    if (e != cudaSuccess) return e;
    const int nblk = (S.V.nv + kAdjKc - 1) / kAdjKc;
    for (int pass = 0; pass < 2; ++pass) {
        int t = 0;
        for (int g = 0; g < P.ngroups[pass]; ++g) {     // stop after each step that reaches a body face
            const int ts = P.step[pass][g], n = P.off[pass][g + 1] - P.off[pass][g];
            k_adjT_wave<<<nblk, 256, 0, st>>>(S, pass, t, ts + 1);
            k_adjT_body<<<n, 256, 0, st>>>(S, pass, P.cells[pass] + P.off[pass][g]);
            t = ts + 1;
        }
        k_adjT_wave<<<nblk, 256, 0, st>>>(S, pass, t, INT_MAX);
        k_adjT_chain<<<2, 512, smem, st>>>(S, pass, 0);
        k_adjT_chain<<<1, 512, smem, st>>>(S, pass, 1);
    }
    return cudaGetLastError();
}

cudaError_t launch_adjoint_apply(const AdjSweepArgs& S, const double* x, double* y, cudaStream_t st)
{
    k_adjT_apply<<<S.L.nc, 256, 0, st>>>(S, x, y);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_restrict_t(const LevelDev& F, const LevelDev& C, int nv, const double* coarse,
                                      double* fine, cudaStream_t st)
{
    k_adjT_restrict<<<F.nc, 256, 0, st>>>(F, C, nv, coarse, fine);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_prolong_t(const LevelDev& F, const LevelDev& C, int nv, const int* ptr, const int* cell,
                                     const double* wgt, const double* fine, double* coarse, cudaStream_t st)
{
    k_adjT_prolong<<<C.nc, 256, 0, st>>>(F, C, nv, ptr, cell, wgt, fine, coarse);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_objective(const AdjDev& A, int obj, int bcid, const int* faces, int nfaces, double* part,
                                     double* dJdf, cudaStream_t st)
{
    if (nfaces > 0) k_adj_objective<<<nfaces, 256, 0, st>>>(A, obj, bcid, faces, part, dJdf);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_dtheta(const AdjDev& A, int bcid, const int* faces, int nfaces, const double* lam,
                                  double* part, cudaStream_t st)
{
    if (nfaces > 0) k_adj_dtheta<<<nfaces, 256, 0, st>>>(A, bcid, faces, lam, part);
    return cudaGetLastError();
}

cudaError_t launch_multi_dot(const double* Vb, int m, size_t n, const double* w, double* part, int nblk,
                             cudaStream_t st)
{
    k_multi_dot<<<nblk, 256, 0, st>>>(Vb, m, n, w, part);
    return cudaGetLastError();
}

cudaError_t launch_multi_axpy(const double* Vb, int m, size_t n, const double* h, double a, double* w,
                              cudaStream_t st)
{
    Coef32 c{};
    for (int q = 0; q < m && q < 33; ++q) c.h[q] = h[q];
    k_multi_axpy<<<1216, 256, 0, st>>>(Vb, m, n, c, a, w);
    return cudaGetLastError();
}

cudaError_t launch_mass_dot(const LevelDev& L, const VelDev& V, const double* x, double* part, cudaStream_t st)
{
    k_mass_dot<<<L.nc, 256, 0, st>>>(L, V, x, part);
    return cudaGetLastError();
}

template <typename F>
cudaError_t launch_to_double(const F* a, double* b, size_t n, cudaStream_t st)
{
    k_to_double<F><<<1216, 256, 0, st>>>(a, b, n);
    return cudaGetLastError();
}
template cudaError_t launch_to_double<float>(const float*, double*, size_t, cudaStream_t);
template cudaError_t launch_to_double<double>(const double*, double*, size_t, cudaStream_t);

__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b, size_t n)
{
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        b[e] = (float)a[e];
}
cudaError_t launch_to_float(const double* a, float* b, size_t n, cudaStream_t st)
{
    k_to_float<<<1216, 256, 0, st>>>(a, b, n);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_macro_m(const AdjDev& A, const double* y, double* m, cudaStream_t st)
{
    k_adj_macro_m<<<A.L.nc, 256, 0, st>>>(A, y, m);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_macro_spread(const LevelDev& L, const VelDev& V, const double* w, double* out,
                                        cudaStream_t st)
{
    k_adj_macro_spread<<<L.nc, 256, 0, st>>>(L, V, w, out);
    return cudaGetLastError();
}

cudaError_t launch_macro_null_dot(const LevelDev& L, const double* w, double* part, int nblk, cudaStream_t st)
{
    k_macro_null_dot<<<nblk, 256, 0, st>>>(L, w, part);
    return cudaGetLastError();
}

cudaError_t launch_macro_null_sub(const LevelDev& L, double coef, double* w, cudaStream_t st)
{
    k_macro_null_sub<<<(L.nc + 127) / 128, 128, 0, st>>>(L, coef, w);
    return cudaGetLastError();
}

cudaError_t launch_block_apply(int nc, const double* binv, const double* r, double* z, cudaStream_t st)
{
    k_block_apply<<<(nc + 127) / 128, 128, 0, st>>>(nc, binv, r, z);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_invD(const LevelDev& L, const VelDev& V, const double* it, double* invD, cudaStream_t st)
{
    k_adj_invD<<<L.nc, 256, 0, st>>>(L, V, it, invD);
    return cudaGetLastError();
}

cudaError_t launch_inv_tau(const GasDev& gas, const double* W, int nc, double* it, cudaStream_t st)
{
    k_inv_tau_of<<<(nc + 127) / 128, 128, 0, st>>>(gas, W, nc, it);
    return cudaGetLastError();
}

} // namespace miugks
