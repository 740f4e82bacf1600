// flux.cu -- Step 1 of the MIUGKS iteration (arXiv 1704.03151, Sec. 2.1):
// time-averaged UGKS interface fluxes of every discrete velocity (Eqs.
// macroResidualCalc, microResidualDef) and the macroscopic residual R
// (Eq. macroResidualDef), plus its RMS (Eq. Residual_Def).
//
// One CTA per face; threads stride over the discrete velocities, which are
// contiguous in memory ([comp][cell][k]), so every load of f is coalesced.
// The three velocity reductions a face needs (interface state W0; heat flux
// and time slope; macroscopic flux) are deterministic block reductions.  The
// equilibrium at the face is evaluated from separable per-axis exponential
// tables (Nu + Nv exponentials per face instead of Nu * Nv).
#include "kernels.cuh"

namespace miugks {
namespace cg = cooperative_groups;

// Sum of N per-CTA totals over the CTAs of a cluster (one face split over its
// CTAs by velocity), in rank order: every thread of every CTA gets the same
// value.  slots: N doubles of this CTA's shared memory, one set per reduction.
template <int N>
__device__ __forceinline__ void cluster_total(cg::cluster_group& cl, double (&v)[N], double* slots)
{
    const int nb = (int)cl.num_blocks();
    if (nb == 1) return;
    if (threadIdx.x == 0)
        #pragma unroll
        for (int q = 0; q < N; ++q) slots[q] = v[q];
    cl.sync();
    #pragma unroll
    for (int q = 0; q < N; ++q) {
        double t = 0.0;
        for (int r = 0; r < nb; ++r) t += cl.map_shared_rank(slots, r)[q];
        v[q] = t;
    }
}

__constant__ double c_series[5][28];   // power-series coefficients of the time integrals
__constant__ float c_series_f[5][28];  // the same rounded to FP32

void upload_series_coefficients()
{
    // q1/dt  = sum_{n>=1} (-1)^{n+1} x^n/(n+1)!
    // q2/dt2 = sum_{n>=1} (-1)^n n x^n/(n+2)!
    // q3/dt2 = sum_{n>=1} (-1)^{n+1} x^n/(n+2)!
    // q4/dt  = sum_{n>=0} (-1)^n x^n/(n+1)!
    // q5/dt2 = sum_{n>=0} (-1)^{n+1} (n+1) x^n/(n+2)!
    double c[5][28] = {};
    double fact[32];
    fact[0] = 1.0;
    for (int n = 1; n < 32; ++n) fact[n] = fact[n - 1] * n;
    for (int n = 0; n < 28; ++n) {
        double s = (n % 2) ? -1.0 : 1.0;                 // (-1)^n
        c[0][n] = n >= 1 ? -s / fact[n + 1] : 0.0;
        c[1][n] = n >= 1 ? s * n / fact[n + 2] : 0.0;
        c[2][n] = n >= 1 ? -s / fact[n + 2] : 0.0;
        c[3][n] = s / fact[n + 1];
        c[4][n] = -s * (n + 1) / fact[n + 2];
    }
    cudaMemcpyToSymbol(c_series, c, sizeof c);
    float cf[5][28];
    for (int m = 0; m < 5; ++m)
        for (int n = 0; n < 28; ++n) cf[m][n] = (float)c[m][n];
    cudaMemcpyToSymbol(c_series_f, cf, sizeof cf);
}

__device__ __forceinline__ void time_coeffs_fast(double dt, double tau, double q[5])
{
    double x = dt / tau;
    if (x < 1.0) {
        double s[5];
        #pragma unroll
        for (int m = 0; m < 5; ++m) {
            double acc = c_series[m][27];
            #pragma unroll
            for (int n = 26; n >= 0; --n) acc = fma(acc, x, c_series[m][n]);
            s[m] = acc;
        }
        q[0] = dt * s[0];
        q[1] = dt * dt * s[1];
        q[2] = dt * dt * s[2];
        q[3] = dt * s[3];
        q[4] = dt * dt * s[4];
    } else {
        time_coeffs(dt, tau, q);
    }
}

// one of the five time integrals (series below x = dt/tau = 1, closed form above)
__device__ __forceinline__ double time_coeff_one(double dt, double tau, int m)
{
    double x = dt / tau;
    if (x < 1.0) {
        double acc = c_series[m][27];
        #pragma unroll
        for (int n = 26; n >= 0; --n) acc = fma(acc, x, c_series[m][n]);
        return (m == 0 || m == 3) ? dt * acc : dt * dt * acc;
    }
    double e = exp(-x), E1 = -expm1(-x);
    switch (m) {
    case 0: return dt - tau * E1;
    case 1: return -tau * dt * (1.0 + e) + 2.0 * tau * tau * E1;
    case 2: return 0.5 * dt * dt - tau * dt + tau * tau * E1;
    case 3: return tau * E1;
    default: return tau * dt * e - tau * tau * E1;
    }
}

// FP32 form of time_coeff_one (mixed-precision face scalars)
__device__ __forceinline__ float time_coeff_one_f(float dt, float tau, int m)
{
    float x = dt / tau;
    if (x < 1.0f) {
        float acc = c_series_f[m][27];
        #pragma unroll
        for (int n = 26; n >= 0; --n) acc = fmaf(acc, x, c_series_f[m][n]);
        return (m == 0 || m == 3) ? dt * acc : dt * dt * acc;
    }
    float e = expf(-x), E1 = -expm1f(-x);
    switch (m) {
    case 0: return dt - tau * E1;
    case 1: return -tau * dt * (1.0f + e) + 2.0f * tau * tau * E1;
    case 2: return 0.5f * dt * dt - tau * dt + tau * tau * E1;
    case 3: return tau * E1;
    default: return tau * dt * e - tau * tau * E1;
    }
}

// van Leer limited slope 2 s1 s2 / (s1 + s2) when s1 s2 > 0, else 0
__device__ __forceinline__ double vl_limited(double s1, double s2)
{
    double p = s1 * s2;
    return p > 0.0 ? 2.0 * p * rcp64(s1 + s2) : 0.0;
}
__device__ __forceinline__ float vl_limited(float s1, float s2)
{
    float p = s1 * s2;   // s1 + s2 has no cancellation here; the fast quotient is within 2 ulp
    return p > 0.0f ? __fdividef(2.0f * p, s1 + s2) : 0.0f;
}

// (a . psi) g split into the reduced components: b gM + a4 hM and b hM + a4 <xi^4>/4 gM
template <typename F>
__device__ __forceinline__ void slope_mom(const F* a, F u, F v, F gM, F hM, F xi4q, F& mG, F& mH)
{
    F b = a[0] + a[1] * u + a[2] * v + F(0.5) * a[3] * (u * u + v * v);
    mG = b * gM + a[3] * hM;
    mH = b * hM + a[3] * xi4q * gM;
}

// Per-velocity arithmetic runs in F (FP64, or FP32 in the mixed form); the
// velocity sums are FP64 (or Kahan-compensated FP32) per thread and combined in
// FP64; the per-face scalars (interface state, slopes, time integrals) are FP64.
// CACHE keeps the upwinded face values and slopes of every velocity in shared
// memory between the three velocity passes; without it (a velocity grid too
// large for shared memory in FP64) the later passes recompute them from f with
// the same arithmetic.
//
// A face may be split over the CTAs of a cluster (launched with a cluster
// dimension): each CTA takes a contiguous chunk of the velocities and caches
// only its chunk, and the three velocity reductions add the CTAs' totals in
// rank order through distributed shared memory.  Boundary faces and faces
// inside a body are done by rank 0 alone.
template <typename F, bool CACHE>
__global__ void __launch_bounds__(256, sizeof(F) == 4 ? 4 : 2) k_face_flux(FaceFluxArgs<F> A)
{
    extern __shared__ double sm[];
    cg::cluster_group cl = cg::this_cluster();
    const int ncl = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    const LevelDev& L = A.L;
    const VelDev& Vg = A.V;
    const int nv = Vg.nv, tid = threadIdx.x, bs = blockDim.x;
    const int axis = A.axis, fi = blockIdx.x / ncl;
    const int chunk = (nv + ncl - 1) / ncl, kb = rank * chunk, ke = min(nv, kb + chunk);
    const int nx = L.nx, ny = L.ny;
    const size_t nc = L.nc, nf = axis == 0 ? L.nfx : L.nfy;
    double* red = sm;                       // 32 * 8
    double* par = red + 256;                // face scalars (FP64), [48]; cluster slots at 48..63
    F* pf = reinterpret_cast<F*>(par + 64); // face constants in F, [64]
    F* f0s = reinterpret_cast<F*>(par + 128);  // [2][chunk] (CACHE)
    F* sgs = f0s + (CACHE ? 2 * chunk : 0); // [2][chunk] (CACHE)
    F* Eu = sgs + (CACHE ? 2 * chunk : 0);  // [nu]
    F* Ev = Eu + Vg.nu;                     // [nvv]
    const int i = axis == 0 ? fi % (nx + 1) : fi % nx;
    const int j = axis == 0 ? fi / (nx + 1) : fi / nx;
    const int bcid = (axis == 0 ? L.fbx : L.fby)[fi];
    const F* __restrict__ fG = A.f;
    const F* __restrict__ fH = A.f + nc * nv;
    F* __restrict__ phG = A.ph + (size_t)fi * nv;
    F* __restrict__ phH = A.ph + (nf + fi) * (size_t)nv;

    if (bcid >= 0) {
        if (rank != 0) return;
        // ---------------- boundary face: free transport of the face distribution
        int outsign, c;
        bface_side(L, axis, i, j, c, outsign);
        const BcDev B = A.bc[bcid];
        const double* Cb = A.Cw + (size_t)bcid * nv;
        const double Hfac = kKint * B.t / 4.0;   // K / (4 lambda_b)
        double rhow = B.rho;
        if (B.type == BC_WALL) {
            double s[2] = {0.0, 0.0};
            for (int k = tid; k < nv; k += bs) {
                double uo = outsign * (axis == 0 ? Vg.u[k] : Vg.v[k]);
                if (uo > 0) s[0] += Vg.w[k] * uo * (double)fG[c * (size_t)nv + k];
                else if (uo < 0) s[1] += Vg.w[k] * uo * Cb[k];
            }
            block_sum<2>(s, red);
            rhow = -s[0] / s[1];
        }
        double Fm[4] = {0, 0, 0, 0};
        for (int k = tid; k < nv; k += bs) {
            double un = axis == 0 ? Vg.u[k] : Vg.v[k];
            double uo = outsign * un;
            double g, h;
            if (uo >= 0 || B.type == BC_OUTFLOW) {
                g = fG[c * (size_t)nv + k]; h = fH[c * (size_t)nv + k];
            } else if (B.type == BC_SYMMETRY) {
                int a = k / Vg.nvv, b = k - a * Vg.nvv;
                int km = axis == 0 ? (Vg.nu - 1 - a) * Vg.nvv + b : a * Vg.nvv + (Vg.nvv - 1 - b);
                g = fG[c * (size_t)nv + km]; h = fH[c * (size_t)nv + km];
            } else {   // wall (rho_w C) or farfield (rho_inf C)
                g = rhow * Cb[k]; h = g * Hfac;
            }
            double pg = un * g, ph = un * h;
            phG[k] = (F)pg; phH[k] = (F)ph;
            double u = Vg.u[k], v = Vg.v[k], w = Vg.w[k];
            Fm[0] += w * pg; Fm[1] += w * u * pg; Fm[2] += w * v * pg;
            Fm[3] += w * (0.5 * (u * u + v * v) * pg + ph);
        }
        block_sum<4>(Fm, red);
        if (tid == 0)
            for (int m = 0; m < 4; ++m) A.Fm[4 * (size_t)fi + m] = Fm[m];
        return;
    }

    if (inactive_face(L, axis, i, j)) {   // inside a body: no flux
        if (rank != 0) return;
        for (int k = tid; k < nv; k += bs) { phG[k] = F(0); phH[k] = F(0); }
        if (tid == 0)
            for (int m = 0; m < 4; ++m) A.Fm[4 * (size_t)fi + m] = 0.0;
        return;
    }
    // ---------------- interior face between cL (lower) and cR (upper)
    // Face constants are computed once (by one thread or one lane each) and
    // broadcast through shared memory as F: an FP64 instruction occupies a
    // GB300 SM sub-partition for as long for one lane as for thirty-two.
    const F* __restrict__ vu = VelT<F>::u(Vg);
    const F* __restrict__ vv = VelT<F>::v(Vg);
    const F* __restrict__ vw = VelT<F>::w(Vg);
    int cL, cR, cLL = -1, cRR = -1;
    if (axis == 0) {
        cL = j * nx + i - 1; cR = cL + 1;
        if (i - 1 > 0 && L.fbx[fi - 1] < 0) cLL = cL - 1;
        if (i + 1 < nx && L.fbx[fi + 1] < 0) cRR = cR + 1;
    } else {
        cL = (j - 1) * nx + i; cR = cL + nx;
        if (j - 1 > 0 && L.fby[fi - nx] < 0) cLL = cL - nx;
        if (j + 1 < ny && L.fby[fi + nx] < 0) cRR = cR + nx;
    }
    // the face's mesh constants (kFluxGeo): par[32..40] in FP64, the first five also in F
    if (tid < kFluxGeo - 1) {
        const double gv = A.geo[(size_t)fi * kFluxGeo + tid];
        par[32 + tid] = gv;
        if (tid < 5) pf[tid] = (F)gv;
    }
    __syncthreads();
    const F r1 = pf[0], r2 = pf[1], r3 = pf[2], fhL = pf[3], fhR = pf[4];
    // van Leer reconstruction and upwinding of velocity k: face value f0 and slope sg of G and H
    auto recon = [&](int k, F (&f0)[2], F (&sg)[2]) {
        const F un = axis == 0 ? vu[k] : vv[k];
        #pragma unroll
        for (int cp = 0; cp < 2; ++cp) {
            const F* fc = cp == 0 ? fG : fH;
            F fL = fc[cL * (size_t)nv + k], fR = fc[cR * (size_t)nv + k];
            F d2 = (fR - fL) * r2;
            F sL = cLL >= 0 ? vl_limited((fL - fc[cLL * (size_t)nv + k]) * r1, d2) : F(0);
            F sR = cRR >= 0 ? vl_limited(d2, (fc[cRR * (size_t)nv + k] - fR) * r3) : F(0);
            F faceL = fL + sL * fhL, faceR = fR - sR * fhR;
            if (un > F(0)) { f0[cp] = faceL; sg[cp] = sL; }
            else if (un < F(0)) { f0[cp] = faceR; sg[cp] = sR; }
            else { f0[cp] = F(0.5) * (faceL + faceR); sg[cp] = F(0.5) * (sL + sR); }
        }
    };
    auto face_vals = [&](int k, F (&f0)[2], F (&sg)[2]) {
        if constexpr (CACHE) {
            const int e = k - kb;
            f0[0] = f0s[e]; f0[1] = f0s[chunk + e]; sg[0] = sgs[e]; sg[1] = sgs[chunk + e];
        } else {
            recon(k, f0, sg);
        }
    };

    // pass 1: reconstruction, upwinding, interface conservative variables
    // (unrolled so that the loads of the next velocity are in flight with this one's arithmetic)
    Acc<F> W0a[4];
    #pragma unroll 2
    for (int k = kb + tid; k < ke; k += bs) {
        F f0[2], sg[2];
        recon(k, f0, sg);
        if constexpr (CACHE) {
            const int e = k - kb;
            f0s[e] = f0[0]; f0s[chunk + e] = f0[1];
            sgs[e] = sg[0]; sgs[chunk + e] = sg[1];
        }
        const F w = vw[k], u = vu[k], v = vv[k], g = f0[0];
        W0a[0].add(w * g); W0a[1].add(w * u * g); W0a[2].add(w * v * g);
        W0a[3].add(w * (F(0.5) * (u * u + v * v) * g + f0[1]));
    }
    double W0[4];
    block_total<4>(W0a, red, W0);
    cluster_total<4>(cl, W0, par + 48);
    // face scalars, spread over the lanes of warp 0: lane 0 the collision time and
    // time step, lanes 1 and 2 the left and right equilibrium slopes
    if (tid < 3) {
        double rho = W0[0], ir = rcp64(rho);
        double U = W0[1] * ir, V = W0[2] * ir;
        double lam = (kKint + 2) * rho * rcp64(4.0 * (W0[3] - 0.5 * (W0[1] * U + W0[2] * V)));
        if (tid == 0) {
            par[0] = rho; par[1] = U; par[2] = V; par[3] = lam;
            if constexpr (sizeof(F) == 8) par[4] = tau_of(A.gas, rho, lam);
            else par[4] = (double)tau_of_f(A.gas, (float)rho, (float)lam);
            par[5] = par[37];
            if (A.shock) {
                double rl, ul, vl, ll, rr, ur, vr, lr;
                prim4(A.W + 4 * (size_t)cL, rl, ul, vl, ll);
                prim4(A.W + 4 * (size_t)cR, rr, ur, vr, lr);
                const double pl = rl / (2.0 * ll), pr = rr / (2.0 * lr);
                par[4] += par[5] * fabs(pl - pr) / (pl + pr);
            }
        } else {
            const double* Wc = A.W + 4 * (size_t)(tid == 1 ? cL : cR);
            double hf, dw[4];
            if constexpr (sizeof(F) == 8) hf = (tid == 1 ? 1.0 : -1.0) * ir * rcp64(tid == 1 ? par[35] : par[36]);
            else hf = (tid == 1 ? 1.0 : -1.0) * ir * (tid == 1 ? par[39] : par[40]);
            for (int m = 0; m < 4; ++m) dw[m] = (W0[m] - Wc[m]) * hf;
            if constexpr (sizeof(F) == 8) {
                micro_slope(dw, U, V, lam, par + (tid == 1 ? 8 : 12));
            } else {
                float dwf[4] = {(float)dw[0], (float)dw[1], (float)dw[2], (float)dw[3]}, af[4];
                micro_slope_t<float>(dwf, (float)U, (float)V, (float)lam, af);
                for (int m = 0; m < 4; ++m) par[(tid == 1 ? 8 : 12) + m] = af[m];
            }
        }
    }
    __syncthreads();
    {
        // warp 0: constants of the equilibrium in F; the other warps: the per-axis exponentials
        const double rho0 = par[0], U0 = par[1], V0 = par[2], lam0 = par[3];
        if (tid < 32) {
            F val = F(0);
            if (tid < 8) val = (F)par[8 + tid];          // aL, aR
            else if (tid == 8) val = (F)U0;
            else if (tid == 9) val = (F)V0;
            else if constexpr (sizeof(F) == 8) {
                if (tid == 10) val = rho0 * lam0 / kPi;
                else if (tid == 11) val = kKint / (4.0 * lam0);
                else if (tid == 12) val = kKint * (kKint + 2.0) / (16.0 * lam0 * lam0);
            } else {                                      // FP32 constants need no FP64 division
                const float fl = (float)lam0;
                if (tid == 10) val = (float)rho0 * fl * (float)(1.0 / kPi);
                else if (tid == 11) val = (float)(kKint / 4.0) / fl;
                else if (tid == 12) val = (float)(kKint * (kKint + 2.0) / 16.0) / (fl * fl);
            }
            if (tid < 13) pf[8 + tid] = val;
        } else {
            for (int e = tid - 32; e < Vg.nu + Vg.nvv; e += bs - 32) {
                const bool isu = e < Vg.nu;
                const double d = isu ? Vg.ua[e] - U0 : Vg.vb[e - Vg.nu] - V0;
                F ex;
                if constexpr (sizeof(F) == 8) {
                    ex = exp(-lam0 * d * d);
                } else {
                    const float df = (float)d;
                    ex = expf(-(float)lam0 * df * df);
                }
                (isu ? Eu[e] : Ev[e - Vg.nu]) = ex;
            }
        }
    }
    __syncthreads();
    const F fU0 = pf[16], fV0 = pf[17], gnorm = pf[18], hfac = pf[19], xi4q = pf[20];
    F aL[4], aR[4];
    #pragma unroll
    for (int m = 0; m < 4; ++m) { aL[m] = pf[8 + m]; aR[m] = pf[12 + m]; }

    // velocity k = a * nvv + b of this thread, stepped by the block size without a division
    const int ka0 = (kb + tid) / Vg.nvv, kb0 = kb + tid - ka0 * Vg.nvv;
    const int sa = bs / Vg.nvv, sb = bs - sa * Vg.nvv;
    // pass 2: heat flux of the interface distribution, compatibility moments for A
    Acc<F> s6a[6];
    for (int k = kb + tid, a = ka0, b = kb0; k < ke; k += bs, a += sa, b += sb) {
        if (b >= Vg.nvv) { b -= Vg.nvv; ++a; }
        const F u = vu[k], v = vv[k], w = vw[k];
        F cx = u - fU0, cy = v - fV0, c2 = cx * cx + cy * cy;
        F f0[2], sg[2];
        face_vals(k, f0, sg);
        F e = F(0.5) * c2 * f0[0] + f0[1];
        s6a[0].add(w * cx * e);
        s6a[1].add(w * cy * e);
        F un = axis == 0 ? u : v;
        if (un != F(0)) {
            F gM = gnorm * Eu[a] * Ev[b], hM = gM * hfac, mG, mH;
            slope_mom<F>(un > F(0) ? aL : aR, u, v, gM, hM, xi4q, mG, mH);
            F wu = w * un;
            s6a[2].add(wu * mG); s6a[3].add(wu * u * mG); s6a[4].add(wu * v * mG);
            s6a[5].add(wu * (F(0.5) * (u * u + v * v) * mG + mH));
        }
    }
    double s6[6];
    block_total<6>(s6a, red, s6);
    cluster_total<6>(cl, s6, par + 52);
    // lane 0: time slope A from compatibility; lanes 1-5: one time integral each
    if (tid < 6) {
        const double rho0 = par[0], U0 = par[1], V0 = par[2], lam0 = par[3];
        if (tid == 0) {
            double dwt[4], ir = -rcp64(rho0);
            for (int m = 0; m < 4; ++m) dwt[m] = s6[2 + m] * ir;
            if constexpr (sizeof(F) == 8) {
                micro_slope(dwt, U0, V0, lam0, par + 16);
            } else {
                float dwf[4] = {(float)dwt[0], (float)dwt[1], (float)dwt[2], (float)dwt[3]}, af[4];
                micro_slope_t<float>(dwf, (float)U0, (float)V0, (float)lam0, af);
                for (int m = 0; m < 4; ++m) par[16 + m] = af[m];
            }
            par[6] = s6[0]; par[7] = s6[1];
        } else {
            if constexpr (sizeof(F) == 8) par[20 + tid - 1] = time_coeff_one(par[5], par[4], tid - 1);
            else par[20 + tid - 1] = time_coeff_one_f((float)par[5], (float)par[4], tid - 1);
        }
    }
    __syncthreads();
    if (tid < 32) {
        const double rho0 = par[0], lam0 = par[3];
        F val = F(0);
        if (tid < 4) val = (F)par[16 + tid];             // A
        else if (tid < 9) val = (F)(par[20 + tid - 4] * par[38]);   // q_i / dt
        else if (tid == 9) {
            if constexpr (sizeof(F) == 8) val = (1.0 - A.gas.pr) * 4.0 * lam0 * lam0 / (5.0 * rho0);
            else val = (float)((1.0 - A.gas.pr) * 0.8) * ((float)lam0 * (float)lam0) / (float)rho0;
        }
        else if (tid == 10) val = (F)par[6];
        else if (tid == 11) val = (F)par[7];
        else if (tid == 12) val = (F)(2.0 * lam0);
        if (tid < 13) pf[24 + tid] = val;
    }
    __syncthreads();
    F As[4];
    #pragma unroll
    for (int m = 0; m < 4; ++m) As[m] = pf[24 + m];
    const F q1 = pf[28], q2 = pf[29], q3 = pf[30], q4 = pf[31], q5 = pf[32];
    const F shk = pf[33], qx = pf[34], qy = pf[35], flam2 = pf[36];

    // pass 3: time-averaged flux of every discrete velocity and its moments
    Acc<F> Fa[4];
    for (int k = kb + tid, a = ka0, b = kb0; k < ke; k += bs, a += sa, b += sb) {
        if (b >= Vg.nvv) { b -= Vg.nvv; ++a; }
        const F u = vu[k], v = vv[k], w = vw[k];
        const F un = axis == 0 ? u : v;
        F cx = u - fU0, cy = v - fV0, c2 = cx * cx + cy * cy;
        F gM = gnorm * Eu[a] * Ev[b], hM = gM * hfac;
        F Fq = shk * (cx * qx + cy * qy);
        F gP = gM * (F(1) + Fq * (flam2 * c2 - F(4)));
        F hP = hM * (F(1) + Fq * (flam2 * c2 - F(2)));
        F mGa, mHa, mGA, mHA;
        slope_mom<F>(un > F(0) ? aL : aR, u, v, gM, hM, xi4q, mGa, mHa);
        slope_mom<F>(As, u, v, gM, hM, xi4q, mGA, mHA);
        F f0[2], sg[2];
        face_vals(k, f0, sg);
        F pg = un * (q1 * gP + q2 * un * mGa + q3 * mGA + q4 * f0[0] + q5 * un * sg[0]);
        F ph = un * (q1 * hP + q2 * un * mHa + q3 * mHA + q4 * f0[1] + q5 * un * sg[1]);
        phG[k] = pg; phH[k] = ph;
        Fa[0].add(w * pg); Fa[1].add(w * u * pg); Fa[2].add(w * v * pg);
        Fa[3].add(w * (F(0.5) * (u * u + v * v) * pg + ph));
    }
    double Fm[4];
    block_total<4>(Fa, red, Fm);
    cluster_total<4>(cl, Fm, par + 58);
    if (tid == 0 && rank == 0)
        for (int m = 0; m < 4; ++m) A.Fm[4 * (size_t)fi + m] = Fm[m];
    if (ncl > 1) cl.sync();   // the other CTAs' slots stay alive until every remote read is done
}

template <typename F>
size_t face_flux_smem(const VelDev& V, bool cache, int ncl)
{
    const size_t chunk = ((size_t)V.nv + ncl - 1) / ncl;
    return sizeof(double) * (256 + 128) + sizeof(F) * ((cache ? 4 * chunk : 0) + V.nu + V.nvv);
}

template <typename F>
cudaError_t launch_face_flux(const FaceFluxArgs<F>& a, cudaStream_t st)
{
    constexpr size_t kSmemMax = 227 * 1024;
    // the cache pays while it leaves room for several CTAs per SM: a face is split
    // over a cluster of 1, 2, 4 or 8 CTAs until each CTA's chunk fits in 64 KB;
    // beyond that the recomputing variant (a few KB) is used
    constexpr size_t kCacheMax = 64 * 1024;
    int ncl = 1;
    while (ncl < 8 && face_flux_smem<F>(a.V, true, ncl) > kCacheMax) ncl *= 2;
    // In FP32 a face that needs a cluster for its cache (the 89^2 grid) runs faster as one CTA
    // that recomputes the reconstruction in each pass (square cylinder: 8.7 against 11.8 ms of flux
    // per iteration); with one CTA per face the cache wins (64^2 cavity 0.34 against 0.42 ms, flat
    // plate 1.48 against 2.08 ms).  FP64 keeps the cluster split: recomputing costs FP64 issue.
    const bool cache = face_flux_smem<F>(a.V, true, ncl) <= kCacheMax && (sizeof(F) == 8 || ncl == 1);
    if (!cache) ncl = 1;
    const size_t smem = face_flux_smem<F>(a.V, cache, ncl);
    if (smem > kSmemMax) return cudaErrorInvalidValue;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_face_flux<F, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kSmemMax);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_face_flux<F, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    int nf = a.axis == 0 ? a.L.nfx : a.L.nfy;
    // FP32 with a small velocity grid: 128 threads, so that more faces (CTAs) overlap their serial
    // scalar phases on an SM (64^2 cavity, 32^2 velocities: 0.27 against 0.34 ms of flux per
    // iteration); with 48^2 or more velocities 256 threads are faster (flat plate 1.48 against
    // 1.72 ms, square cylinder 8.7 against 9.6 ms)
    int threads = (a.V.nv / ncl < 256 || (sizeof(F) == 4 && a.V.nv / ncl <= 1536)) ? 128 : 256;
    if (!cache) {
        k_face_flux<F, false><<<nf, threads, smem, st>>>(a);
        return cudaGetLastError();
    }
    if (ncl == 1) {
        k_face_flux<F, true><<<nf, threads, smem, st>>>(a);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nf * ncl), 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)ncl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_face_flux<F, true>, a);
}
template cudaError_t launch_face_flux<double>(const FaceFluxArgs<double>&, cudaStream_t);
template cudaError_t launch_face_flux<float>(const FaceFluxArgs<float>&, cudaStream_t);

// R_i = -(1/V_i) sum_j S_ij F_ij
__global__ void k_cell_residual(LevelDev L, const double* __restrict__ Fx, const double* __restrict__ Fy,
                                double* __restrict__ R)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= L.nc) return;
    int i = c % L.nx, j = c / L.nx;
    if (L.solid[c]) {
        for (int m = 0; m < 4; ++m) R[4 * (size_t)c + m] = 0.0;
        return;
    }
    double V = L.dx[i] * L.dy[j];
    const double* FW = Fx + 4 * (size_t)(j * (L.nx + 1) + i);
    const double* FE = FW + 4;
    const double* FS = Fy + 4 * (size_t)(j * L.nx + i);
    const double* FN = Fy + 4 * (size_t)((j + 1) * L.nx + i);
    for (int m = 0; m < 4; ++m)
        R[4 * (size_t)c + m] = -(L.dy[j] * (FE[m] - FW[m]) + L.dx[i] * (FN[m] - FS[m])) / V;
}

cudaError_t launch_cell_residual(const LevelDev& L, const double* Fx, const double* Fy, double* R, cudaStream_t st)
{
    k_cell_residual<<<(L.nc + 127) / 128, 128, 0, st>>>(L, Fx, Fy, R);
    return cudaGetLastError();
}

// sum of squares of R per component: per-block partials, then one block
// partial sums of R^2 per component and the count of unphysical cells
// (non-positive density or internal energy, or NaN) per CTA
__global__ void k_rms_partial(const double* __restrict__ R, const double* __restrict__ W, int nc,
                              double* __restrict__ part)
{
    __shared__ double red[32 * 5];
    double s[5] = {0, 0, 0, 0, 0};
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        for (int m = 0; m < 4; ++m) s[m] += R[4 * (size_t)c + m] * R[4 * (size_t)c + m];
        const double* w = W + 4 * (size_t)c;
        // rho e_int = E - |m|^2 / (2 rho), tested as rho E - |m|^2 / 2 > 0 with rho > 0
        const double e2 = w[3] * w[0] - 0.5 * (w[1] * w[1] + w[2] * w[2]);
        if (!(w[0] > 0.0) || !(e2 > 0.0)) s[4] += 1.0;
    }
    block_sum<5>(s, red);
    if (threadIdx.x == 0)
        for (int m = 0; m < 5; ++m) part[5 * blockIdx.x + m] = s[m];
}

__global__ void k_rms_final(const double* __restrict__ part, int nblk, int nfluid, double* __restrict__ out)
{
    __shared__ double red[32 * 5];
    double s[5] = {0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblk; b += blockDim.x)
        for (int m = 0; m < 5; ++m) s[m] += part[5 * b + m];
    block_sum<5>(s, red);
    if (threadIdx.x == 0) {
        for (int m = 0; m < 4; ++m) out[m] = sqrt(s[m] / nfluid);
        out[4] = s[4];
    }
}

// RMS over the fluid cells (R is zero in bodies)
cudaError_t launch_rms(const double* R, const double* W, int nc, int nfluid, double* part, double* out, cudaStream_t st)
{
    int nblk = 64;
    k_rms_partial<<<nblk, 256, 0, st>>>(R, W, nc, part);
    k_rms_final<<<1, 64, 0, st>>>(part, nblk, nfluid, out);
    return cudaGetLastError();
}

} // namespace miugks
