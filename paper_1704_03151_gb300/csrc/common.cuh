// common.cuh -- device-side model functions and shared types of the MIUGKS
// CUDA library (arXiv 1704.03151).  Units: R = 1/2, lambda = 1/T, p = rho T / 2;
// 2-D monatomic gas with one internal degree of freedom carried by the reduced
// distributions G (comp 0) and H (comp 1).
#pragma once
#include <cuda_runtime.h>
#include <cooperative_groups.h>
#include <stdint.h>

namespace miugks {

constexpr int kKint = 1;                       // internal degrees of freedom
constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxLevels = 8;
constexpr int kMaxBcs = 64;                    // boundary conditions per solver
constexpr int kMaxLine = 512;                  // longest grid line (cells) of the micro sweep kernels

enum BcType { BC_WALL = 0, BC_SYMMETRY = 1, BC_FARFIELD = 2, BC_OUTFLOW = 3 };

struct BcDev { int type; double rho, u, v, t; };

// velocity space: k = a * nvv + b, u_k = ua[a], v_k = vb[b]
struct VelDev {
    int nu, nvv, nv;
    const double *u, *v, *w;     // per discrete velocity
    const double *ua, *vb;       // per-axis nodes
    const float *uf, *vf, *wf;   // u, v, w rounded to FP32 (for the mixed-precision kernels)
    double umax, vmax;           // largest |u|, |v|
    // Coupling classes of the evolution sweep, per pass (0 forward, 1 backward),
    // from the signs of u and v: the blocks of four consecutive velocities that
    // hold a velocity coupled to both its x and its y upwind neighbour (swept as
    // a wavefront), and every other velocity, listed as those coupled along rows
    // only, along columns only, and to no neighbour (in that order in lk)
    const int* wblk[2];
    int nwblk[2];
    const int* lk[2];
    int nrow[2], ncol[2], nelem[2];
};

// one grid level (all device pointers)
struct LevelDev {
    int nx, ny, nc, nfx, nfy;
    const double *xn, *yn, *xc, *yc, *dx, *dy;
    const int *fbx, *fby;        // face BC id, -1 interior (or inactive: no fluid cell on either side)
    const double *rdx, *rdy;     // 1/dx, 1/dy
    const unsigned char* solid;  // per cell: 1 inside a body (no state, never updated)
    const int* ubc;              // fluid cells with a boundary face on the east or north side
    int nubc;
};

// The fluid cell of boundary x-face (axis 0, i in 0..nx) or y-face (axis 1,
// j in 0..ny) and the sign of the face's outward normal seen from it: the face
// lies on the domain edge or between a fluid cell and a body.
__device__ __forceinline__ void bface_side(const LevelDev& L, int axis, int i, int j, int& c, int& outsign)
{
    const int nx = L.nx;
    if (axis == 0) {
        const bool lo = i > 0 && !L.solid[j * nx + i - 1];
        c = lo ? j * nx + i - 1 : j * nx + i;
        outsign = lo ? 1 : -1;
    } else {
        const bool lo = j > 0 && !L.solid[(j - 1) * nx + i];
        c = lo ? (j - 1) * nx + i : j * nx + i;
        outsign = lo ? 1 : -1;
    }
}
// a face without a BC id that does not join two fluid cells (inside a body)
__device__ __forceinline__ bool inactive_face(const LevelDev& L, int axis, int i, int j)
{
    const int nx = L.nx;
    if (axis == 0) return i == 0 || i == nx || L.solid[j * nx + i - 1] || L.solid[j * nx + i];
    return j == 0 || j == L.ny || L.solid[(j - 1) * nx + i] || L.solid[j * nx + i];
}

struct GasDev { double mu_ref, omega, pr; };

// per-velocity nodes and weights in the arithmetic type
template <typename F> struct VelT;
template <> struct VelT<double> {
    static __device__ __forceinline__ const double* u(const VelDev& V) { return V.u; }
    static __device__ __forceinline__ const double* v(const VelDev& V) { return V.v; }
    static __device__ __forceinline__ const double* w(const VelDev& V) { return V.w; }
};
template <> struct VelT<float> {
    static __device__ __forceinline__ const float* u(const VelDev& V) { return V.uf; }
    static __device__ __forceinline__ const float* v(const VelDev& V) { return V.vf; }
    static __device__ __forceinline__ const float* w(const VelDev& V) { return V.wf; }
};


// ---------------------------------------------------------------------------
// gas model
__device__ __forceinline__ void prim4(const double* W, double& rho, double& U, double& V, double& lam)
{
    rho = W[0];
    double ir = 1.0 / W[0];
    U = W[1] * ir;
    V = W[2] * ir;
    double eint = W[3] - 0.5 * (W[1] * U + W[2] * V);
    lam = (kKint + 2) * rho / (4.0 * eint);
}

__device__ __forceinline__ double tau_of(const GasDev& g, double rho, double lam)
{
    double T = 1.0 / lam;
    return g.mu_ref * pow(T, g.omega) / (0.5 * rho * T);
}
// the same in FP32 (mixed-precision face scalars)
__device__ __forceinline__ float tau_of_f(const GasDev& g, float rho, float lam)
{
    float T = 1.0f / lam;
    return (float)g.mu_ref * powf(T, (float)g.omega) / (0.5f * rho * T);
}

// Time integrals of the UGKS integral solution over [0, dt] (x = dt/tau):
// q[0..4] multiply g0, u_n a g0, A g0, f0, u_n sigma.  Series in x below 1.
__device__ __forceinline__ void time_coeffs(double dt, double tau, double q[5])
{
    double x = dt / tau;
    if (x < 1.0) {
        // Horner-free explicit sums of the power series, terms x^n / n!
        double pn = 1.0;             // x^n / n!
        double s1 = 0, s2 = 0, s3 = 0, s4 = 0, s5 = 0;
        #pragma unroll 1
        for (int n = 0; n < 26; ++n) {
            double sg = (n & 1) ? -1.0 : 1.0;
            s4 += sg * pn / (n + 1);                      // (-1)^n x^n/(n+1)!
            // m = n + 1 terms use x^{m-1}/(m-1)! = pn
            int m = n + 1;
            s5 += -sg * pn / (m + 1);                     // (-1)^m m x^{m-1}/(m+1)! = (-1)^m x^{m-1}/((m+1) (m-1)!)
            if (m >= 2) s2 += -sg * (1.0 - m) * pn / ((double)m * (m + 1));
            double pn1 = pn * x / (n + 1);                // x^{n+1}/(n+1)!
            // n+1 >= 1 terms of q1, q3
            s1 += sg * pn1 / (n + 2);                     // (-1)^{n+2} x^{n+1}/(n+2)!
            s3 += sg * pn1 / ((double)(n + 2) * (n + 3));
            pn = pn1;
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

// moments dw (already divided by rho) -> slope coefficients of a Maxwellian at (U, V, lam)
template <typename T>
__device__ __forceinline__ void micro_slope_t(const T dw[4], T U, T V, T lam, T a[4])
{
    const T Kp2 = T(kKint + 2.0);
    T c = U * U + V * V + Kp2 / (T(2) * lam);
    T R4 = T(2) * dw[3] - c * dw[0];
    T R3 = dw[2] - V * dw[0];
    T R2 = dw[1] - U * dw[0];
    a[3] = T(4) * lam * lam / Kp2 * (R4 - T(2) * U * R2 - T(2) * V * R3);
    a[2] = T(2) * lam * R3 - V * a[3];
    a[1] = T(2) * lam * R2 - U * a[3];
    a[0] = dw[0] - U * a[1] - V * a[2] - T(0.5) * a[3] * c;
}
__device__ __forceinline__ void micro_slope(const double dw[4], double U, double V, double lam, double a[4])
{
    micro_slope_t<double>(dw, U, V, lam, a);
}

// Reciprocal by the Newton-Raphson iteration y <- y + y (1 - x y) (quadratic
// convergence) from a single-precision seed: two steps take the 24-bit seed to
// double precision (within 1 ulp of 1/x).  Outside the seed's exponent range
// the IEEE division is used.
__device__ __forceinline__ double rcp64(double x)
{
    double ax = fabs(x);
    if (!(ax > 1e-30 && ax < 1e30)) return 1.0 / x;
    double y = (double)__frcp_rn((float)x);
    double e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    e = fma(-x, y, 1.0);
    return fma(y, e, y);
}

template <typename T>
__device__ __forceinline__ T van_leer(T s1, T s2)
{
    T p = s1 * s2;
    return p > T(0) ? T(2) * p / (s1 + s2) : T(0);
}

// ---------------------------------------------------------------------------
// Per-thread accumulator of velocity sums: plain FP64 in the FP64 form, a
// Kahan-compensated FP32 sum in the mixed form (its value is taken in FP64).
template <typename T> struct Acc;
template <> struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct Acc<float> {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x)
    {
        float y = x - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// ---------------------------------------------------------------------------
// deterministic block reduction of N doubles (fixed tree order); every thread
// receives the result.  scratch: at least 32 * N doubles of shared memory.
template <int N>
__device__ __forceinline__ void block_sum(double (&v)[N], double* scratch)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    #pragma unroll
    for (int q = 0; q < N; ++q) {
        double x = v[q];
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        v[q] = x;
    }
    __syncthreads();
    if (lane == 0) {
        #pragma unroll
        for (int q = 0; q < N; ++q) scratch[warp * N + q] = v[q];
    }
    __syncthreads();
    #pragma unroll
    for (int q = 0; q < N; ++q) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += scratch[w * N + q];
        v[q] = s;
    }
    __syncthreads();
}

// Block reduction of per-thread velocity sums into FP64 totals, broadcast to
// every thread.  FP64 form: FP64 shuffle tree per warp.  Mixed form: each warp
// reduces its Kahan pairs as float-float numbers (error-free TwoSum in FP32),
// then warp 0 alone adds the per-warp totals in FP64.  scratch: 32 * N doubles.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

template <int N>
__device__ __forceinline__ void block_total(Acc<float> (&a)[N], double* scratch, double (&out)[N])
{
    // float-float pairs all the way; one conversion to FP64 per value at the end
    // (an FP64 instruction costs a warp as much as thirty-two lanes of it)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    float* fs = reinterpret_cast<float*>(scratch);    // [32][N][2] per-warp pairs
    #pragma unroll
    for (int q = 0; q < N; ++q) {
        float hi = a[q].s, lo = -a[q].c;
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            float h2 = __shfl_xor_sync(0xffffffffu, hi, o), l2 = __shfl_xor_sync(0xffffffffu, lo, o);
            float s, e;
            two_sum(hi, h2, s, e);
            lo = lo + l2 + e;
            hi = s;
        }
        if (lane == 0) { fs[(warp * N + q) * 2] = hi; fs[(warp * N + q) * 2 + 1] = lo; }
    }
    __syncthreads();
    if (warp == 0) {
        #pragma unroll
        for (int q = 0; q < N; ++q) {
            float hi = lane < nw ? fs[(lane * N + q) * 2] : 0.0f, lo = lane < nw ? fs[(lane * N + q) * 2 + 1] : 0.0f;
            #pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                float h2 = __shfl_xor_sync(0xffffffffu, hi, o), l2 = __shfl_xor_sync(0xffffffffu, lo, o);
                float s, e;
                two_sum(hi, h2, s, e);
                lo = lo + l2 + e;
                hi = s;
            }
            if (lane == q) scratch[32 * N - N + q] = (double)hi + (double)lo;
        }
    }
    __syncthreads();
    #pragma unroll
    for (int q = 0; q < N; ++q) out[q] = scratch[32 * N - N + q];
    __syncthreads();
}

template <int N>
__device__ __forceinline__ void block_total(Acc<double> (&a)[N], double* scratch, double (&out)[N])
{
    #pragma unroll
    for (int q = 0; q < N; ++q) out[q] = a[q].s;
    block_sum<N>(out, scratch);
}

} // namespace miugks
