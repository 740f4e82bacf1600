// micro.cu -- evolution step of MIUGKS (arXiv 1704.03151, Secs. 2.1.2, 2.3,
// 2.4, 3.2): the microscopic residual with the predicted equilibrium (Eq.
// microResidualDef, Shakhov equilibrium), the upwind implicit operator (Eqs.
// microUpwind, microFinalDefect, evolutionCoefficients), its LU-SGS smoother,
// the residual renewal of the CS cycle (Eq. renewResidualMicro), and the
// moment update (Steps 6-7).
//
// LU-SGS on the GPU.  The sweep order is the serial lexicographic one; every
// cell depends only on its two lower (forward) or upper (backward) neighbours,
// so anti-diagonals can run in parallel.  Discrete velocities are independent
// except at boundary cells, where the diffuse-wall ghost (Eq. delta_f_on_wall)
// couples the incoming velocities of a cell to a sum over its outgoing ones.
// On the lower side (forward sweep) the boundary cells form two lines, the
// first column and the first row, and each line only depends on itself; the
// same holds for the last column and row in the backward sweep.  At a line
// cell, the velocities leaving through the boundary face (outgoing) need no
// ghost, and the incoming ones need only the cell's wall density, a sum over
// the outgoing ones.  Each sweep is therefore two launches:
//   * k_sgs_chain: one thread-block cluster per boundary line solves the
//     corner cell, then every outgoing velocity along the line, then the wall
//     density of every line cell (partial sums combined through distributed
//     shared memory with one hardware cluster barrier);
//   * k_sgs_wave: every CTA owns a contiguous chunk of discrete velocities and
//     sweeps all cells diagonal by diagonal, with only __syncthreads between
//     diagonals (no grid-wide synchronisation); the incoming velocities of
//     line cells are ordinary updates there, their ghost term being known.
#include "kernels.cuh"
#include "async.cuh"
#include <algorithm>
#include <climits>

namespace cg = cooperative_groups;

namespace miugks {

constexpr int kChainCluster = 8;
constexpr int kChainThreads = 128;    // 4 warps: one per SM sub-partition
constexpr int kChainKptMax = 16;      // local velocities per thread in the chain kernel (at most)
constexpr int kInteriorKc = 4;        // velocities per CTA in the wavefront kernel
constexpr size_t kSweepSplitMinCv = 20u << 20;   // cell-velocity pairs of a level from which the sweep is split

// asynchronous 4- or 8-byte global -> shared copies (LDGSTS), completed per commit group
template <typename F>
__device__ __forceinline__ void cp_async_elem(F* sdst, const F* gsrc)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    if constexpr (sizeof(F) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gsrc) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
// wait until at most n (0..7) of this thread's most recent groups are pending
__device__ __forceinline__ void cp_async_wait(int n)
{
    switch (n) {
    case 0: asm volatile("cp.async.wait_group 0;\n" ::: "memory"); break;
    case 1: asm volatile("cp.async.wait_group 1;\n" ::: "memory"); break;
    case 2: asm volatile("cp.async.wait_group 2;\n" ::: "memory"); break;
    case 3: asm volatile("cp.async.wait_group 3;\n" ::: "memory"); break;
    case 4: asm volatile("cp.async.wait_group 4;\n" ::: "memory"); break;
    case 5: asm volatile("cp.async.wait_group 5;\n" ::: "memory"); break;
    case 6: asm volatile("cp.async.wait_group 6;\n" ::: "memory"); break;
    default: asm volatile("cp.async.wait_group 7;\n" ::: "memory"); break;
    }
}

constexpr int kWaveRingMax = 8;       // cells or diagonals of inputs in flight in the sweep kernels (at most)

// (1/V) sum over the faces with u_n > 0 of u_n S = |u|/dx + |v|/dy
template <typename F>
__device__ __forceinline__ F geomD(const LevelDev& L, int i, int j, F u, F v)
{
    return fabs(u) * (F)L.rdx[i] + fabs(v) * (F)L.rdy[j];
}
template <typename F>
__device__ __forceinline__ F geomD_r(F rdxi, F rdyj, F u, F v)
{
    return fabs(u) * rdxi + fabs(v) * rdyj;
}

// coefficient (1/V) u_n S of a neighbour (or ghost) through the face with outward normal
// outsign * e_axis, zero unless u_n < 0; rS = S/V = 1/dx (x-faces) or 1/dy (y-faces)
template <typename F>
__device__ __forceinline__ F Dface(int axis, int outsign, F rS, F u, F v)
{
    F un = (axis == 0 ? u : v);
    un = outsign < 0 ? -un : un;
    return un < F(0) ? un * rS : F(0);
}

__device__ __forceinline__ double recip(double x) { return rcp64(x); }
__device__ __forceinline__ float recip(float x) { return 1.0f / x; }

// ---------------------------------------------------------------------------
// Steps 3-4 on the finest level
template <typename F>
__global__ void __launch_bounds__(256) k_micro_residual(MicroArgs M, GasDev gas, const double* __restrict__ Wt,
                                                        const double* __restrict__ q, const F* __restrict__ f,
                                                        const F* __restrict__ phx, const F* __restrict__ phy,
                                                        double dtn_inv, double* __restrict__ inv_tau,
                                                        F* __restrict__ invD, F* __restrict__ r)
{
    extern __shared__ double sm[];
    const LevelDev& L = M.L;
    const VelDev& Vg = M.V;
    const int c = blockIdx.x, nv = Vg.nv, nx = L.nx;
    const int i = c % nx, j = c / nx;
    const size_t nc = L.nc;
    // cell constants: FP64 state from thread 0, then one constant per lane of warp 0
    // (an FP64 instruction costs a warp as much as thirty-two lanes of it)
    double* cs = sm;                            // cell scalars (FP64), [8]
    F* cf = reinterpret_cast<F*>(sm + 8);       // cell constants in F, [16]
    F* Eu = reinterpret_cast<F*>(sm + 24);
    F* Ev = Eu + Vg.nu;
    if (threadIdx.x == 0) {
        double rho, U, V, lam;
        prim4(Wt + 4 * (size_t)c, rho, U, V, lam);
        double it;
        if constexpr (sizeof(F) == 8) it = 1.0 / tau_of(gas, rho, lam);
        else it = (double)(1.0f / tau_of_f(gas, (float)rho, (float)lam));
        cs[0] = rho; cs[1] = U; cs[2] = V; cs[3] = lam; cs[4] = it;
        inv_tau[c] = it + dtn_inv;
    }
    __syncthreads();
    {
        const double rho = cs[0], U = cs[1], V = cs[2], lam = cs[3], itau = cs[4];
        const int t = threadIdx.x;
        if (t < 32) {
            F val = F(0);
            switch (t) {
            case 0: val = (F)(rho * lam / kPi); break;
            case 1: val = (F)(kKint / (4.0 * lam)); break;
            case 2: val = (F)(2.0 * lam); break;
            case 3: val = (F)((1.0 - gas.pr) * 4.0 * lam * lam / (5.0 * rho)); break;
            case 4: val = (F)q[2 * (size_t)c]; break;
            case 5: val = (F)q[2 * (size_t)c + 1]; break;
            case 6: val = (F)U; break;
            case 7: val = (F)V; break;
            case 8: val = (F)L.rdx[i]; break;
            case 9: val = (F)L.rdy[j]; break;
            case 10: val = (F)itau; break;
            case 11: val = (F)(itau + dtn_inv); break;
            default: break;
            }
            if (t < 12) cf[t] = val;
        } else {
            for (int e = t - 32; e < Vg.nu + Vg.nvv; e += blockDim.x - 32) {
                const bool isu = e < Vg.nu;
                const double d = isu ? Vg.ua[e] - U : Vg.vb[e - Vg.nu] - V;
                F ex;
                if constexpr (sizeof(F) == 8) ex = exp(-lam * d * d);
                else ex = expf((float)(-lam * d * d));
                (isu ? Eu[e] : Ev[e - Vg.nu]) = ex;
            }
        }
    }
    __syncthreads();
    const F gnorm = cf[0], hfac = cf[1], flam2 = cf[2], shk = cf[3], qx = cf[4], qy = cf[5], fU = cf[6], fV = cf[7];
    const F rdxi = cf[8], rdyj = cf[9], fitau = cf[10], fdiag = cf[11];
    const F* __restrict__ vu = VelT<F>::u(Vg);
    const F* __restrict__ vv = VelT<F>::v(Vg);
    const size_t nfx = L.nfx, nfy = L.nfy;
    const size_t fW = (size_t)j * (nx + 1) + i, fE = fW + 1, fS = (size_t)j * nx + i, fN = (size_t)(j + 1) * nx + i;
    const bool body = L.solid[c];   // cells in a body: zero residual
    for (int k = threadIdx.x; k < nv; k += blockDim.x) {
        int a = k / Vg.nvv, b = k - a * Vg.nvv;
        const F u = vu[k], v = vv[k];
        F cx = u - fU, cy = v - fV, c2 = cx * cx + cy * cy;
        F gM = gnorm * Eu[a] * Ev[b], hM = gM * hfac;
        F Fq = shk * (cx * qx + cy * qy);
        F gt[2] = {gM * (F(1) + Fq * (flam2 * c2 - F(4))), hM * (F(1) + Fq * (flam2 * c2 - F(2)))};
        #pragma unroll
        for (int cp = 0; cp < 2; ++cp) {
            const F* px = phx + cp * nfx * nv;
            const F* py = phy + cp * nfy * nv;
            F div = (px[fE * nv + k] - px[fW * nv + k]) * rdxi + (py[fN * nv + k] - py[fS * nv + k]) * rdyj;
            r[(cp * nc + c) * nv + k] = body ? F(0) : (gt[cp] - f[(cp * nc + c) * nv + k]) * fitau - div;
        }
        invD[(size_t)c * nv + k] = recip(fdiag + geomD_r<F>(rdxi, rdyj, u, v));
    }
}

template <typename F>
cudaError_t launch_micro_residual(const MicroArgs& m, GasDev gas, const double* Wt, const double* q, const F* f,
                                  const F* phx, const F* phy, double dtn_inv, double* inv_tau, F* invD, F* r,
                                  cudaStream_t st)
{
    size_t smem = sizeof(double) * 24 + sizeof(F) * (m.V.nu + m.V.nvv);
    k_micro_residual<F><<<m.L.nc, m.V.nv >= 256 ? 256 : 128, smem, st>>>(m, gas, Wt, q, f, phx, phy, dtn_inv,
                                                                          inv_tau, invD, r);
    return cudaGetLastError();
}
template cudaError_t launch_micro_residual<double>(const MicroArgs&, GasDev, const double*, const double*,
                                                   const double*, const double*, const double*, double, double*,
                                                   double*, double*, cudaStream_t);
template cudaError_t launch_micro_residual<float>(const MicroArgs&, GasDev, const double*, const double*,
                                                  const float*, const float*, const float*, double, double*, float*,
                                                  float*, cudaStream_t);

template <typename F>
__global__ void k_coarse_coeffs(MicroArgs M, GasDev gas, const double* __restrict__ Wt, double dtn_inv,
                                double* __restrict__ inv_tau, F* __restrict__ invD)
{
    const LevelDev& L = M.L;
    const int c = blockIdx.x, i = c % L.nx, j = c / L.nx;
    __shared__ F sc[3];
    if (threadIdx.x == 0) {
        double rho, U, V, lam;
        prim4(Wt + 4 * (size_t)c, rho, U, V, lam);
        double it;
        if constexpr (sizeof(F) == 8) it = 1.0 / tau_of(gas, rho, lam);
        else it = (double)(1.0f / tau_of_f(gas, (float)rho, (float)lam));
        it += dtn_inv;
        inv_tau[c] = it;
        sc[0] = (F)it; sc[1] = (F)L.rdx[i]; sc[2] = (F)L.rdy[j];
    }
    __syncthreads();
    const F fit = sc[0], rdxi = sc[1], rdyj = sc[2];
    const F* __restrict__ vu = VelT<F>::u(M.V);
    const F* __restrict__ vv = VelT<F>::v(M.V);
    for (int k = threadIdx.x; k < M.V.nv; k += blockDim.x)
        invD[(size_t)c * M.V.nv + k] = recip(fit + geomD_r<F>(rdxi, rdyj, vu[k], vv[k]));
}

template <typename F>
cudaError_t launch_coarse_coeffs(const MicroArgs& m, GasDev gas, const double* Wt, double dtn_inv, double* inv_tau,
                                 F* invD, cudaStream_t st)
{
    k_coarse_coeffs<F><<<m.L.nc, 128, 0, st>>>(m, gas, Wt, dtn_inv, inv_tau, invD);
    return cudaGetLastError();
}
template cudaError_t launch_coarse_coeffs<double>(const MicroArgs&, GasDev, const double*, double, double*, double*,
                                                  cudaStream_t);
template cudaError_t launch_coarse_coeffs<float>(const MicroArgs&, GasDev, const double*, double, double*, float*,
                                                 cudaStream_t);

// ---------------------------------------------------------------------------
// boundary faces of a cell on one sweep side (0 lower = west/south, 1 upper = east/north)
struct BFace { int bc, axis, outsign; double rS; };   // rS = face area / cell volume

// (of a fluid cell: its faces with a BC id, on the domain edge or on a body)
__device__ __forceinline__ int side_faces(const LevelDev& L, int i, int j, int side, BFace* bf)
{
    int n = 0;
    const int nx = L.nx;
    const int w = L.fbx[j * (nx + 1) + i], e = L.fbx[j * (nx + 1) + i + 1];
    const int so = L.fby[j * nx + i], no = L.fby[(j + 1) * nx + i];
    if (side != 1 && w >= 0) bf[n++] = {w, 0, -1, L.rdx[i]};
    if (side != 1 && so >= 0) bf[n++] = {so, 1, -1, L.rdy[j]};
    if (side != 0 && e >= 0) bf[n++] = {e, 0, 1, L.rdx[i]};
    if (side != 0 && no >= 0) bf[n++] = {no, 1, 1, L.rdy[j]};
    return n;
}

// local velocity m of chain CTA `rank` -> global k (or -1); groups pair u-rows a and nu-1-a
__device__ __forceinline__ int chain_k(const VelDev& Vg, int rank, int m, int* mirror_u_local, int* mirror_v_local)
{
    int nvv = Vg.nvv, nu = Vg.nu;
    int s = m / (2 * nvv), rem = m - s * 2 * nvv, side = rem / nvv, b = rem - side * nvv;
    int g = rank + s * kChainCluster;
    int ngroups = (nu + 1) / 2;
    if (g >= ngroups) return -1;
    int a = side == 0 ? g : nu - 1 - g;
    if (side == 1 && a == g) return -1;             // middle row of an odd grid
    int sideu = (nu - 1 - g == g) ? 0 : 1 - side;   // local side holding the u-mirror
    *mirror_u_local = s * 2 * nvv + sideu * nvv + b;
    *mirror_v_local = s * 2 * nvv + side * nvv + (nvv - 1 - b);
    return a * nvv + b;
}

// Cluster-wide deterministic sum of NR values with a fixed summation tree:
// each warp reduces its lanes with xor shuffles, lane 0 publishes the warp's
// partial in this CTA's shared slot, one cluster barrier, then every warp
// loads the 32 partials of the cluster (8 CTAs x 4 warps, one per lane, read
// through distributed shared memory) and reduces them with xor shuffles.
// Every thread ends with the same sum.  Slots are double-buffered by event.
template <typename T, int NR>
__device__ __forceinline__ void cluster_sum(cg::cluster_group& cl, T (&v)[NR], T* slots, int& ev)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    #pragma unroll
    for (int q = 0; q < NR; ++q)
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    T* my = slots + (ev & 1) * (4 * 4);                // [warp][q]
    if (lane == 0)
        #pragma unroll
        for (int q = 0; q < NR; ++q) my[warp * 4 + q] = v[q];
    cl.sync();
    const T* src = cl.map_shared_rank(my, lane >> 2);
    #pragma unroll
    for (int q = 0; q < NR; ++q) {
        T x = src[(lane & 3) * 4 + q];
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        v[q] = x;
    }
    ++ev;
}


// Cells 1.. of a boundary line, given the values of cell 0 in xprev: on the
// domain edge, cell 0 is the corner; along a body, cell 0 is the fluid cell
// before the line (a wavefront cell).  Cell st is (i0 + st di, j0 + st dj).  Every such cell has one boundary face on the sweep side, with a
// fixed orientation along the line, so velocities split into
//   outgoing (u_n >= 0 at that face): no ghost term, a recurrence along the
//     line per velocity (phase A, inputs streamed RA cells ahead through a
//     ring of asynchronous shared-memory copies);
//   incoming (u_n < 0): the ghost term needs the cell's wall density, a sum
//     over its outgoing velocities (phase A': per CTA, P threads per cell;
//     phase B: over the cluster, one exchange; published in rho_out), or the
//     mirrored outgoing value (symmetry).  With the ghost known, an incoming
//     velocity of a line cell is an ordinary cell update, done by the
//     wavefront kernel.
// The arithmetic per cell is that of the serial sweep; only the order in which
// independent velocities are visited changes.
template <typename F, int kChainKpt>
__device__ void chain_rest(cg::cluster_group& cl, const MicroArgs& M, const double* __restrict__ iZw,
                           const F* __restrict__ invD, const F* __restrict__ r, F* __restrict__ x, int pass,
                           int line, int i0, int j0, int di, int dj, int len, const int (&kk)[kChainKpt],
                           F (&xprev)[kChainKpt][2],
                           F* __restrict__ rho_out, F* ring, int RA, const int* lk, const F* lw, int nloc)
{
    __shared__ F part[kMaxLine];              // wall sum of this CTA's velocities per cell
    __shared__ F rho_s[kMaxLine];
    __shared__ F lm_nbS[kMaxLine], lm_itau[kMaxLine];
    __shared__ F psum[kChainThreads];
    const LevelDev& L = M.L;
    const VelDev& Vg = M.V;
    const int nx = L.nx, nv = Vg.nv;
    const size_t nc = L.nc;
    const int tid = threadIdx.x, B = blockDim.x;
    const int nb_axis = line == 0 ? 1 : 0, nb_sign = pass == 0 ? -1 : 1;
    // orientation of the line's boundary face (column lines: x-faces, row lines: y-faces)
    const int f_axis = line == 0 ? 0 : 1, f_out = pass == 0 ? -1 : 1;
    auto cell = [&](int st, int& i, int& j) { i = i0 + st * di; j = j0 + st * dj; };
    auto face_bc = [&](int i, int j) {   // the line face of cell (i, j): west / south (forward), east / north
        return f_axis == 0 ? L.fbx[j * (nx + 1) + i + (f_out > 0)] : L.fby[(j + (f_out > 0)) * nx + i];
    };
    for (int st = tid; st < len; st += B) {
        int i, j;
        cell(st, i, j);
        lm_nbS[st] = (F)(nb_axis == 0 ? L.rdx[i] : L.rdy[j]);
        lm_itau[st] = (F)M.inv_tau[j * nx + i];
    }
    // per velocity: Dn = an * nbS (the neighbour along the line) and
    // D = itau + gfix + gvar * nbS (|u|/dx + |v|/dy with the line's fixed spacing in gfix)
    int ifx, jfx;
    cell(0, ifx, jfx);
    F an[kChainKpt], gfix[kChainKpt], gvar[kChainKpt];
    bool outg[kChainKpt];
    #pragma unroll
    for (int t = 0; t < kChainKpt; ++t) {
        const int k = kk[t];
        const F u = k < 0 ? F(0) : (F)Vg.u[k], v = k < 0 ? F(0) : (F)Vg.v[k];
        const F uo = f_out < 0 ? -(f_axis == 0 ? u : v) : (f_axis == 0 ? u : v);
        outg[t] = k >= 0 && uo >= F(0);
        const F un = nb_sign < 0 ? -(nb_axis == 0 ? u : v) : (nb_axis == 0 ? u : v);
        an[t] = un < F(0) ? un : F(0);
        gfix[t] = line == 0 ? fabs(u) * (F)L.rdx[ifx] : fabs(v) * (F)L.rdy[jfx];
        gvar[t] = line == 0 ? fabs(v) : fabs(u);
    }
    __syncthreads();
    // ---- phase A: outgoing velocities
    {
        F xp[kChainKpt][2];
        #pragma unroll
        for (int t = 0; t < kChainKpt; ++t) { xp[t][0] = xprev[t][0]; xp[t][1] = xprev[t][1]; }
        const F* src = pass == 0 ? r : x;
        const size_t rstride = (size_t)kChainKpt * 3 * B;
        auto issue = [&](int st) {
            if (st < len) {
                int i, j;
                cell(st, i, j);
                const size_t c = (size_t)j * nx + i;
                F* rs = ring + (size_t)(st % RA) * rstride;
                #pragma unroll
                for (int t = 0; t < kChainKpt; ++t) {
                    if (!outg[t]) continue;
                    const int k = kk[t];
                    cp_async_elem(rs + (t * 3 + 0) * B + tid, invD + c * nv + k);
                    cp_async_elem(rs + (t * 3 + 1) * B + tid, src + c * nv + k);
                    cp_async_elem(rs + (t * 3 + 2) * B + tid, src + (nc + c) * nv + k);
                }
            }
            cp_async_commit();
        };
        for (int q = 1; q < RA; ++q) issue(q);
        for (int st = 1; st < len; ++st) {
            issue(st + RA - 1);
            cp_async_wait(RA - 1);
            const F* rs = ring + (size_t)(st % RA) * rstride;
            int i, j;
            cell(st, i, j);
            const size_t c = (size_t)j * nx + i;
            const F nbS = lm_nbS[st], itau = lm_itau[st];
            #pragma unroll
            for (int t = 0; t < kChainKpt; ++t) {
                if (!outg[t]) continue;
                const int k = kk[t];
                const F Dn = an[t] * nbS, id = rs[(t * 3) * B + tid];
                const F D = pass == 1 ? itau + (gfix[t] + gvar[t] * nbS) : F(0);
                #pragma unroll
                for (int cp = 0; cp < 2; ++cp) {
                    const F in = rs[(t * 3 + 1 + cp) * B + tid];
                    const F base = pass == 0 ? in - Dn * xp[t][cp] : D * in - Dn * xp[t][cp];
                    const F xv = base * id;
                    x[(cp * nc + c) * nv + k] = xv;
                    xp[t][cp] = xv;
                }
            }
        }
        cp_async_wait(0);
    }
    __syncthreads();   // this CTA's outgoing values along the line are in x
    // ---- phase A': wall sum over this CTA's outgoing velocities, P threads per cell
    {
        const int ncell = len - 1;
        const int P = ncell >= B ? 1 : B / ncell, per = B / P;
        for (int s0 = 0; s0 < ncell; s0 += per) {
            const int st = 1 + s0 + tid / P, p = tid % P;
            const bool mine = tid / P < per && st < len;
            F sum = F(0);
            if (mine) {
                int i, j;
                cell(st, i, j);
                if (M.bc[face_bc(i, j)].type == BC_WALL) {
                    // eight independent loads in flight (the values of incoming velocities are not
                    // read: they belong to the previous sweep and may be anything)
                    const F* xc0 = x + (size_t)(j * nx + i) * nv;
                    F acc[8] = {F(0), F(0), F(0), F(0), F(0), F(0), F(0), F(0)};
                    int q = p;
                    for (; q + 7 * P < nloc; q += 8 * P) {
                        F xv[8];
                        #pragma unroll
                        for (int u8 = 0; u8 < 8; ++u8) {
                            const int qq = q + u8 * P;
                            xv[u8] = lw[qq] != F(0) ? xc0[lk[qq]] : F(0);
                        }
                        #pragma unroll
                        for (int u8 = 0; u8 < 8; ++u8) acc[u8] += lw[q + u8 * P] * xv[u8];
                    }
                    for (int u8 = 0; q < nloc; q += P, ++u8)
                        if (lw[q] != F(0)) acc[u8] += lw[q] * xc0[lk[q]];
                    sum = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
                }
            }
            if (P == 1) {
                if (mine) part[st] = sum;
            } else {
                psum[tid] = sum;
                __syncthreads();
                if (mine && p == 0) {
                    F t = F(0);
                    for (int q = 0; q < P; ++q) t += psum[tid + q];
                    part[st] = t;
                }
                __syncthreads();
            }
        }
    }
    cl.sync();
    // ---- phase B: wall density of every cell of the line (fixed summation order)
    for (int st = 1 + tid; st < len; st += B) {
        int i, j;
        cell(st, i, j);
        const int bc = face_bc(i, j);
        F rho = F(0);
        if (M.bc[bc].type == BC_WALL) {
            F sum = F(0);
            for (int rk = 0; rk < kChainCluster; ++rk) sum += cl.map_shared_rank(part, rk)[st];
            rho = -sum * (F)iZw[bc * 4 + f_axis * 2 + (f_out > 0)];
        }
        rho_s[st] = rho;
    }
    __syncthreads();
    // the incoming velocities of cells 1.. are finished by the wavefront kernel
    if (cl.block_rank() == 0)
        for (int st = tid; st < len; st += B) rho_out[st] = st == 0 ? F(0) : rho_s[st];
}

template <typename F, int kChainKpt>
__global__ void __cluster_dims__(kChainCluster, 1, 1) __launch_bounds__(kChainThreads)
k_sgs_chain(MicroArgs M, const double* __restrict__ Zw, const F* __restrict__ invD, const F* __restrict__ r,
            F* __restrict__ x, const F* __restrict__ xcorner, F* __restrict__ rho_lines, int pass, int RA)
{
    const double* __restrict__ iZw = Zw + 4 * kMaxBcs;          // reciprocals of the wall normalisations
    __shared__ F slots[2 * 4 * 4];
    extern __shared__ double xsm_raw[];
    F* xsm = reinterpret_cast<F*>(xsm_raw);  // [2][nloc] current cell values of this CTA's velocities
    cg::cluster_group cl = cg::this_cluster();
    const LevelDev& L = M.L;
    const VelDev& Vg = M.V;
    const int rank = cl.block_rank(), line = blockIdx.x / kChainCluster;
    const int nx = L.nx, ny = L.ny, nv = Vg.nv;
    const size_t nc = L.nc;
    const int ngroups = (Vg.nu + 1) / 2;
    const int nloc = ((ngroups + kChainCluster - 1) / kChainCluster) * 2 * Vg.nvv;
    int ev = 0;
    int kk[kChainKpt], mu[kChainKpt], mvv[kChainKpt];
    #pragma unroll
    for (int t = 0; t < kChainKpt; ++t) {
        int m = threadIdx.x + t * blockDim.x;
        kk[t] = m < nloc ? chain_k(Vg, rank, m, &mu[t], &mvv[t]) : -1;
    }
    F xprev[kChainKpt][2];
    const int len = line == 0 ? ny : nx;
    auto cell_of = [&](int st, int& ci, int& cj) {
        if (pass == 0) { ci = line == 0 ? 0 : st; cj = line == 0 ? st : 0; }
        else { ci = line == 0 ? nx - 1 : nx - 1 - st; cj = line == 0 ? ny - 1 - st : ny - 1; }
    };
    // per-velocity inputs of the current and the next cell (prefetched one step ahead)
    F cin[kChainKpt][2], cdi[kChainKpt], nin[kChainKpt][2], ndi[kChainKpt];
    double citau = 0.0, nitau = 0.0;
    auto load = [&](int st, F (&in)[kChainKpt][2], F (&di)[kChainKpt], double& it) {
        int ci, cj;
        cell_of(st, ci, cj);
        const int cc = cj * nx + ci;
        it = M.inv_tau[cc];
        #pragma unroll
        for (int t = 0; t < kChainKpt; ++t) {
            int k = kk[t];
            if (k < 0) continue;
            di[t] = invD[(size_t)cc * nv + k];
            #pragma unroll
            for (int cp = 0; cp < 2; ++cp) {
                size_t id = (cp * nc + cc) * nv + k;
                // backward: the corner's forward value comes from a copy taken before the
                // launch, because the column line overwrites the corner while the row line reads it
                in[t][cp] = pass == 0 ? r[id] : (st == 0 ? xcorner[cp * nv + k] : x[id]);
            }
        }
    };
    load(0, cin, cdi, citau);
    for (int s = 0; s < 1; ++s) {   // the corner cell; the rest of the line follows in three phases
        (void)nin; (void)ndi; (void)nitau;
        // cell of this step
        int i, j;
        cell_of(s, i, j);
        const int c = j * nx + i;
        const F itau = (F)citau;
        // interior neighbour along the line (the previous cell), if any
        int nb_axis = line == 0 ? 1 : 0, nb_sign = pass == 0 ? -1 : 1;
        const F nbS = (F)(nb_axis == 0 ? L.rdx[i] : L.rdy[j]);
        BFace bf[2];
        int nb = side_faces(L, i, j, pass, bf);
        int nwall = 0, nsym = 0;
        bool has_out = false;
        for (int b = 0; b < nb; ++b) {
            int t = M.bc[bf[b].bc].type;
            nwall += t == BC_WALL;
            nsym += t == BC_SYMMETRY;
            has_out = has_out || t == BC_OUTFLOW;
        }
        F base[kChainKpt][2], den[kChainKpt], xc[kChainKpt][2];   // den holds 1/denominator
        #pragma unroll
        for (int t = 0; t < kChainKpt; ++t) {
            int k = kk[t];
            if (k < 0) continue;
            const F u = (F)Vg.u[k], v = (F)Vg.v[k];
            const F Dn = s > 0 ? Dface<F>(nb_axis, nb_sign, nbS, u, v) : F(0);
            // 1/D from the precomputed table unless an outflow face adds to the diagonal
            F D = F(0);
            if (has_out || pass == 1) D = itau + geomD<F>(L, i, j, u, v);
            if (has_out) {
                F dd = D;
                for (int b = 0; b < nb; ++b)
                    if (M.bc[bf[b].bc].type == BC_OUTFLOW) dd += Dface<F>(bf[b].axis, bf[b].outsign, (F)bf[b].rS, u, v);
                den[t] = recip(dd);
            } else {
                den[t] = cdi[t];
            }
            #pragma unroll
            for (int cp = 0; cp < 2; ++cp) {
                F y = s > 0 ? Dn * xprev[t][cp] : F(0);
                base[t][cp] = pass == 0 ? cin[t][cp] - y : D * cin[t][cp] - y;
                xc[t][cp] = base[t][cp] * den[t];
            }
        }
        if (nwall == 2 && nb == 2) {
            // two walls at a corner: 2x2 system for the two ghost densities
            double z[2];
            F acc[4] = {0, 0, 0, 0};
            for (int b = 0; b < 2; ++b) z[b] = Zw[bf[b].bc * 4 + bf[b].axis * 2 + (bf[b].outsign > 0)];
            #pragma unroll
            for (int t = 0; t < kChainKpt; ++t) {
                int k = kk[t];
                if (k < 0) continue;
                const F u = (F)Vg.u[k], v = (F)Vg.v[k], w = (F)Vg.w[k];
                for (int b = 0; b < 2; ++b) {
                    F uo = bf[b].axis == 0 ? u : v;
                    uo = bf[b].outsign < 0 ? -uo : uo;
                    if (!(uo > F(0))) continue;
                    acc[b] += w * uo * base[t][0] * den[t];
                    int o = 1 - b;
                    F Do = Dface<F>(bf[o].axis, bf[o].outsign, (F)bf[o].rS, u, v);
                    if (Do != F(0)) acc[2 + b] += w * uo * Do * (F)M.Cw[(size_t)bf[o].bc * nv + k] * den[t];
                }
            }
            cluster_sum<F, 4>(cl, acc, slots, ev);
            double cc0 = -acc[0] / z[0], cc1 = -acc[1] / z[1], mm0 = acc[2] / z[0], mm1 = acc[3] / z[1];
            double rho2[2];
            rho2[0] = (cc0 + mm0 * cc1) / (1.0 - mm0 * mm1);
            rho2[1] = cc1 + mm1 * rho2[0];
            const F rho[2] = {(F)rho2[0], (F)rho2[1]};
            #pragma unroll
            for (int t = 0; t < kChainKpt; ++t) {
                int k = kk[t];
                if (k < 0) continue;
                const F u = (F)Vg.u[k], v = (F)Vg.v[k];
                for (int cp = 0; cp < 2; ++cp) {
                    F a = base[t][cp];
                    for (int b = 0; b < 2; ++b) {
                        F Db = Dface<F>(bf[b].axis, bf[b].outsign, (F)bf[b].rS, u, v);
                        F C = (F)(M.Cw[(size_t)bf[b].bc * nv + k] * (cp == 0 ? 1.0 : kKint * M.bc[bf[b].bc].t / 4.0));
                        if (Db != F(0)) a -= Db * C * rho[b];
                    }
                    xc[t][cp] = a * den[t];
                }
            }
        } else if (nwall + nsym > 0) {
            // substitution rounds (exact for every other combination; one round without symmetry)
            int rounds = nsym > 0 ? 3 : 1;
            for (int rd = 0; rd < rounds; ++rd) {
                F rho = F(0);
                int wb = -1;
                for (int b = 0; b < nb; ++b) if (M.bc[bf[b].bc].type == BC_WALL) wb = b;
                if (nsym > 0) {
                    #pragma unroll
                    for (int t = 0; t < kChainKpt; ++t) {
                        int m = threadIdx.x + t * blockDim.x;
                        if (kk[t] >= 0) { xsm[m] = xc[t][0]; xsm[nloc + m] = xc[t][1]; }
                    }
                    __syncthreads();
                }
                if (wb >= 0) {
                    F acc[1] = {F(0)};
                    #pragma unroll
                    for (int t = 0; t < kChainKpt; ++t) {
                        int k = kk[t];
                        if (k < 0) continue;
                        F uo = (F)(bf[wb].axis == 0 ? Vg.u[k] : Vg.v[k]);
                        uo = bf[wb].outsign < 0 ? -uo : uo;
                        if (uo > F(0)) acc[0] += (F)Vg.w[k] * uo * xc[t][0];
                    }
                    cluster_sum<F, 1>(cl, acc, slots, ev);
                    rho = -acc[0] * (F)iZw[bf[wb].bc * 4 + bf[wb].axis * 2 + (bf[wb].outsign > 0)];
                }
                F xn[kChainKpt][2];
                #pragma unroll
                for (int t = 0; t < kChainKpt; ++t) {
                    int k = kk[t];
                    if (k < 0) continue;
                    const F u = (F)Vg.u[k], v = (F)Vg.v[k];
                    for (int cp = 0; cp < 2; ++cp) {
                        F a = base[t][cp];
                        for (int b = 0; b < nb; ++b) {
                            F Db = Dface<F>(bf[b].axis, bf[b].outsign, (F)bf[b].rS, u, v);
                            if (Db == F(0)) continue;
                            int ty = M.bc[bf[b].bc].type;
                            if (ty == BC_WALL)
                                a -= Db * (F)(M.Cw[(size_t)bf[b].bc * nv + k] *
                                              (cp == 0 ? 1.0 : kKint * M.bc[bf[b].bc].t / 4.0)) * rho;
                            else if (ty == BC_SYMMETRY)
                                a -= Db * xsm[cp * nloc + (bf[b].axis == 0 ? mu[t] : mvv[t])];
                        }
                        xn[t][cp] = a * den[t];
                    }
                }
                if (nsym > 0) __syncthreads();
                #pragma unroll
                for (int t = 0; t < kChainKpt; ++t)
                    if (kk[t] >= 0) { xc[t][0] = xn[t][0]; xc[t][1] = xn[t][1]; }
            }
        }
        // store (the corner is written by the column line only) and carry along the line
        const bool write = !(line == 1 && s == 0);
        #pragma unroll
        for (int t = 0; t < kChainKpt; ++t) {
            int k = kk[t];
            if (k < 0) continue;
            xprev[t][0] = xc[t][0];
            xprev[t][1] = xc[t][1];
            if (write) {
                x[c * (size_t)nv + k] = xc[t][0];
                x[(nc + c) * (size_t)nv + k] = xc[t][1];
            }
        }
    }
    if (len > 1) {
        // this CTA's velocities with their outgoing wall weights w u_n (0 when not outgoing)
        F* lw = xsm + 2 * nloc;
        F* ring = lw + nloc;
        int* lk = reinterpret_cast<int*>(ring + (size_t)RA * kChainKpt * 3 * blockDim.x);
        const int f_axis = line == 0 ? 0 : 1;
        #pragma unroll
        for (int t = 0; t < kChainKpt; ++t) {
            const int m = threadIdx.x + t * blockDim.x;
            if (m >= nloc) continue;
            const int k = kk[t];
            F wuo = F(0);
            if (k >= 0) {
                const F un = (F)(f_axis == 0 ? Vg.u[k] : Vg.v[k]), uo = pass == 0 ? -un : un;
                wuo = uo > F(0) ? (F)Vg.w[k] * uo : F(0);
            }
            lk[m] = k;
            lw[m] = wuo;
        }
        const int i0 = pass == 0 ? 0 : nx - 1, j0 = pass == 0 ? 0 : ny - 1, sg = pass == 0 ? 1 : -1;
        chain_rest<F, kChainKpt>(cl, M, iZw, invD, r, x, pass, line, i0, j0, line == 0 ? 0 : sg, line == 0 ? sg : 0,
                                 len, kk, xprev, rho_lines + line * kMaxLine, ring, RA, lk, lw, nloc);
    }
    cl.sync();   // keep every CTA's shared memory alive until all remote reads are done
}


// The lines along bodies of one sweep pass that start after the same
// wavefront step, one cluster per line.  Cell 0 of a line is the fluid cell
// before it, whose values (all velocities) the wavefront has already written
// to x; chain_rest walks the line's outgoing velocities and publishes the
// wall densities, and the wavefront then finishes its incoming velocities.
template <typename F, int kChainKpt>
__global__ void __cluster_dims__(kChainCluster, 1, 1) __launch_bounds__(kChainThreads)
k_sgs_chain_body(MicroArgs M, const double* __restrict__ Zw, const F* __restrict__ invD, const F* __restrict__ r,
                 F* __restrict__ x, F* __restrict__ rho_lines, int pass, int q0, int RA)
{
    const double* __restrict__ iZw = Zw + 4 * kMaxBcs;
    extern __shared__ double xsm_raw[];
    F* xsm = reinterpret_cast<F*>(xsm_raw);
    cg::cluster_group cl = cg::this_cluster();
    const VelDev& Vg = M.V;
    const int rank = cl.block_rank(), nv = Vg.nv, nx = M.L.nx;
    const size_t nc = M.L.nc;
    const int* ld = M.P.lines[pass] + 8 * (q0 + blockIdx.x / kChainCluster);
    const int i0 = ld[0], j0 = ld[1], di = ld[2], dj = ld[3], len = ld[4], line = ld[5], slot = ld[6];
    const int ngroups = (Vg.nu + 1) / 2;
    const int nloc = ((ngroups + kChainCluster - 1) / kChainCluster) * 2 * Vg.nvv;
    int kk[kChainKpt], mu[kChainKpt], mvv[kChainKpt];
    #pragma unroll
    for (int t = 0; t < kChainKpt; ++t) {
        int m = threadIdx.x + t * blockDim.x;
        kk[t] = m < nloc ? chain_k(Vg, rank, m, &mu[t], &mvv[t]) : -1;
    }
    F xprev[kChainKpt][2];
    const size_t c0 = (size_t)j0 * nx + i0;
    #pragma unroll
    for (int t = 0; t < kChainKpt; ++t) {
        xprev[t][0] = xprev[t][1] = F(0);
        if (kk[t] >= 0) {
            xprev[t][0] = x[c0 * nv + kk[t]];
            xprev[t][1] = x[(nc + c0) * nv + kk[t]];
        }
    }
    F* lw = xsm + 2 * nloc;
    F* ring = lw + nloc;
    int* lk = reinterpret_cast<int*>(ring + (size_t)RA * kChainKpt * 3 * blockDim.x);
    #pragma unroll
    for (int t = 0; t < kChainKpt; ++t) {
        const int m = threadIdx.x + t * blockDim.x;
        if (m >= nloc) continue;
        const int k = kk[t];
        F wuo = F(0);
        if (k >= 0) {
            const F un = (F)(line == 0 ? Vg.u[k] : Vg.v[k]), uo = pass == 0 ? -un : un;
            wuo = uo > F(0) ? (F)Vg.w[k] * uo : F(0);
        }
        lk[m] = k;
        lw[m] = wuo;
    }
    __syncthreads();
    chain_rest<F, kChainKpt>(cl, M, iZw, invD, r, x, pass, line, i0, j0, di, dj, len, kk, xprev, rho_lines + slot,
                             ring, RA, lk, lw, nloc);
    cl.sync();   // keep every CTA's shared memory alive until all remote reads are done
}


// four consecutive values through 16-byte accesses (16-byte aligned for float, 32 for double)
__device__ __forceinline__ void ld4(const float* p, float (&v)[4])
{
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4])
{
    const double2 t0 = *reinterpret_cast<const double2*>(p), t1 = *reinterpret_cast<const double2*>(p + 2);
    v[0] = t0.x; v[1] = t0.y; v[2] = t1.x; v[3] = t1.y;
}
__device__ __forceinline__ void st4(float* p, const float (&v)[4])
{
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double (&v)[4])
{
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
}

// the kInteriorKc values of consecutive velocities at gsrc (nk of them exist) into sdst
template <typename F, bool VEC>
__device__ __forceinline__ void cp_async_k4(F* sdst, const F* gsrc, int nk)
{
    if constexpr (VEC) {
        cp_async16(sdst, gsrc);
        if constexpr (sizeof(F) == 8)
            if (nk > 2) cp_async16(sdst + 2, gsrc + 2);
    } else if (sizeof(F) == 4 && nk == kInteriorKc && (reinterpret_cast<uintptr_t>(gsrc) & 7) == 0) {
        // FP32 with a velocity count that is not a multiple of four: the run of four
        // values still starts on an 8- or 16-byte boundary for half of the cells
        // (sdst is 16-byte aligned)
        if ((reinterpret_cast<uintptr_t>(gsrc) & 15) == 0) {
            cp_async16(sdst, gsrc);
        } else {
            const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gsrc) : "memory");
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa + 8), "l"(gsrc + 2) : "memory");
        }
    } else {
        #pragma unroll
        for (int q = 0; q < kInteriorKc; ++q)
            if (q < nk) cp_async_elem(sdst + q, gsrc + q);
    }
}

// store a run of four FP32 values with the widest accesses its address allows
__device__ __forceinline__ void st4_any(float* p, const float (&v)[4])
{
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    if ((a & 15) == 0) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else if ((a & 7) == 0) {
        *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
        *reinterpret_cast<float2*>(p + 2) = make_float2(v[2], v[3]);
    } else {
        p[0] = v[0];
        *reinterpret_cast<float2*>(p + 1) = make_float2(v[1], v[2]);
        p[3] = v[3];
    }
}

// Inputs of the boundary-line cells for k_sgs_wave, after their line walk
// (k_sgs_chain, k_sgs_chain_body): per fold entry e in [e0, e0 + ne) (a cell
// of a line, from the plan's table) and velocity, the right-hand side b of G
// and H and 1/D, laid out as the wavefront's ring entries,
// fold[blk][e][3][kInteriorKc] (blk = k / kInteriorKc).  Outgoing velocities
// and the corner carry their final value (applied as is).  Incoming ones carry
// the ghost term folded in: forward b = r - g, backward b = (D x - g) / D, with
// g = Db C rho_s (wall) or Db x_mirror (symmetry), and 1/(D + Db) in place of
// 1/D at an outflow face.
template <typename F>
__global__ void k_line_fold(MicroArgs M, const F* __restrict__ invD, const F* __restrict__ r,
                            const F* __restrict__ x, const F* __restrict__ rho_lines, F* __restrict__ fold, int pass,
                            int e0, int ne)
{
    constexpr int K = kInteriorKc;
    const LevelDev& L = M.L;
    const VelDev& Vg = M.V;
    const int nx = L.nx, nv = Vg.nv, nls = M.P.nl_max;
    const size_t nc = L.nc;
    const int nblk = (nv + K - 1) / K;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nblk * ne * K) return;
    const int kk = t % K, e = e0 + (t / K) % ne, blk = t / (K * ne), kq = blk * K + kk;
    const int4 lc = M.P.lcell[pass][e];                  // {cell, line axis, density slot, final}
    const int c = lc.x, line = lc.y, i = c % nx, j = c / nx, fout = pass == 0 ? -1 : 1;
    F b[2] = {F(0), F(0)}, iv = F(1);
    if (kq < nv) {
        const size_t id = (size_t)c * nv + kq;
        const F u = (F)Vg.u[kq], v = (F)Vg.v[kq];
        const F uo = fout < 0 ? -(line == 0 ? u : v) : (line == 0 ? u : v);   // u_n at the line face
        if (lc.w || uo >= F(0)) {
            b[0] = x[id];
            b[1] = x[nc * nv + id];
        } else {
            const int bc = line == 0 ? L.fbx[j * (nx + 1) + i + (fout > 0)] : L.fby[(j + (fout > 0)) * nx + i];
            const BcDev Bc = M.bc[bc];
            const F Db = uo * (line == 0 ? (F)L.rdx[i] : (F)L.rdy[j]);
            const F D = (F)M.inv_tau[c] + geomD<F>(L, i, j, u, v);
            iv = Bc.type == BC_OUTFLOW ? recip(D + Db) : invD[id];
            int km = 0;
            if (Bc.type == BC_SYMMETRY) {
                const int a2 = kq / Vg.nvv, b2 = kq - a2 * Vg.nvv;
                km = line == 0 ? (Vg.nu - 1 - a2) * Vg.nvv + b2 : a2 * Vg.nvv + (Vg.nvv - 1 - b2);
            }
            #pragma unroll
            for (int cp = 0; cp < 2; ++cp) {
                F g = F(0);
                if (Bc.type == BC_WALL)
                    g = Db * ((F)(M.Cw[(size_t)bc * nv + kq] * (cp == 0 ? 1.0 : kKint * Bc.t / 4.0)) * rho_lines[lc.z]);
                else if (Bc.type == BC_SYMMETRY)
                    g = Db * x[cp * nc * nv + (size_t)c * nv + km];   // an outgoing velocity: final
                b[cp] = pass == 0 ? r[cp * nc * nv + id] - g : (D * x[cp * nc * nv + id] - g) * iv;
            }
        }
    }
    F* o = fold + ((size_t)(blk * nls + e) * 3) * K + kk;
    o[0] = b[0];
    o[K] = b[1];
    o[2 * K] = iv;
}

// Wavefront steps [dd0, dd1) of one sweep over every cell for the
// kInteriorKc velocities of this CTA, in anti-diagonal order, one thread per
// cell of the diagonal handling the 2 x kInteriorKc values (G and H,
// consecutive velocities) of its cell.  Ordinary update: (forward)
// x = (b - D_W x_W - D_S x_S) / D with b the residual, (backward)
// x = b - (D_E x_E + D_N x_N) / D with b the forward value.  Boundary-line
// cells take b and 1/D from k_line_fold and drop the neighbour across their
// line face; cells in a body are zero.  Values of the previous diagonal stay
// in shared memory (a segment after the first reloads them from x); the inputs
// of the next R - 1 diagonals are in flight as asynchronous copies into a ring
// of R shared buffers, so the per-diagonal path only touches shared memory.
// BODIES: cell codes from the plan's table (a mesh with bodies); without
// bodies the code of a cell follows from its position (the edge column and row).
template <typename F, int R, bool VEC, bool BODIES>
__global__ void __launch_bounds__(512) k_sgs_wave(MicroArgs M, const F* __restrict__ invD, const F* __restrict__ r,
                                                  F* __restrict__ x, const F* __restrict__ fold, int pass, int dd0,
                                                  int dd1, int listed)
{
    // this CTA's block of velocities: every block, or the listed wavefront-class blocks
    const int blk = listed ? M.V.wblk[pass][blockIdx.x] : blockIdx.x;
    extern __shared__ __align__(16) double sraw[];
    constexpr int K = kInteriorKc, W = 2 * K;
    const LevelDev& L = M.L;
    const VelDev& Vg = M.V;
    const int nx = L.nx, ny = L.ny, nv = Vg.nv;
    const size_t nc = L.nc;
    const int B = blockDim.x, tid = threadIdx.x;
    const int k0 = blk * K, nk = min(K, nv - k0);
    const int nd = nx + ny - 1, nls = M.P.nl_max;
    const int* __restrict__ code = M.P.code[pass];
    F* sx = reinterpret_cast<F*>(sraw);                 // [2][nx][W] values of the previous diagonal
    F* ring = sx + 2 * (size_t)nx * W;                  // [R][3][B][K] b (G, H) and 1/D of upcoming diagonals
    F* srdx = ring + (size_t)R * 3 * B * K;             // [nx] 1/dx
    F* srdy = srdx + nx;                                // [ny] 1/dy
    int* cring = reinterpret_cast<int*>(srdy + ny);     // [R][B] cell codes of the upcoming diagonals
    const F* src = pass == 0 ? r : x;
    const int ib = pass == 0 ? 0 : nx - 1, jb = pass == 0 ? 0 : ny - 1;   // the edge column and row of the pass
    // code of this thread's cell on wavefront step dd (with bodies; loaded one step before it is needed)
    auto code_of = [&](int dd) {
        if (!BODIES || dd >= dd1) return -3;
        const int d = pass == 0 ? dd : nd - 1 - dd;
        const int ilo = max(0, d - (ny - 1)), ncell = min(nx - 1, d) - ilo + 1;
        return tid < ncell ? code[(d - ilo - tid) * nx + ilo + tid] : -3;
    };
    auto issue = [&](int dd, int cd) {
        if (dd < dd1) {
            const int d = pass == 0 ? dd : nd - 1 - dd;
            const int ilo = max(0, d - (ny - 1)), ncell = min(nx - 1, d) - ilo + 1;
            if (tid < ncell) {
                const int i = ilo + tid, j = d - i;
                F* ra = ring + ((size_t)(dd % R) * 3 * B + tid) * K;
                if constexpr (BODIES) {
                    cring[(dd % R) * B + tid] = cd;     // read back by this thread when swept
                } else {                                // without bodies the position gives the code
                    cd = i != ib && j != jb ? -1 : ((i == ib ? (pass == 0 ? j : ny - 1 - j)
                                                             : ny + (pass == 0 ? i : nx - 1 - i)) << 2);
                }
                if (cd == -1) {
                    const size_t e = ((size_t)j * nx + i) * nv + k0;
                    cp_async_k4<F, VEC>(ra, src + e, nk);
                    cp_async_k4<F, VEC>(ra + (size_t)B * K, src + nc * nv + e, nk);
                    cp_async_k4<F, VEC>(ra + (size_t)2 * B * K, invD + e, nk);
                } else if (cd >= 0) {                   // a boundary-line cell: its folded inputs
                    const F* fo = fold + ((size_t)(blk * nls + (cd >> 2)) * 3) * K;
                    cp_async_k4<F, true>(ra, fo, K);
                    cp_async_k4<F, true>(ra + (size_t)B * K, fo + K, K);
                    cp_async_k4<F, true>(ra + (size_t)2 * B * K, fo + 2 * K, K);
                }
            }
        }
        cp_async_commit();
    };
    if constexpr (R > 1)
        for (int dd = dd0; dd < dd0 + R - 1; ++dd) issue(dd, code_of(dd));
    // cell codes of the next four issues, loaded four sweep steps before they are used
    // (one step is shorter than a global load)
    int cd_next = code_of(dd0 + R - 1), cd_n1 = code_of(dd0 + R), cd_n2 = code_of(dd0 + R + 1),
        cd_n3 = code_of(dd0 + R + 2);
    // prologue: diagonal buffers (the previous segment's last diagonal from x) and spacings
    for (int q = tid; q < 2 * nx * W; q += B) sx[q] = F(0);
    __syncthreads();
    if (dd0 > 0) {
        const int d = pass == 0 ? dd0 - 1 : nd - dd0;
        const int ilo = max(0, d - (ny - 1)), ncell = min(nx - 1, d) - ilo + 1;
        F* prev = sx + (size_t)((dd0 + 1) & 1) * nx * W;
        for (int q = tid; q < ncell * W; q += B) {
            const int i = ilo + q / W, w = q % W, cp = w / K, kk = w % K;
            if (kk < nk) prev[(size_t)i * W + w] = x[(cp * nc + (size_t)(d - i) * nx + i) * nv + k0 + kk];
        }
    }
    for (int q = tid; q < nx; q += B) srdx[q] = (F)L.rdx[q];
    for (int q = tid; q < ny; q += B) srdy[q] = (F)L.rdy[q];
    // per velocity: neighbour coefficients (zero where the upwind neighbour is on the other side)
    // and which velocities leave through a column / row line face
    F cu[K], cv[K];
    unsigned outc = 0, outr = 0;
    #pragma unroll
    for (int kk = 0; kk < K; ++kk) {
        const int kq = k0 + kk;
        const F u = kq < nv ? (F)Vg.u[kq] : F(0), v = kq < nv ? (F)Vg.v[kq] : F(0);
        cu[kk] = pass == 0 ? (u > F(0) ? -u : F(0)) : (u < F(0) ? u : F(0));
        cv[kk] = pass == 0 ? (v > F(0) ? -v : F(0)) : (v < F(0) ? v : F(0));
        if ((pass == 0 ? -u : u) >= F(0)) outc |= 1u << kk;
        if ((pass == 0 ? -v : v) >= F(0)) outr |= 1u << kk;
    }
    const int xo = pass == 0 ? -1 : 1;                  // x neighbour: i - 1 (forward) or i + 1
    __syncthreads();
    for (int dd = dd0; dd < dd1; ++dd) {
        if constexpr (R == 1) {
            issue(dd, cd_next);
            cd_next = code_of(dd + 1);
            cp_async_wait_n<0>();
        } else {
            cp_async_wait_n<R - 2>();
        }
        const int d = pass == 0 ? dd : nd - 1 - dd;
        const int ilo = max(0, d - (ny - 1)), ncell = min(nx - 1, d) - ilo + 1;
        const F* prev = sx + (size_t)((dd + 1) & 1) * nx * W;
        F* cur = sx + (size_t)(dd & 1) * nx * W;
        if (tid < ncell) {
            const int i = ilo + tid, j = d - i;
            int cd = -1;
            if constexpr (BODIES) cd = cring[(dd % R) * B + tid];
            const F* ra = ring + ((size_t)(dd % R) * 3 * B + tid) * K;
            static_assert(K == 4, "vector accesses assume four velocities per CTA");
            F res[2][K];
            if (BODIES && cd == -2) {                   // in a body
                #pragma unroll
                for (int kk = 0; kk < K; ++kk) res[0][kk] = res[1][kk] = F(0);
            } else {
                F a[2][K], iv[K], pwv[2][K], psv[2][K];
                ld4(ra, a[0]);
                ld4(ra + (size_t)B * K, a[1]);
                ld4(ra + (size_t)2 * B * K, iv);
                bool hx = i != ib, hy = j != jb;
                if constexpr (BODIES) { hx = !(cd >= 0 && (cd & 2)); hy = !(cd >= 0 && (cd & 1)); }
                const F fx = hx ? srdx[i] : F(0), fy = hy ? srdy[j] : F(0);
                const F* pw = prev + (size_t)(hx ? i + xo : i) * W;
                const F* ps = prev + (size_t)i * W;
                ld4(pw, pwv[0]);
                ld4(pw + K, pwv[1]);
                ld4(ps, psv[0]);
                ld4(ps + K, psv[1]);
                // boundary-line cell: the final values (corner, outgoing velocities) are applied as is
                const unsigned ld = hx && hy ? 0u : (!hx && !hy ? 0xFu : (!hx ? outc : outr));
                #pragma unroll
                for (int cp = 0; cp < 2; ++cp)
                    #pragma unroll
                    for (int kk = 0; kk < K; ++kk) {
                        const F y = cu[kk] * fx * pwv[cp][kk] + cv[kk] * fy * psv[cp][kk];
                        const F rv = pass == 0 ? (a[cp][kk] - y) * iv[kk] : a[cp][kk] - y * iv[kk];
                        res[cp][kk] = (ld >> kk) & 1u ? a[cp][kk] : rv;
                    }
            }
            #pragma unroll
            for (int cp = 0; cp < 2; ++cp) {
                F* xd = x + (cp * nc + (size_t)j * nx + i) * nv + k0;
                st4(cur + (size_t)i * W + cp * K, res[cp]);
                if constexpr (VEC) {
                    if (nk == K) {
                        st4(xd, res[cp]);
                    } else {                            // double, nv = 2 mod 4: the last two values do not exist
                        xd[0] = res[cp][0];
                        xd[1] = res[cp][1];
                    }
                } else if constexpr (sizeof(F) == 4) {
                    if (nk == K) {
                        st4_any(xd, res[cp]);
                    } else {
                        #pragma unroll
                        for (int kk = 0; kk < K; ++kk)
                            if (kk < nk) xd[kk] = res[cp][kk];
                    }
                } else {
                    #pragma unroll
                    for (int kk = 0; kk < K; ++kk)
                        if (kk < nk) xd[kk] = res[cp][kk];
                }
            }
        }
        if constexpr (R > 1) {
            issue(dd + R - 1, cd_next);
            cd_next = cd_n1;
            cd_n1 = cd_n2;
            cd_n2 = cd_n3;
            cd_n3 = code_of(dd + R + 3);                // consumed four steps later
        }
        __syncthreads();
    }
    cp_async_wait_n<0>();
}

// Wavefront steps [dd0, dd1) of one sweep pass for the velocities that are
// coupled to one upwind neighbour only, or to none (the sign of u or v puts the
// other neighbour downwind, and its coefficient is an exact zero): such a
// velocity is independent along every row (coupled along x only) or every
// column (along y only), or every cell (neither), so one thread per (line,
// velocity) walks the cells of its line that lie on the segment's diagonals,
// with no barrier.  Consecutive threads take consecutive velocities of the
// same line, so every access is coalesced, and each thread loads the inputs of
// four cells before it updates them in order.  The update of a cell is the
// wavefront kernel's with the zero coupling left out; boundary-line cells take
// their folded inputs (incoming velocities) or keep the value of their line
// walk (outgoing velocities and the corner), as in the wavefront kernel.  The
// backward pass leaves the uncoupled velocities as they are (x = x).
// Block b: rows (class 0) first, nbr blocks of 128 velocities per row, then
// columns (class 1), nbc per column, then cells of no coupling by rows, nbe per
// row (0 in the backward pass).
template <typename F, bool BODIES>
__global__ void __launch_bounds__(128) k_sgs_lines(MicroArgs M, const F* __restrict__ invD, const F* __restrict__ r,
                                                   F* __restrict__ x, const F* __restrict__ fold, int pass, int dd0,
                                                   int dd1, int nbr, int nbc, int nbe)
{
    constexpr int K = kInteriorKc, U = 4;
    const LevelDev& L = M.L;
    const VelDev& Vg = M.V;
    const int nx = L.nx, ny = L.ny, nv = Vg.nv, nd = nx + ny - 1, nls = M.P.nl_max;
    const size_t nc = L.nc;
    int b = blockIdx.x, cls, line, q;
    if (b < nbr * ny) {
        cls = 0; line = b / nbr; q = (b % nbr) * 128 + threadIdx.x;
        if (q >= Vg.nrow[pass]) return;
    } else if ((b -= nbr * ny) < nbc * nx) {
        cls = 1; line = b / nbc; q = (b % nbc) * 128 + threadIdx.x;
        if (q >= Vg.ncol[pass]) return;
        q += Vg.nrow[pass];
    } else {
        b -= nbc * nx;
        cls = 2; line = b / nbe; q = (b % nbe) * 128 + threadIdx.x;
        if (q >= Vg.nelem[pass]) return;
        q += Vg.nrow[pass] + Vg.ncol[pass];
    }
    const int k = Vg.lk[pass][q];
    const F u = (F)Vg.u[k], v = (F)Vg.v[k];
    const F cu = pass == 0 ? (u > F(0) ? -u : F(0)) : (u < F(0) ? u : F(0));
    const F cv = pass == 0 ? (v > F(0) ? -v : F(0)) : (v < F(0) ? v : F(0));
    const F cc = cls == 0 ? cu : cls == 1 ? cv : F(0);   // coefficient of the neighbour along the line
    // the line's cells on diagonals [dlo, dhi): position p along the line (i for rows, j for columns)
    const int dlo = pass == 0 ? dd0 : nd - dd1, dhi = pass == 0 ? dd1 : nd - dd0;
    const int len = cls == 1 ? ny : nx;
    const int p0 = max(0, dlo - line), p1 = min(len, dhi - line);
    if (p1 <= p0) return;
    const int n = p1 - p0, step = pass == 0 ? 1 : -1, pfirst = pass == 0 ? p0 : p1 - 1;
    const int ib = pass == 0 ? 0 : nx - 1, jb = pass == 0 ? 0 : ny - 1;
    const int* __restrict__ code = M.P.code[pass];
    const F* src = pass == 0 ? r : x;
    const int kb = k / K, kk = k - kb * K;
    auto cell_of = [&](int p) { return cls == 1 ? p * nx + line : line * nx + p; };
    // value of the upwind neighbour of the first cell (from an earlier segment), 0 at the line's start
    F xp[2] = {F(0), F(0)};
    const int pnb = pfirst - step;
    if (cls != 2 && pnb >= 0 && pnb < len) {
        const size_t cn = (size_t)cell_of(pnb) * nv + k;
        xp[0] = x[cn];
        xp[1] = x[nc * nv + cn];
    }
    for (int s0 = 0; s0 < n; s0 += U) {
        // inputs of up to U cells: kind 0 ordinary, 1 folded (incoming at a line face),
        // 2 final (outgoing at a line face, or the corner), 3 in a body
        F a[U][2], iv[U], rd[U];
        int kind[U];
        #pragma unroll
        for (int t = 0; t < U; ++t) {
            kind[t] = 2;
            a[t][0] = a[t][1] = iv[t] = rd[t] = F(0);
            if (s0 + t >= n) continue;
            const int p = pfirst + (s0 + t) * step;
            const int c = cell_of(p), i = cls == 1 ? line : p, j = cls == 1 ? p : line;
            bool hasx, hasy;
            int e = 0;
            if constexpr (BODIES) {
                const int cd = code[c];
                if (cd == -2) { kind[t] = 3; continue; }
                hasx = cd >= 0 && (cd & 2);
                hasy = cd >= 0 && (cd & 1);
                e = cd >> 2;
            } else {
                hasx = i == ib;
                hasy = j == jb;
                e = hasx ? (pass == 0 ? j : ny - 1 - j) : ny + (pass == 0 ? i : nx - 1 - i);
            }
            // the line face across which this class's velocities enter, and the one they leave by
            const bool fin = cls == 0 ? hasy : cls == 1 ? hasx : (hasx || hasy);
            const bool fld = !fin && (cls == 0 ? hasx : cls == 1 ? hasy : false);
            const size_t id = (size_t)c * nv + k;
            if (fin) {
                kind[t] = 2;
                if (cls != 2) { a[t][0] = x[id]; a[t][1] = x[nc * nv + id]; }
            } else if (fld) {
                kind[t] = 1;
                const F* fo = fold + ((size_t)(kb * nls + e) * 3) * K + kk;
                a[t][0] = fo[0]; a[t][1] = fo[K]; iv[t] = fo[2 * K];
            } else {
                kind[t] = 0;
                a[t][0] = src[id]; a[t][1] = src[nc * nv + id]; iv[t] = invD[id];
                rd[t] = cls == 0 ? (F)L.rdx[i] : cls == 1 ? (F)L.rdy[j] : F(0);
            }
        }
        #pragma unroll
        for (int t = 0; t < U; ++t) {
            if (s0 + t >= n) continue;
            const int p = pfirst + (s0 + t) * step;
            const size_t id = (size_t)cell_of(p) * nv + k;
            F res[2];
            #pragma unroll
            for (int cp = 0; cp < 2; ++cp) {
                if (kind[t] == 3) res[cp] = F(0);
                else if (kind[t] == 2) res[cp] = a[t][cp];
                else if (kind[t] == 1) res[cp] = pass == 0 ? a[t][cp] * iv[t] : a[t][cp];
                else {
                    const F y = cls == 2 ? F(0) : cc * rd[t] * xp[cp];
                    res[cp] = pass == 0 ? (a[t][cp] - y) * iv[t] : a[t][cp] - y * iv[t];
                }
                xp[cp] = res[cp];
            }
            if (kind[t] != 2) {
                x[id] = res[0];
                x[nc * nv + id] = res[1];
            }
        }
    }
}

// Sum of squares of n values (deterministic: fixed grid, fixed per-thread order,
// fixed reduction tree), for the decisions of the adaptive multigrid cycle.
constexpr int kSumsqBlocks = 128;
template <typename T>
__global__ void k_sumsq_part(const T* __restrict__ a, size_t n, double* __restrict__ part)
{
    __shared__ double red[32];
    double s[1] = {0.0};
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const double v = (double)a[q];
        s[0] += v * v;
    }
    block_sum<1>(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}
__global__ void k_sumsq_final(const double* __restrict__ part, int nb, double* __restrict__ out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double t = 0.0;
        for (int b = 0; b < nb; ++b) t += part[b];
        *out = t;
    }
}
template <typename T>
cudaError_t launch_sumsq(const T* a, size_t n, double* part, double* out, cudaStream_t st)
{
    k_sumsq_part<T><<<kSumsqBlocks, 256, 0, st>>>(a, n, part);
    k_sumsq_final<<<1, 32, 0, st>>>(part, kSumsqBlocks, out);
    return cudaGetLastError();
}
template cudaError_t launch_sumsq<float>(const float*, size_t, double*, double*, cudaStream_t);
template cudaError_t launch_sumsq<double>(const double*, size_t, double*, double*, cudaStream_t);

// Coupling classes of one pass (0 forward, 1 backward) for the velocity nodes
// (u_k, v_k): the wavefront blocks and the lists of the other velocities.
void sweep_classes(const double* u, const double* v, int nv, int pass, std::vector<int>& wblk, std::vector<int>& lk,
                   int& nrow, int& ncol, int& nelem)
{
    const int K = kInteriorKc, nblk = (nv + K - 1) / K;
    auto cx = [&](int k) { return pass == 0 ? u[k] > 0.0 : u[k] < 0.0; };
    auto cy = [&](int k) { return pass == 0 ? v[k] > 0.0 : v[k] < 0.0; };
    std::vector<int> rows, cols, elem;
    wblk.clear();
    for (int b = 0; b < nblk; ++b) {
        bool wave = false;
        for (int k = b * K; k < std::min(nv, b * K + K); ++k) wave = wave || (cx(k) && cy(k));
        if (wave) { wblk.push_back(b); continue; }
        for (int k = b * K; k < std::min(nv, b * K + K); ++k)
            (cx(k) ? rows : cy(k) ? cols : elem).push_back(k);
    }
    nrow = (int)rows.size(); ncol = (int)cols.size(); nelem = (int)elem.size();
    lk = rows;
    lk.insert(lk.end(), cols.begin(), cols.end());
    lk.insert(lk.end(), elem.begin(), elem.end());
}

// sweep scratch (elements of the storage type): corner copy, wall densities of
// the edge lines and the body lines, folded line inputs
size_t micro_fold_offset(int nv, int nlines) { return ((2 * (size_t)nv + (2 + (size_t)nlines) * kMaxLine + 3) / 4) * 4; }
size_t micro_scratch_elems(int nv, int nl, int nlines)
{
    return micro_fold_offset(nv, nlines) + (size_t)((nv + kInteriorKc - 1) / kInteriorKc) * nl * 3 * kInteriorKc;
}

template <typename F>
cudaError_t launch_micro_sgs(const MicroArgs& m, const SweepPlanHost& plan, const double* Zw, const F* invD,
                             const F* r, F* x, F* xcorner, cudaStream_t st)
{
    int nlines = 0;
    for (int p = 0; p < 2; ++p)
        for (int b = 0; b < plan.nbrk[p]; ++b)
            nlines = std::max(nlines, plan.brk[p][b].q0 + plan.brk[p][b].nq);
    F* rho_lines = xcorner + 2 * (size_t)m.V.nv;       // (2 + body lines) x kMaxLine wall densities
    F* fold = xcorner + micro_fold_offset(m.V.nv, nlines);
    const int ngroups = (m.V.nu + 1) / 2;
    const int nloc = ((ngroups + kChainCluster - 1) / kChainCluster) * 2 * m.V.nvv;
    if (nloc > kChainKptMax * kChainThreads) return cudaErrorInvalidValue;
    if (m.L.nx > kMaxLine || m.L.ny > kMaxLine) return cudaErrorInvalidValue;
    const int kpt = (nloc + kChainThreads - 1) / kChainThreads;
    const size_t rslot = sizeof(F) * (size_t)(kpt <= 1 ? 1 : kpt <= 2 ? 2 : kpt <= 4 ? 4 : kpt <= 8 ? 8 : 16) * 3 *
                         kChainThreads;
    int RA = (int)((96 * 1024) / rslot);
    RA = RA < 1 ? 1 : (RA > kWaveRingMax ? kWaveRingMax : RA);
    size_t smem = sizeof(F) * 2 * nloc + (sizeof(F) + sizeof(int)) * (size_t)nloc + rslot * RA;
    void (*chain)(MicroArgs, const double*, const F*, const F*, F*, const F*, F*, int, int) =
        kpt <= 1 ? k_sgs_chain<F, 1> : kpt <= 2 ? k_sgs_chain<F, 2> : kpt <= 4 ? k_sgs_chain<F, 4>
                 : kpt <= 8 ? k_sgs_chain<F, 8> : k_sgs_chain<F, 16>;
    void (*chain_b)(MicroArgs, const double*, const F*, const F*, F*, F*, int, int, int) =
        kpt <= 1 ? k_sgs_chain_body<F, 1> : kpt <= 2 ? k_sgs_chain_body<F, 2> : kpt <= 4 ? k_sgs_chain_body<F, 4>
                 : kpt <= 8 ? k_sgs_chain_body<F, 8> : k_sgs_chain_body<F, 16>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(chain, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (nlines > 0) {
            e = cudaFuncSetAttribute(chain_b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
    }
    const int nblk = (m.V.nv + kInteriorKc - 1) / kInteriorKc;
    const int maxdiag = m.L.nx < m.L.ny ? m.L.nx : m.L.ny;
    const int nthr = ((maxdiag + 31) / 32) * 32;       // one thread per cell of the longest diagonal
    const bool vec = (m.V.nv * sizeof(F)) % 16 == 0;
    const size_t nl = (size_t)m.L.nx + m.L.ny;
    const size_t fixed = sizeof(F) * (2 * (size_t)m.L.nx * 2 * kInteriorKc + nl);
    const size_t slot = sizeof(F) * 3 * (size_t)nthr * kInteriorKc + sizeof(int) * (size_t)nthr;
    constexpr size_t kSmemMax = 227 * 1024;
    if (fixed + slot > kSmemMax) return cudaErrorInvalidValue;
    const size_t rfit = (kSmemMax - fixed) / slot;
    // On a large level the wavefront kernel takes only the blocks of velocities coupled in
    // both directions and the line-class kernel the rest; on a small one the wavefront's
    // dependency chain, not its traffic, sets the time and one wavefront launch over every
    // block is faster than two launches.
    const bool split = plan.split == 1 || (plan.split == 0 && (size_t)m.L.nc * m.V.nv >= kSweepSplitMinCv);
    // Ring depth: the deepest of 8, 4, 2 stages whose shared memory lets the launch's CTAs
    // be resident in the fewest rounds (a CTA's time is the dependency chain of its steps,
    // so a second round of CTAs doubles the launch).
    int R = rfit >= 8 ? 8 : rfit >= 4 ? 4 : rfit >= 2 ? 2 : 1;
    {
        static int nsm = 0, smem_sm = 0, resv = 0;
        if (nsm == 0) {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
            cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
            cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
        }
        const long grid = split ? std::max(m.V.nwblk[0], m.V.nwblk[1]) : nblk;
        auto rounds = [&](int r) -> long {
            const long per = std::min<long>((long)smem_sm / (long)(fixed + slot * r + resv), 2048 / nthr);
            return per > 0 ? (grid + per * nsm - 1) / (per * nsm) : LONG_MAX;
        };
        if (nsm > 0 && smem_sm > 0 && R >= 2) {
            int best = R;
            for (int r = R / 2; r >= 2; r /= 2)
                if (rounds(r) < rounds(best)) best = r;
            R = best;
        }
    }
    void (*wave)(MicroArgs, const F*, const F*, F*, const F*, int, int, int, int);
    if (m.P.bodies) {
        if (vec) wave = R == 8 ? k_sgs_wave<F, 8, true, true> : R == 4 ? k_sgs_wave<F, 4, true, true> : R == 2 ? k_sgs_wave<F, 2, true, true> : k_sgs_wave<F, 1, true, true>;
        else wave = R == 8 ? k_sgs_wave<F, 8, false, true> : R == 4 ? k_sgs_wave<F, 4, false, true> : R == 2 ? k_sgs_wave<F, 2, false, true> : k_sgs_wave<F, 1, false, true>;
    } else {
        if (vec) wave = R == 8 ? k_sgs_wave<F, 8, true, false> : R == 4 ? k_sgs_wave<F, 4, true, false> : R == 2 ? k_sgs_wave<F, 2, true, false> : k_sgs_wave<F, 1, true, false>;
        else wave = R == 8 ? k_sgs_wave<F, 8, false, false> : R == 4 ? k_sgs_wave<F, 4, false, false> : R == 2 ? k_sgs_wave<F, 2, false, false> : k_sgs_wave<F, 1, false, false>;
    }
    const size_t wsmem = fixed + slot * R;
    if (wsmem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(wave, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsmem);
        if (e != cudaSuccess) return e;
    }
    void (*lines)(MicroArgs, const F*, const F*, F*, const F*, int, int, int, int, int, int) =
        m.P.bodies ? k_sgs_lines<F, true> : k_sgs_lines<F, false>;
    // one segment (split: see above)
    // timing mode: an event pair around a launch, with the cell-velocity pairs it sweeps
    auto timed = [&](int kind, double units, auto&& launch) {
        SweepTimer* T = plan.timer;
        if (!T) { launch(); return cudaGetLastError(); }
        while ((int)T->ev.size() < 2 * (T->used + 1)) {
            cudaEvent_t e;
            cudaError_t ce = cudaEventCreate(&e);
            if (ce != cudaSuccess) return ce;
            T->ev.push_back(e);
        }
        if ((int)T->kind.size() <= T->used) { T->kind.resize(T->used + 1); T->units.resize(T->used + 1); }
        cudaError_t e = cudaEventRecord(T->ev[2 * T->used], st);
        if (e != cudaSuccess) return e;
        launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = cudaEventRecord(T->ev[2 * T->used + 1], st)) != cudaSuccess) return e;
        T->kind[T->used] = kind;
        T->units[T->used] = units;
        T->used++;
        return cudaSuccess;
    };
    auto segment = [&](int pass, int dd, int end) {
        const int nw = split ? m.V.nwblk[pass] : nblk;
        const int nbr = (m.V.nrow[pass] + 127) / 128, nbc = (m.V.ncol[pass] + 127) / 128;
        const int nbe = pass == 0 ? (m.V.nelem[pass] + 127) / 128 : 0;
        const int nb = split ? nbr * m.L.ny + nbc * m.L.nx + nbe * m.L.ny : 0;
        double cells = 0.0;                            // cells on the segment's diagonals
        for (int q = dd; q < end; ++q) {
            const int d = pass == 0 ? q : m.L.nx + m.L.ny - 2 - q;
            cells += std::min(m.L.nx - 1, d) - std::max(0, d - (m.L.ny - 1)) + 1;
        }
        const double kl = (double)m.V.nrow[pass] + m.V.ncol[pass] + (pass == 0 ? m.V.nelem[pass] : 0);
        const double kw = std::min((double)nw * kInteriorKc, (double)m.V.nv);
        cudaError_t e = cudaSuccess;
        if (nb > 0 && (e = timed(1, cells * kl, [&] {
                lines<<<nb, 128, 0, st>>>(m, invD, r, x, fold, pass, dd, end, nbr, nbc, nbe);
            })) != cudaSuccess)
            return e;
        if (nw > 0 && (e = timed(0, cells * kw, [&] {
                wave<<<nw, nthr, wsmem, st>>>(m, invD, r, x, fold, pass, dd, end, split ? 1 : 0);
            })) != cudaSuccess)
            return e;
        return cudaSuccess;
    };
    auto fold_range = [&](int pass, int e0, int ne) {
        const int n = nblk * ne * kInteriorKc;
        if (n > 0) k_line_fold<F><<<(n + 255) / 256, 256, 0, st>>>(m, invD, r, x, rho_lines, fold, pass, e0, ne);
        return cudaGetLastError();
    };
    const size_t nc = m.L.nc, nv = m.V.nv, corner = (size_t)m.L.nc - 1;
    const int nd = m.L.nx + m.L.ny - 1;
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1)
            for (int cp = 0; cp < 2; ++cp) {
                cudaError_t e = cudaMemcpyAsync(xcorner + cp * nv, x + (cp * nc + corner) * nv, nv * sizeof(F),
                                                cudaMemcpyDeviceToDevice, st);
                if (e != cudaSuccess) return e;
            }
        chain<<<2 * kChainCluster, kChainThreads, smem, st>>>(m, Zw, invD, r, x, xcorner, rho_lines, pass, RA);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if ((e = fold_range(pass, 0, m.P.nl[pass])) != cudaSuccess) return e;
        // wavefront segments between the body lines' walks
        int dd = 0;
        for (int b = 0; b <= plan.nbrk[pass]; ++b) {
            const int end = b < plan.nbrk[pass] ? plan.brk[pass][b].dd : nd;
            if (end > dd) {
                if ((e = segment(pass, dd, end)) != cudaSuccess) return e;
                dd = end;
            }
            if (b < plan.nbrk[pass]) {
                const SweepBreak& k = plan.brk[pass][b];
                chain_b<<<k.nq * kChainCluster, kChainThreads, smem, st>>>(m, Zw, invD, r, x, rho_lines, pass, k.q0, RA);
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
                if ((e = fold_range(pass, k.e0, k.ne)) != cudaSuccess) return e;
            }
        }
    }
    return cudaSuccess;
}
template cudaError_t launch_micro_sgs<double>(const MicroArgs&, const SweepPlanHost&, const double*, const double*,
                                              const double*, double*, double*, cudaStream_t);
template cudaError_t launch_micro_sgs<float>(const MicroArgs&, const SweepPlanHost&, const double*, const float*,
                                             const float*, float*, float*, cudaStream_t);

// ---------------------------------------------------------------------------
// r -= A x (full operator with every neighbour and ghost), acc += x
template <typename F>
__global__ void __launch_bounds__(256) k_micro_renew(MicroArgs M, const double* __restrict__ Zw, const F* __restrict__ x,
                                                     F* __restrict__ r, F* __restrict__ acc, int renew)
{
    __shared__ double red[32 * 4];
    const LevelDev& L = M.L;
    const VelDev& Vg = M.V;
    const int c = blockIdx.x, nx = L.nx, nv = Vg.nv, i = c % nx, j = c / nx;
    const size_t nc = L.nc;
    const bool vec = sizeof(F) == 4 && (nv & 3) == 0;   // 16-byte accesses over four velocities
    if (acc) {
        if (vec) {
            for (int cp = 0; cp < 2; ++cp)
                for (int g = threadIdx.x; g < nv / 4; g += blockDim.x) {
                    const size_t id = (cp * nc + c) * nv + 4 * g;
                    F xa[4], aa[4];
                    ld4(x + id, xa);
                    ld4(acc + id, aa);
                    #pragma unroll
                    for (int q = 0; q < 4; ++q) aa[q] = aa[q] + xa[q];
                    st4(acc + id, aa);
                }
        } else {
            // four velocities a block apart per thread: coalesced, eight loads in flight
            const int bs = blockDim.x;
            for (int cp = 0; cp < 2; ++cp)
                for (int k0 = threadIdx.x; k0 < nv; k0 += 4 * bs) {
                    const size_t id0 = (cp * nc + c) * nv + k0;
                    F xa[4], aa[4];
                    #pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (k0 + q * bs < nv) { xa[q] = x[id0 + q * bs]; aa[q] = acc[id0 + q * bs]; }
                    #pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (k0 + q * bs < nv) acc[id0 + q * bs] = aa[q] + xa[q];
                }
        }
    }
    if (!renew || L.solid[c]) return;   // a body keeps a zero residual
    BFace bf[4];
    int nb = side_faces(L, i, j, 2, bf);
    __shared__ F srho[4], sgeo[3];
    const F* __restrict__ vu = VelT<F>::u(Vg);
    const F* __restrict__ vv = VelT<F>::v(Vg);
    const F* __restrict__ vw = VelT<F>::w(Vg);
    int nwall = 0;
    for (int b = 0; b < nb; ++b) nwall += M.bc[bf[b].bc].type == BC_WALL;
    if (nwall > 0) {
        Acc<F> sa[4];
        for (int k = threadIdx.x; k < nv; k += blockDim.x)
            for (int b = 0; b < nb; ++b) {
                if (M.bc[bf[b].bc].type != BC_WALL) continue;
                F uo = bf[b].axis == 0 ? vu[k] : vv[k];
                uo = bf[b].outsign < 0 ? -uo : uo;
                if (uo > F(0)) sa[b].add(vw[k] * uo * x[c * (size_t)nv + k]);
            }
        double sd[4];
        block_total<4>(sa, red, sd);
        if (threadIdx.x == 0)
            for (int b = 0; b < 4; ++b)
                srho[b] = b < nb && M.bc[bf[b].bc].type == BC_WALL
                              ? (F)(-sd[b] / Zw[bf[b].bc * 4 + bf[b].axis * 2 + (bf[b].outsign > 0)]) : F(0);
    }
    if (threadIdx.x == 0) {
        sgeo[0] = (F)M.inv_tau[c]; sgeo[1] = (F)L.rdx[i]; sgeo[2] = (F)L.rdy[j];
        if (nwall == 0) srho[0] = srho[1] = srho[2] = srho[3] = F(0);
    }
    __syncthreads();
    F rho[4] = {srho[0], srho[1], srho[2], srho[3]};
    const F itau = sgeo[0], rdxi = sgeo[1], rdyj = sgeo[2];
    if (vec && nb == 0) {
        // interior cell: four velocities per thread, both components, 16-byte accesses
        for (int g = threadIdx.x; g < nv / 4; g += blockDim.x) {
            F u[4], v[4], cW[4], cE[4], cS[4], cN[4], dg[4];
            ld4(vu + 4 * g, u);
            ld4(vv + 4 * g, v);
            #pragma unroll
            for (int q = 0; q < 4; ++q) {
                dg[q] = itau + geomD_r<F>(rdxi, rdyj, u[q], v[q]);
                cW[q] = Dface<F>(0, -1, rdxi, u[q], v[q]);
                cE[q] = Dface<F>(0, 1, rdxi, u[q], v[q]);
                cS[q] = Dface<F>(1, -1, rdyj, u[q], v[q]);
                cN[q] = Dface<F>(1, 1, rdyj, u[q], v[q]);
            }
            #pragma unroll
            for (int cp = 0; cp < 2; ++cp) {
                const size_t id = (cp * nc + c) * nv + 4 * g;
                F xc[4], xw[4], xe[4], xs[4], xn[4], rr[4];
                ld4(x + id, xc);
                ld4(x + id - nv, xw);
                ld4(x + id + nv, xe);
                ld4(x + id - (size_t)nx * nv, xs);
                ld4(x + id + (size_t)nx * nv, xn);
                ld4(r + id, rr);
                #pragma unroll
                for (int q = 0; q < 4; ++q) {
                    F a = dg[q] * xc[q];
                    a += cW[q] * xw[q];
                    a += cE[q] * xe[q];
                    a += cS[q] * xs[q];
                    a += cN[q] * xn[q];
                    rr[q] = rr[q] - a;
                }
                st4(r + id, rr);
            }
        }
        return;
    }
    if (nb == 0) {
        // interior cell, any velocity count: four velocities a block apart per thread, so
        // that every access is coalesced and 24 loads are in flight per thread (one
        // velocity at a time leaves the cell's two DRAM streams latency-bound)
        const int bs = blockDim.x;
        for (int cp = 0; cp < 2; ++cp) {
            const F* xb = x + cp * nc * nv;
            F* rb = r + cp * nc * nv;
            for (int k0 = threadIdx.x; k0 < nv; k0 += 4 * bs) {
                F xc[4], xw[4], xe[4], xs[4], xn[4], rr[4];
                #pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int k = k0 + q * bs;
                    if (k < nv) {
                        const size_t id = (size_t)c * nv + k;
                        xc[q] = xb[id]; xw[q] = xb[id - nv]; xe[q] = xb[id + nv];
                        xs[q] = xb[id - (size_t)nx * nv]; xn[q] = xb[id + (size_t)nx * nv]; rr[q] = rb[id];
                    }
                }
                #pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int k = k0 + q * bs;
                    if (k < nv) {
                        const F u = vu[k], v = vv[k];
                        F a = (itau + geomD_r<F>(rdxi, rdyj, u, v)) * xc[q];
                        a += Dface<F>(0, -1, rdxi, u, v) * xw[q];
                        a += Dface<F>(0, 1, rdxi, u, v) * xe[q];
                        a += Dface<F>(1, -1, rdyj, u, v) * xs[q];
                        a += Dface<F>(1, 1, rdyj, u, v) * xn[q];
                        rb[(size_t)c * nv + k] = rr[q] - a;
                    }
                }
            }
        }
        return;
    }
    // interior neighbours (faces without a BC id)
    const bool hw = L.fbx[j * (nx + 1) + i] < 0, he = L.fbx[j * (nx + 1) + i + 1] < 0;
    const bool hs = L.fby[j * nx + i] < 0, hn = L.fby[(j + 1) * nx + i] < 0;
    for (int cp = 0; cp < 2; ++cp) {
        const F* xb = x + cp * nc * nv;
        F* rb = r + cp * nc * nv;
        for (int k = threadIdx.x; k < nv; k += blockDim.x) {
            const F u = vu[k], v = vv[k];
            size_t id = (size_t)c * nv + k;
            F a = (itau + geomD_r<F>(rdxi, rdyj, u, v)) * xb[id];
            if (hw) a += Dface<F>(0, -1, rdxi, u, v) * xb[id - nv];
            if (he) a += Dface<F>(0, 1, rdxi, u, v) * xb[id + nv];
            if (hs) a += Dface<F>(1, -1, rdyj, u, v) * xb[id - (size_t)nx * nv];
            if (hn) a += Dface<F>(1, 1, rdyj, u, v) * xb[id + (size_t)nx * nv];
            for (int b = 0; b < nb; ++b) {
                F Db = Dface<F>(bf[b].axis, bf[b].outsign, (F)bf[b].rS, u, v);
                if (Db == F(0)) continue;
                int ty = M.bc[bf[b].bc].type;
                if (ty == BC_WALL)
                    a += Db * (F)(M.Cw[(size_t)bf[b].bc * nv + k] * (cp == 0 ? 1.0 : kKint * M.bc[bf[b].bc].t / 4.0)) * rho[b];
                else if (ty == BC_SYMMETRY) {
                    int aa = k / Vg.nvv, bb = k - aa * Vg.nvv;
                    int km = bf[b].axis == 0 ? (Vg.nu - 1 - aa) * Vg.nvv + bb : aa * Vg.nvv + (Vg.nvv - 1 - bb);
                    a += Db * xb[(size_t)c * nv + km];
                } else if (ty == BC_OUTFLOW) {
                    a += Db * xb[id];
                }
            }
            rb[id] = rb[id] - a;
        }
    }
}

template <typename F>
cudaError_t launch_micro_renew(const MicroArgs& m, const double* Zw, const F* x, F* r, F* acc, int renew,
                                 cudaStream_t st)
{
    k_micro_renew<F><<<m.L.nc, m.V.nv >= 256 ? 256 : 128, 0, st>>>(m, Zw, x, r, acc, renew);
    return cudaGetLastError();
}
template cudaError_t launch_micro_renew<double>(const MicroArgs&, const double*, const double*, double*, double*,
                                                int, cudaStream_t);
template cudaError_t launch_micro_renew<float>(const MicroArgs&, const double*, const float*, float*, float*, int,
                                               cudaStream_t);

// ---------------------------------------------------------------------------
// Steps 6-7: f += df (when df != null), then W = sum w psi f and q = sum w c (c^2 G/2 + H)
template <typename F>
__global__ void __launch_bounds__(256) k_update_moments(LevelDev L, VelDev Vg, F* __restrict__ f, const F* __restrict__ df,
                                                        double* __restrict__ W, double* __restrict__ q)
{
    __shared__ double red[32 * 4];
    const int c = blockIdx.x, nv = Vg.nv;
    const size_t nc = L.nc;
    __shared__ F sUV[2];
    F* fG = f + (size_t)c * nv;
    F* fH = f + (nc + c) * (size_t)nv;
    const F* __restrict__ vu = VelT<F>::u(Vg);
    const F* __restrict__ vv = VelT<F>::v(Vg);
    const F* __restrict__ vw = VelT<F>::w(Vg);
    __shared__ int sok;
    // Each thread takes four velocities a block apart per round and issues all their
    // loads before the arithmetic (the summation order is that of k = tid, tid + bs, ...).
    const int bs = blockDim.x;
    Acc<F> sa[4];
    for (int k0 = threadIdx.x; k0 < nv; k0 += 4 * bs) {
        F g[4], h[4];
        #pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = k0 + q * bs;
            if (k < nv) {
                g[q] = fG[k]; h[q] = fH[k];
                if (df) {
                    g[q] = g[q] + df[(size_t)c * nv + k];
                    h[q] = h[q] + df[(nc + c) * (size_t)nv + k];
                }
            }
        }
        #pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = k0 + q * bs;
            if (k < nv) {
                const F u = vu[k], v = vv[k], w = vw[k];
                sa[0].add(w * g[q]); sa[1].add(w * u * g[q]); sa[2].add(w * v * g[q]);
                sa[3].add(w * (F(0.5) * (u * u + v * v) * g[q] + h[q]));
            }
        }
    }
    double s[4];
    block_total<4>(sa, red, s);
    if (df) {
        // commit f + df, unless it would leave the cell with non-positive density or
        // internal energy: then the cell keeps f and its moments are those of f
        if (threadIdx.x == 0) sok = s[0] > 0.0 && s[3] * s[0] - 0.5 * (s[1] * s[1] + s[2] * s[2]) > 0.0;
        __syncthreads();
        if (sok) {
            for (int k0 = threadIdx.x; k0 < nv; k0 += 4 * bs) {
                F g[4], h[4], dg[4], dh[4];
                #pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int k = k0 + q * bs;
                    if (k < nv) {
                        g[q] = fG[k]; h[q] = fH[k];
                        dg[q] = df[(size_t)c * nv + k]; dh[q] = df[(nc + c) * (size_t)nv + k];
                    }
                }
                #pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int k = k0 + q * bs;
                    if (k < nv) { fG[k] = g[q] + dg[q]; fH[k] = h[q] + dh[q]; }
                }
            }
        } else {
            Acc<F> sb[4];
            for (int k = threadIdx.x; k < nv; k += blockDim.x) {
                const F g = fG[k], h = fH[k], u = vu[k], v = vv[k], w = vw[k];
                sb[0].add(w * g); sb[1].add(w * u * g); sb[2].add(w * v * g);
                sb[3].add(w * (F(0.5) * (u * u + v * v) * g + h));
            }
            block_total<4>(sb, red, s);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double ir = rcp64(s[0]);
        sUV[0] = (F)(s[1] * ir);
        sUV[1] = (F)(s[2] * ir);
    }
    __syncthreads();
    const F fU = sUV[0], fV = sUV[1];
    Acc<F> ta[2];
    for (int k0 = threadIdx.x; k0 < nv; k0 += 4 * bs) {
        F g[4], h[4];
        #pragma unroll
        for (int q = 0; q < 4; ++q)
            if (k0 + q * bs < nv) { g[q] = fG[k0 + q * bs]; h[q] = fH[k0 + q * bs]; }
        #pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = k0 + q * bs;
            if (k < nv) {
                F cx = vu[k] - fU, cy = vv[k] - fV;
                F e = F(0.5) * (cx * cx + cy * cy) * g[q] + h[q];
                ta[0].add(vw[k] * cx * e);
                ta[1].add(vw[k] * cy * e);
            }
        }
    }
    double t[2];
    block_total<2>(ta, red, t);
    if (threadIdx.x == 0) {
        for (int m = 0; m < 4; ++m) W[4 * (size_t)c + m] = s[m];
        q[2 * (size_t)c] = t[0];
        q[2 * (size_t)c + 1] = t[1];
    }
}

template <typename F>
cudaError_t launch_update_moments(const LevelDev& L, const VelDev& V, F* f, const F* df, double* W, double* q,
                                  cudaStream_t st)
{
    k_update_moments<F><<<L.nc, V.nv >= 256 ? 256 : 128, 0, st>>>(L, V, f, df, W, q);
    return cudaGetLastError();
}
template <typename F>
cudaError_t launch_moments(const LevelDev& L, const VelDev& V, const F* f, double* W, double* q, cudaStream_t st)
{
    return launch_update_moments<F>(L, V, const_cast<F*>(f), nullptr, W, q, st);
}
template cudaError_t launch_update_moments<double>(const LevelDev&, const VelDev&, double*, const double*, double*,
                                                   double*, cudaStream_t);
template cudaError_t launch_moments<double>(const LevelDev&, const VelDev&, const double*, double*, double*,
                                            cudaStream_t);
template cudaError_t launch_update_moments<float>(const LevelDev&, const VelDev&, float*, const float*, double*,
                                                  double*, cudaStream_t);
template cudaError_t launch_moments<float>(const LevelDev&, const VelDev&, const float*, double*, double*,
                                           cudaStream_t);

// discrete Maxwellian of (rho, U, V, T) per cell
// Full-multigrid start-up: a fine cell whose prolonged state f has
// non-positive density or internal energy takes the f of its coarse cell
// (fc, the next coarser mesh with ncx cells per row).  One CTA per fine cell.
template <typename F>
__global__ void __launch_bounds__(256) k_state_fallback(LevelDev L, VelDev Vg, int ncx, size_t ncc,
                                                        const F* __restrict__ fc, F* __restrict__ f)
{
    __shared__ double red[32 * 4];
    const int c = blockIdx.x, nv = Vg.nv, i = c % L.nx, j = c / L.nx;
    const size_t nc = L.nc, cc = (size_t)(j / 2) * ncx + i / 2;
    const F* __restrict__ vu = VelT<F>::u(Vg);
    const F* __restrict__ vv = VelT<F>::v(Vg);
    const F* __restrict__ vw = VelT<F>::w(Vg);
    Acc<F> sa[4];
    for (int k = threadIdx.x; k < nv; k += blockDim.x) {
        const F g = f[(size_t)c * nv + k], h = f[(nc + c) * (size_t)nv + k], u = vu[k], v = vv[k], w = vw[k];
        sa[0].add(w * g); sa[1].add(w * u * g); sa[2].add(w * v * g);
        sa[3].add(w * (F(0.5) * (u * u + v * v) * g + h));
    }
    double s[4];
    block_total<4>(sa, red, s);
    if (s[0] > 0.0 && s[3] * s[0] - 0.5 * (s[1] * s[1] + s[2] * s[2]) > 0.0) return;
    for (int k = threadIdx.x; k < nv; k += blockDim.x) {
        f[(size_t)c * nv + k] = fc[cc * nv + k];
        f[(nc + c) * (size_t)nv + k] = fc[(ncc + cc) * nv + k];
    }
}
template <typename F>
cudaError_t launch_state_fallback(const LevelDev& L, const VelDev& V, int ncx, size_t ncc, const F* fc, F* f,
                                  cudaStream_t st)
{
    k_state_fallback<F><<<L.nc, V.nv >= 256 ? 256 : 128, 0, st>>>(L, V, ncx, ncc, fc, f);
    return cudaGetLastError();
}
template cudaError_t launch_state_fallback<double>(const LevelDev&, const VelDev&, int, size_t, const double*,
                                                   double*, cudaStream_t);
template cudaError_t launch_state_fallback<float>(const LevelDev&, const VelDev&, int, size_t, const float*, float*,
                                                  cudaStream_t);

template <typename F>
// The Maxwellian of velocity k = a nv_y + b factors into rho lam/pi e^{-lam (u_a - U)^2}
// times e^{-lam (v_b - V)^2}: nu + nv_y exponentials per cell (in FP64, tabled in shared
// memory), then two FP64 products per velocity.
__global__ void k_init_maxwell(LevelDev L, VelDev Vg, const double* __restrict__ prim, F* __restrict__ f)
{
    extern __shared__ double etab[];      // [nu] rho lam/pi e^{-lam (u_a - U)^2}, [nvv] e^{-lam (v_b - V)^2}
    const int c = blockIdx.x, nv = Vg.nv, nu = Vg.nu, nvv = Vg.nvv, tid = threadIdx.x, bs = blockDim.x;
    const size_t nc = L.nc;
    const double rho = prim[4 * c], U = prim[4 * c + 1], V = prim[4 * c + 2], lam = 1.0 / prim[4 * c + 3];
    const double hfac = kKint / (4.0 * lam);
    for (int e = tid; e < nu + nvv; e += bs) {
        if (e < nu) {
            const double d = Vg.ua[e] - U;
            etab[e] = rho * (lam / kPi) * exp(-lam * d * d);
        } else {
            const double d = Vg.vb[e - nu] - V;
            etab[e] = exp(-lam * d * d);
        }
    }
    __syncthreads();
    // velocity k = a * nvv + b of this thread, stepped by the block size without a division
    const int sa = bs / nvv, sb = bs - sa * nvv;
    int a = tid / nvv, b = tid - a * nvv;
    for (int k = tid; k < nv; k += bs, a += sa, b += sb) {
        if (b >= nvv) { b -= nvv; ++a; }
        const double g = etab[a] * etab[nu + b];
        f[(size_t)c * nv + k] = (F)g;
        f[(nc + c) * (size_t)nv + k] = (F)(g * hfac);
    }
}
template <typename F>
cudaError_t launch_init_maxwell(const LevelDev& L, const VelDev& V, const double* prim, F* f, cudaStream_t st)
{
    k_init_maxwell<F><<<L.nc, V.nv >= 256 ? 256 : 128, (V.nu + V.nvv) * sizeof(double), st>>>(L, V, prim, f);
    return cudaGetLastError();
}
template cudaError_t launch_init_maxwell<double>(const LevelDev&, const VelDev&, const double*, double*, cudaStream_t);
template cudaError_t launch_init_maxwell<float>(const LevelDev&, const VelDev&, const double*, float*, cudaStream_t);

// wall pressure, shear and heat flux of the faces in `faces` (axis * 2^30 + face index)
template <typename F>
__global__ void k_wall_quantities(LevelDev L, VelDev Vg, const BcDev* __restrict__ bc, const double* __restrict__ Cw,
                                  const F* __restrict__ f, int bcid, const int* __restrict__ faces,
                                  double* __restrict__ out)
{
    __shared__ double red[32 * 4];
    const int code = faces[blockIdx.x];
    const int axis = code >> 30, fi = code & ((1 << 30) - 1);
    const int nx = L.nx, nv = Vg.nv;
    const size_t nc = L.nc;
    int i = axis == 0 ? fi % (nx + 1) : fi % nx, j = axis == 0 ? fi / (nx + 1) : fi / nx;
    int outsign, c;
    bface_side(L, axis, i, j, c, outsign);
    const BcDev B = bc[bcid];
    const double* Cb = Cw + (size_t)bcid * nv;
    double s[2] = {0, 0};
    for (int k = threadIdx.x; k < nv; k += blockDim.x) {
        double uo = outsign * (axis == 0 ? Vg.u[k] : Vg.v[k]);
        if (uo > 0) s[0] += Vg.w[k] * uo * (double)f[(size_t)c * nv + k];
        else if (uo < 0) s[1] += Vg.w[k] * uo * Cb[k];
    }
    block_sum<2>(s, red);
    double rhow = -s[0] / s[1];
    double t[3] = {0, 0, 0};
    double Uwt = axis == 0 ? B.v : B.u;
    for (int k = threadIdx.x; k < nv; k += blockDim.x) {
        double u = Vg.u[k], v = Vg.v[k];
        double uo = outsign * (axis == 0 ? u : v), ut = axis == 0 ? v : u;
        double g, h;
        if (uo >= 0) { g = f[(size_t)c * nv + k]; h = f[(nc + c) * (size_t)nv + k]; }
        else { g = rhow * Cb[k]; h = g * kKint * B.t / 4.0; }
        double du = u - B.u, dv = v - B.v;
        t[0] += Vg.w[k] * uo * uo * g;
        t[1] += Vg.w[k] * uo * (ut - Uwt) * g;
        t[2] += Vg.w[k] * uo * (0.5 * (du * du + dv * dv) * g + h);
    }
    block_sum<3>(t, red);
    if (threadIdx.x == 0)
        for (int m = 0; m < 3; ++m) out[3 * blockIdx.x + m] = t[m];
}
template <typename F>
cudaError_t launch_wall_quantities(const LevelDev& L, const VelDev& V, const BcDev* bc, const double* Cw, const F* f,
                                   int bcid, const int* faces, int nfaces, double* out, cudaStream_t st)
{
    if (nfaces == 0) return cudaSuccess;
    k_wall_quantities<F><<<nfaces, 128, 0, st>>>(L, V, bc, Cw, f, bcid, faces, out);
    return cudaGetLastError();
}
template cudaError_t launch_wall_quantities<double>(const LevelDev&, const VelDev&, const BcDev*, const double*,
                                                    const double*, int, const int*, int, double*, cudaStream_t);
template cudaError_t launch_wall_quantities<float>(const LevelDev&, const VelDev&, const BcDev*, const double*,
                                                   const float*, int, const int*, int, double*, cudaStream_t);

} // namespace miugks
