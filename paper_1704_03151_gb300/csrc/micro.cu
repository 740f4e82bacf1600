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
// same holds for the last column and row in the backward sweep.  Each sweep is
// therefore two launches:
//   * k_sgs_chain: one thread-block cluster per boundary line walks the line
//     cell by cell; the velocities of a cell are spread over the CTAs of the
//     cluster and the wall sums are combined through distributed shared
//     memory with a hardware cluster barrier;
//   * k_sgs_interior: every CTA owns a contiguous chunk of discrete
//     velocities and sweeps the remaining cells diagonal by diagonal, with only
//     __syncthreads between diagonals (no grid-wide synchronisation).
#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace miugks {

constexpr int kChainCluster = 8;
constexpr int kChainThreads = 256;
constexpr int kChainKpt = 8;          // local velocities per thread in the chain kernel
constexpr int kInteriorKc = 4;        // velocities per CTA in the interior kernel

__device__ __forceinline__ double geomD(const LevelDev& L, int i, int j, double u, double v)
{
    return (fabs(u) * L.dy[j] + fabs(v) * L.dx[i]) / (L.dx[i] * L.dy[j]);
}

// coefficient of a neighbour (or ghost) through the face with outward normal outsign * e_axis
__device__ __forceinline__ double Dface(int axis, int outsign, double S, double V, double u, double v)
{
    double un = outsign * (axis == 0 ? u : v);
    return un < 0 ? un * S / V : 0.0;
}

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
    double* Eu = sm;
    double* Ev = sm + Vg.nu;
    double rho, U, V, lam;
    prim4(Wt + 4 * (size_t)c, rho, U, V, lam);
    const double itau = 1.0 / tau_of(gas, rho, lam);
    for (int a = threadIdx.x; a < Vg.nu; a += blockDim.x) { double d = Vg.ua[a] - U; Eu[a] = exp(-lam * d * d); }
    for (int b = threadIdx.x; b < Vg.nvv; b += blockDim.x) { double d = Vg.vb[b] - V; Ev[b] = exp(-lam * d * d); }
    if (threadIdx.x == 0) inv_tau[c] = itau + dtn_inv;
    __syncthreads();
    const double gnorm = rho * lam / kPi, hfac = kKint / (4.0 * lam);
    const double shk = (1.0 - gas.pr) * 4.0 * lam * lam / (5.0 * rho);
    const double qx = q[2 * (size_t)c], qy = q[2 * (size_t)c + 1];
    const double Vol = L.dx[i] * L.dy[j], dxi = L.dx[i], dyj = L.dy[j];
    const size_t nfx = L.nfx, nfy = L.nfy;
    const size_t fW = (size_t)j * (nx + 1) + i, fE = fW + 1, fS = (size_t)j * nx + i, fN = (size_t)(j + 1) * nx + i;
    for (int k = threadIdx.x; k < nv; k += blockDim.x) {
        int a = k / Vg.nvv, b = k - a * Vg.nvv;
        double u = Vg.u[k], v = Vg.v[k];
        double cx = u - U, cy = v - V, c2 = cx * cx + cy * cy;
        double gM = gnorm * Eu[a] * Ev[b], hM = gM * hfac;
        double Fq = shk * (cx * qx + cy * qy);
        double gt[2] = {gM * (1.0 + Fq * (2.0 * lam * c2 - 4.0)), hM * (1.0 + Fq * (2.0 * lam * c2 - 2.0))};
        #pragma unroll
        for (int cp = 0; cp < 2; ++cp) {
            const F* px = phx + cp * nfx * nv;
            const F* py = phy + cp * nfy * nv;
            double div = (dyj * ((double)px[fE * nv + k] - (double)px[fW * nv + k]) +
                          dxi * ((double)py[fN * nv + k] - (double)py[fS * nv + k])) / Vol;
            r[(cp * nc + c) * nv + k] = (F)((gt[cp] - (double)f[(cp * nc + c) * nv + k]) * itau - div);
        }
        invD[(size_t)c * nv + k] = (F)(1.0 / (itau + dtn_inv + geomD(L, i, j, u, v)));
    }
}

template <typename F>
cudaError_t launch_micro_residual(const MicroArgs& m, GasDev gas, const double* Wt, const double* q, const F* f,
                                  const F* phx, const F* phy, double dtn_inv, double* inv_tau, F* invD, F* r,
                                  cudaStream_t st)
{
    size_t smem = sizeof(double) * (m.V.nu + m.V.nvv);
    k_micro_residual<F><<<m.L.nc, m.V.nv >= 256 ? 256 : 128, smem, st>>>(m, gas, Wt, q, f, phx, phy, dtn_inv,
                                                                          inv_tau, invD, r);
    return cudaGetLastError();
}
template cudaError_t launch_micro_residual<double>(const MicroArgs&, GasDev, const double*, const double*,
                                                   const double*, const double*, const double*, double, double*,
                                                   double*, double*, cudaStream_t);

template <typename F>
__global__ void k_coarse_coeffs(MicroArgs M, GasDev gas, const double* __restrict__ Wt, double dtn_inv,
                                double* __restrict__ inv_tau, F* __restrict__ invD)
{
    const LevelDev& L = M.L;
    const int c = blockIdx.x, i = c % L.nx, j = c / L.nx;
    double rho, U, V, lam;
    prim4(Wt + 4 * (size_t)c, rho, U, V, lam);
    double it = 1.0 / tau_of(gas, rho, lam) + dtn_inv;
    if (threadIdx.x == 0) inv_tau[c] = it;
    for (int k = threadIdx.x; k < M.V.nv; k += blockDim.x)
        invD[(size_t)c * M.V.nv + k] = (F)(1.0 / (it + geomD(L, i, j, M.V.u[k], M.V.v[k])));
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

// ---------------------------------------------------------------------------
// boundary faces of a cell on one sweep side (0 lower = west/south, 1 upper = east/north)
struct BFace { int bc, axis, outsign; double S; };

__device__ __forceinline__ int side_faces(const LevelDev& L, int i, int j, int side, BFace* bf)
{
    int n = 0, nx = L.nx, ny = L.ny;
    if (side != 1 && i == 0) bf[n++] = {L.fbx[j * (nx + 1)], 0, -1, L.dy[j]};
    if (side != 1 && j == 0) bf[n++] = {L.fby[i], 1, -1, L.dx[i]};
    if (side != 0 && i == nx - 1) bf[n++] = {L.fbx[j * (nx + 1) + nx], 0, 1, L.dy[j]};
    if (side != 0 && j == ny - 1) bf[n++] = {L.fby[ny * nx + i], 1, 1, L.dx[i]};
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

// cluster-wide deterministic sum of NR values: block reduce, publish in own
// shared slot, cluster barrier, read every rank's slot in rank order.
template <int NR>
__device__ __forceinline__ void cluster_sum(cg::cluster_group& cl, double (&v)[NR], double* red, double* slots,
                                            int& ev)
{
    block_sum<NR>(v, red);
    double* my = slots + (ev & 1) * 8;
    if (threadIdx.x == 0)
        for (int q = 0; q < NR; ++q) my[q] = v[q];
    cl.sync();
    for (int q = 0; q < NR; ++q) v[q] = 0.0;
    for (int rk = 0; rk < kChainCluster; ++rk) {
        const double* other = cl.map_shared_rank(my, rk);
        for (int q = 0; q < NR; ++q) v[q] += other[q];
    }
    ++ev;
}

template <typename F>
__global__ void __cluster_dims__(kChainCluster, 1, 1) __launch_bounds__(kChainThreads)
k_sgs_chain(MicroArgs M, const double* __restrict__ Zw, const F* __restrict__ r, F* __restrict__ x,
            const F* __restrict__ xcorner, int pass)
{
    __shared__ double red[32 * 4];
    __shared__ double slots[16];
    extern __shared__ double xsm[];          // [2][nloc] current cell values of this CTA's velocities
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
    double xprev[kChainKpt][2];
    const int len = line == 0 ? ny : nx;
    for (int s = 0; s < len; ++s) {
        // cell of this step
        int i, j;
        if (pass == 0) { i = line == 0 ? 0 : s; j = line == 0 ? s : 0; }
        else { i = line == 0 ? nx - 1 : nx - 1 - s; j = line == 0 ? ny - 1 - s : ny - 1; }
        const int c = j * nx + i;
        const double Vol = L.dx[i] * L.dy[j], itau = M.inv_tau[c];
        // interior neighbour along the line (the previous cell), if any
        int nb_axis = line == 0 ? 1 : 0, nb_sign = pass == 0 ? -1 : 1;
        double nbS = nb_axis == 0 ? L.dy[j] : L.dx[i];
        BFace bf[2];
        int nb = side_faces(L, i, j, pass, bf);
        int nwall = 0, nsym = 0;
        for (int b = 0; b < nb; ++b) {
            int t = M.bc[bf[b].bc].type;
            nwall += t == BC_WALL;
            nsym += t == BC_SYMMETRY;
        }
        double base[kChainKpt][2], den[kChainKpt], xc[kChainKpt][2];
        #pragma unroll
        for (int t = 0; t < kChainKpt; ++t) {
            int k = kk[t];
            if (k < 0) continue;
            double u = Vg.u[k], v = Vg.v[k];
            double D = itau + geomD(L, i, j, u, v);
            double Dn = s > 0 ? Dface(nb_axis, nb_sign, nbS, Vol, u, v) : 0.0;
            den[t] = D;
            for (int b = 0; b < nb; ++b)
                if (M.bc[bf[b].bc].type == BC_OUTFLOW) den[t] += Dface(bf[b].axis, bf[b].outsign, bf[b].S, Vol, u, v);
            #pragma unroll
            for (int cp = 0; cp < 2; ++cp) {
                double y = s > 0 ? Dn * xprev[t][cp] : 0.0;
                size_t id = (cp * nc + c) * nv + k;
                // backward: the corner's forward value comes from a copy taken before the
                // launch, because the column line overwrites the corner while the row line reads it
                double xs = pass == 0 ? 0.0 : (s == 0 ? (double)xcorner[cp * nv + k] : (double)x[id]);
                base[t][cp] = pass == 0 ? (double)r[id] - y : D * xs - y;
                xc[t][cp] = base[t][cp] / den[t];
            }
        }
        if (nwall == 2 && nb == 2) {
            // two walls at a corner: 2x2 system for the two ghost densities
            double z[2], acc[4] = {0, 0, 0, 0};
            for (int b = 0; b < 2; ++b) z[b] = Zw[bf[b].bc * 4 + bf[b].axis * 2 + (bf[b].outsign > 0)];
            #pragma unroll
            for (int t = 0; t < kChainKpt; ++t) {
                int k = kk[t];
                if (k < 0) continue;
                double u = Vg.u[k], v = Vg.v[k], w = Vg.w[k];
                for (int b = 0; b < 2; ++b) {
                    double uo = bf[b].outsign * (bf[b].axis == 0 ? u : v);
                    if (!(uo > 0)) continue;
                    acc[b] += w * uo * base[t][0] / den[t];
                    int o = 1 - b;
                    double Do = Dface(bf[o].axis, bf[o].outsign, bf[o].S, Vol, u, v);
                    if (Do != 0.0) acc[2 + b] += w * uo * Do * M.Cw[(size_t)bf[o].bc * nv + k] / den[t];
                }
            }
            cluster_sum<4>(cl, acc, red, slots, ev);
            double cc0 = -acc[0] / z[0], cc1 = -acc[1] / z[1], mm0 = acc[2] / z[0], mm1 = acc[3] / z[1];
            double rho[2];
            rho[0] = (cc0 + mm0 * cc1) / (1.0 - mm0 * mm1);
            rho[1] = cc1 + mm1 * rho[0];
            #pragma unroll
            for (int t = 0; t < kChainKpt; ++t) {
                int k = kk[t];
                if (k < 0) continue;
                double u = Vg.u[k], v = Vg.v[k];
                for (int cp = 0; cp < 2; ++cp) {
                    double a = base[t][cp];
                    for (int b = 0; b < 2; ++b) {
                        double Db = Dface(bf[b].axis, bf[b].outsign, bf[b].S, Vol, u, v);
                        double C = M.Cw[(size_t)bf[b].bc * nv + k] * (cp == 0 ? 1.0 : kKint * M.bc[bf[b].bc].t / 4.0);
                        if (Db != 0.0) a -= Db * C * rho[b];
                    }
                    xc[t][cp] = a / den[t];
                }
            }
        } else if (nwall + nsym > 0) {
            // substitution rounds (exact for every other combination; one round without symmetry)
            int rounds = nsym > 0 ? 3 : 1;
            for (int rd = 0; rd < rounds; ++rd) {
                double rho = 0.0;
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
                    double acc[1] = {0.0};
                    #pragma unroll
                    for (int t = 0; t < kChainKpt; ++t) {
                        int k = kk[t];
                        if (k < 0) continue;
                        double uo = bf[wb].outsign * (bf[wb].axis == 0 ? Vg.u[k] : Vg.v[k]);
                        if (uo > 0) acc[0] += Vg.w[k] * uo * xc[t][0];
                    }
                    cluster_sum<1>(cl, acc, red, slots, ev);
                    rho = -acc[0] / Zw[bf[wb].bc * 4 + bf[wb].axis * 2 + (bf[wb].outsign > 0)];
                }
                double xn[kChainKpt][2];
                #pragma unroll
                for (int t = 0; t < kChainKpt; ++t) {
                    int k = kk[t];
                    if (k < 0) continue;
                    double u = Vg.u[k], v = Vg.v[k];
                    for (int cp = 0; cp < 2; ++cp) {
                        double a = base[t][cp];
                        for (int b = 0; b < nb; ++b) {
                            double Db = Dface(bf[b].axis, bf[b].outsign, bf[b].S, Vol, u, v);
                            if (Db == 0.0) continue;
                            int ty = M.bc[bf[b].bc].type;
                            if (ty == BC_WALL)
                                a -= Db * M.Cw[(size_t)bf[b].bc * nv + k] *
                                     (cp == 0 ? 1.0 : kKint * M.bc[bf[b].bc].t / 4.0) * rho;
                            else if (ty == BC_SYMMETRY)
                                a -= Db * xsm[cp * nloc + (bf[b].axis == 0 ? mu[t] : mvv[t])];
                        }
                        xn[t][cp] = a / den[t];
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
                x[c * (size_t)nv + k] = (F)xc[t][0];
                x[(nc + c) * (size_t)nv + k] = (F)xc[t][1];
            }
        }
    }
    cl.sync();   // keep every CTA's shared memory alive until all remote reads are done
}

template <typename F>
__global__ void __launch_bounds__(128) k_sgs_interior(MicroArgs M, const F* __restrict__ invD,
                                                      const F* __restrict__ r, F* __restrict__ x, int pass)
{
    const LevelDev& L = M.L;
    const VelDev& Vg = M.V;
    const int nx = L.nx, ny = L.ny, nv = Vg.nv;
    const size_t nc = L.nc;
    const int k0 = blockIdx.x * kInteriorKc;
    // interior region: forward i >= 1, j >= 1; backward i <= nx-2, j <= ny-2
    const int ilo0 = pass == 0 ? 1 : 0, ihi0 = pass == 0 ? nx - 1 : nx - 2;
    const int jlo0 = pass == 0 ? 1 : 0, jhi0 = pass == 0 ? ny - 1 : ny - 2;
    if (ihi0 < ilo0 || jhi0 < jlo0) return;
    const int dlo = ilo0 + jlo0, dhi = ihi0 + jhi0;
    for (int dd = 0; dd <= dhi - dlo; ++dd) {
        int d = pass == 0 ? dlo + dd : dhi - dd;
        int ilo = max(ilo0, d - jhi0), ihi = min(ihi0, d - jlo0);
        int nel = (ihi - ilo + 1) * kInteriorKc * 2;
        for (int e = threadIdx.x; e < nel; e += blockDim.x) {
            int slot = e / (2 * kInteriorKc), rem = e - slot * 2 * kInteriorKc;
            int cp = rem / kInteriorKc, k = k0 + rem - cp * kInteriorKc;
            if (k >= nv) continue;
            int i = ilo + slot, j = d - i;
            int c = j * nx + i;
            double u = Vg.u[k], v = Vg.v[k];
            double idx = 1.0 / L.dx[i], idy = 1.0 / L.dy[j];
            F* xb = x + cp * nc * nv;
            size_t id = (size_t)c * nv + k;
            if (pass == 0) {
                double dW = u > 0 ? -u * idx : 0.0, dS = v > 0 ? -v * idy : 0.0;
                double base = (double)r[cp * nc * nv + id] - dW * (double)xb[id - nv] - dS * (double)xb[id - (size_t)nx * nv];
                xb[id] = (F)(base * (double)invD[id]);
            } else {
                double dE = u < 0 ? u * idx : 0.0, dN = v < 0 ? v * idy : 0.0;
                double y = dE * (double)xb[id + nv] + dN * (double)xb[id + (size_t)nx * nv];
                xb[id] = (F)((double)xb[id] - y * (double)invD[id]);
            }
        }
        __syncthreads();
    }
}

template <typename F>
cudaError_t launch_micro_sgs(const MicroArgs& m, const double* Zw, const F* invD, const F* r, F* x, F* xcorner,
                             cudaStream_t st)
{
    const int ngroups = (m.V.nu + 1) / 2;
    const int nloc = ((ngroups + kChainCluster - 1) / kChainCluster) * 2 * m.V.nvv;
    if (nloc > kChainKpt * kChainThreads) return cudaErrorInvalidValue;
    size_t smem = sizeof(double) * 2 * nloc;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_sgs_chain<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    int nblk_int = (m.V.nv + kInteriorKc - 1) / kInteriorKc;
    const size_t nc = m.L.nc, nv = m.V.nv, corner = (size_t)m.L.nc - 1;
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1)
            for (int cp = 0; cp < 2; ++cp) {
                cudaError_t e = cudaMemcpyAsync(xcorner + cp * nv, x + (cp * nc + corner) * nv, nv * sizeof(F),
                                                cudaMemcpyDeviceToDevice, st);
                if (e != cudaSuccess) return e;
            }
        k_sgs_chain<F><<<2 * kChainCluster, kChainThreads, smem, st>>>(m, Zw, r, x, xcorner, pass);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_sgs_interior<F><<<nblk_int, 128, 0, st>>>(m, invD, r, x, pass);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}
template cudaError_t launch_micro_sgs<double>(const MicroArgs&, const double*, const double*, const double*, double*,
                                              double*, cudaStream_t);

// ---------------------------------------------------------------------------
// r -= A x (full operator with every neighbour and ghost), acc += x
template <typename F>
__global__ void __launch_bounds__(256) k_micro_renew(MicroArgs M, const double* __restrict__ Zw, const F* __restrict__ x,
                                                     F* __restrict__ r, F* __restrict__ acc, int renew)
{
    __shared__ double red[32 * 4];
    const LevelDev& L = M.L;
    const VelDev& Vg = M.V;
    const int c = blockIdx.x, nx = L.nx, ny = L.ny, nv = Vg.nv, i = c % nx, j = c / nx;
    const size_t nc = L.nc;
    if (acc)
        for (int e = threadIdx.x; e < 2 * nv; e += blockDim.x) {
            int cp = e / nv, k = e - cp * nv;
            size_t id = (cp * nc + c) * nv + k;
            acc[id] = (F)((double)acc[id] + (double)x[id]);
        }
    if (!renew) return;
    BFace bf[4];
    int nb = side_faces(L, i, j, 2, bf);
    double rho[4] = {0, 0, 0, 0};
    int nwall = 0;
    for (int b = 0; b < nb; ++b) nwall += M.bc[bf[b].bc].type == BC_WALL;
    if (nwall > 0) {
        double s[4] = {0, 0, 0, 0};
        for (int k = threadIdx.x; k < nv; k += blockDim.x)
            for (int b = 0; b < nb; ++b) {
                if (M.bc[bf[b].bc].type != BC_WALL) continue;
                double uo = bf[b].outsign * (bf[b].axis == 0 ? Vg.u[k] : Vg.v[k]);
                if (uo > 0) s[b] += Vg.w[k] * uo * (double)x[c * (size_t)nv + k];
            }
        block_sum<4>(s, red);
        for (int b = 0; b < nb; ++b)
            if (M.bc[bf[b].bc].type == BC_WALL) rho[b] = -s[b] / Zw[bf[b].bc * 4 + bf[b].axis * 2 + (bf[b].outsign > 0)];
    }
    const double Vol = L.dx[i] * L.dy[j], itau = M.inv_tau[c];
    for (int e = threadIdx.x; e < 2 * nv; e += blockDim.x) {
        int cp = e / nv, k = e - cp * nv;
        double u = Vg.u[k], v = Vg.v[k];
        const F* xb = x + cp * nc * nv;
        size_t id = (size_t)c * nv + k;
        double a = (itau + geomD(L, i, j, u, v)) * (double)xb[id];
        if (i > 0) a += Dface(0, -1, L.dy[j], Vol, u, v) * (double)xb[id - nv];
        if (i < nx - 1) a += Dface(0, 1, L.dy[j], Vol, u, v) * (double)xb[id + nv];
        if (j > 0) a += Dface(1, -1, L.dx[i], Vol, u, v) * (double)xb[id - (size_t)nx * nv];
        if (j < ny - 1) a += Dface(1, 1, L.dx[i], Vol, u, v) * (double)xb[id + (size_t)nx * nv];
        for (int b = 0; b < nb; ++b) {
            double Db = Dface(bf[b].axis, bf[b].outsign, bf[b].S, Vol, u, v);
            if (Db == 0.0) continue;
            int ty = M.bc[bf[b].bc].type;
            if (ty == BC_WALL)
                a += Db * M.Cw[(size_t)bf[b].bc * nv + k] * (cp == 0 ? 1.0 : kKint * M.bc[bf[b].bc].t / 4.0) * rho[b];
            else if (ty == BC_SYMMETRY) {
                int aa = k / Vg.nvv, bb = k - aa * Vg.nvv;
                int km = bf[b].axis == 0 ? (Vg.nu - 1 - aa) * Vg.nvv + bb : aa * Vg.nvv + (Vg.nvv - 1 - bb);
                a += Db * (double)xb[(size_t)c * nv + km];
            } else if (ty == BC_OUTFLOW) {
                a += Db * (double)xb[id];
            }
        }
        r[cp * nc * nv + id] = (F)((double)r[cp * nc * nv + id] - a);
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

// ---------------------------------------------------------------------------
// Steps 6-7: f += df (when df != null), then W = sum w psi f and q = sum w c (c^2 G/2 + H)
template <typename F>
__global__ void __launch_bounds__(256) k_update_moments(LevelDev L, VelDev Vg, F* __restrict__ f, const F* __restrict__ df,
                                                        double* __restrict__ W, double* __restrict__ q)
{
    __shared__ double red[32 * 4];
    const int c = blockIdx.x, nv = Vg.nv;
    const size_t nc = L.nc;
    F* fG = f + (size_t)c * nv;
    F* fH = f + (nc + c) * (size_t)nv;
    double s[4] = {0, 0, 0, 0};
    for (int k = threadIdx.x; k < nv; k += blockDim.x) {
        double g = fG[k], h = fH[k];
        if (df) {
            g = (double)(F)(g + (double)df[(size_t)c * nv + k]);
            h = (double)(F)(h + (double)df[(nc + c) * (size_t)nv + k]);
            fG[k] = (F)g; fH[k] = (F)h;
        }
        double u = Vg.u[k], v = Vg.v[k], w = Vg.w[k];
        s[0] += w * g; s[1] += w * u * g; s[2] += w * v * g; s[3] += w * (0.5 * (u * u + v * v) * g + h);
    }
    block_sum<4>(s, red);
    double rho, U, V, lam;
    prim4(s, rho, U, V, lam);
    double t[2] = {0, 0};
    for (int k = threadIdx.x; k < nv; k += blockDim.x) {
        double cx = Vg.u[k] - U, cy = Vg.v[k] - V;
        double e = 0.5 * (cx * cx + cy * cy) * (double)fG[k] + (double)fH[k];
        t[0] += Vg.w[k] * cx * e;
        t[1] += Vg.w[k] * cy * e;
    }
    block_sum<2>(t, red);
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

// discrete Maxwellian of (rho, U, V, T) per cell
template <typename F>
__global__ void k_init_maxwell(LevelDev L, VelDev Vg, const double* __restrict__ prim, F* __restrict__ f)
{
    const int c = blockIdx.x, nv = Vg.nv;
    const size_t nc = L.nc;
    double rho = prim[4 * c], U = prim[4 * c + 1], V = prim[4 * c + 2], lam = 1.0 / prim[4 * c + 3];
    for (int k = threadIdx.x; k < nv; k += blockDim.x) {
        double du = Vg.u[k] - U, dv = Vg.v[k] - V;
        double g = rho * (lam / kPi) * exp(-lam * (du * du + dv * dv));
        f[(size_t)c * nv + k] = (F)g;
        f[(nc + c) * (size_t)nv + k] = (F)(g * kKint / (4.0 * lam));
    }
}
template <typename F>
cudaError_t launch_init_maxwell(const LevelDev& L, const VelDev& V, const double* prim, F* f, cudaStream_t st)
{
    k_init_maxwell<F><<<L.nc, 128, 0, st>>>(L, V, prim, f);
    return cudaGetLastError();
}
template cudaError_t launch_init_maxwell<double>(const LevelDev&, const VelDev&, const double*, double*, cudaStream_t);

// wall pressure, shear and heat flux of the faces in `faces` (axis * 2^30 + face index)
template <typename F>
__global__ void k_wall_quantities(LevelDev L, VelDev Vg, const BcDev* __restrict__ bc, const double* __restrict__ Cw,
                                  const F* __restrict__ f, int bcid, const int* __restrict__ faces,
                                  double* __restrict__ out)
{
    __shared__ double red[32 * 4];
    const int code = faces[blockIdx.x];
    const int axis = code >> 30, fi = code & ((1 << 30) - 1);
    const int nx = L.nx, ny = L.ny, nv = Vg.nv;
    const size_t nc = L.nc;
    int i = axis == 0 ? fi % (nx + 1) : fi % nx, j = axis == 0 ? fi / (nx + 1) : fi / nx;
    int outsign = (axis == 0 ? i == 0 : j == 0) ? -1 : 1;
    int c = axis == 0 ? j * nx + (i == 0 ? 0 : nx - 1) : (j == 0 ? 0 : ny - 1) * nx + i;
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

} // namespace miugks
