// solver.cu -- host side of the MIUGKS library: the C ABI of include/miugks.h,
// the mesh hierarchy (Sec. 3.1), device memory, and the multigrid cycles of
// Sec. 2.4 (Eq. FASCYC for the prediction, Eq. CSCYC for the evolution)
// driving the kernels of flux.cu, macro.cu and micro.cu on one CUDA stream.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/miugks.h"
#include "kernels.cuh"

using namespace miugks;

namespace {

struct HLevel {
    int nx = 0, ny = 0, nc = 0, nfx = 0, nfy = 0;
    std::vector<double> xn, yn, xc, yc, dx, dy;
    std::vector<int> fbx, fby;
    std::vector<unsigned char> solid;   // 1 in a body
    int nfluid = 0;
    LevelDev dev{};
    SweepPlanDev plan{};                // sweep order tables (device)
    std::vector<SweepBreak> brk[2];     // body-line walks between wavefront segments
    int nlines = 0;                     // body lines (larger pass)
    // transposed sweep (adjoint preconditioner): the cells with one wall face of a body on
    // a pass's side, cell * 4 + face, grouped by wavefront step (AdjBodyPlan)
    int* adjb[2] = {nullptr, nullptr};
    std::vector<int> adjstep[2], adjoff[2];
    int* pidx = nullptr;      // prolongation stencil from the next coarser level
    double* pw = nullptr;
    int* sidx = nullptr;      // the same for a state (cells in bodies take their coarse cell's value)
    double* sw = nullptr;
    // prediction work, [nc][4]
    double *Wn = nullptr, *Wc = nullptr, *Rc = nullptr, *P = nullptr, *R = nullptr, *dW = nullptr, *gx = nullptr,
           *gy = nullptr, *Wt = nullptr, *idiag = nullptr, *T = nullptr;
    // evolution work, [2][nc][nv] (invD [nc][nv]); element type double, or float in the mixed form
    void *r = nullptr, *df = nullptr, *dl = nullptr, *invD = nullptr;
    // W and F cycles (second coarse visit of the CS cycle): the restricted residual and
    // the first visit's correction, allocated when such a cycle is selected
    void *r0 = nullptr, *acc = nullptr;
    double* inv_tau = nullptr;
};

} // namespace

struct miugks_solver {
    std::string err;
    miugks_opts opts{};
    cudaStream_t st = nullptr;
    std::vector<void*> allocs;
    int L = 1, nu = 0, nvv = 0, nv = 0, nbc = 0;
    double umax = 0, vmax = 0;
    GasDev gas{};
    std::vector<BcDev> bch;
    std::vector<double> uh, vh, wh, uah, vbh;
    std::vector<float> ufh, vfh, wfh;
    VelDev vel{};
    BcDev* bc = nullptr;
    double *Cw = nullptr, *Zw = nullptr;
    std::vector<double> Cwh;
    HLevel lev[kMaxLevels];
    // finest-level state (f, face fluxes and the corner scratch in the per-velocity type)
    bool mixed = false;
    size_t fsz = sizeof(double);
    void *f = nullptr, *phx = nullptr, *phy = nullptr, *xcorner = nullptr;
    double* fgeo[2] = {nullptr, nullptr};   // finest level: mesh constants of the interface flux per face
    double *W = nullptr, *q = nullptr, *R = nullptr, *Fx = nullptr, *Fy = nullptr;
    double *rms_part = nullptr, *rms_out = nullptr;
    double dtp_min = 0;
    int iter = 0;
    int cycle = 0;                              // 0 V, 1 W, 2 F, 3 adaptive (both multigrid cycles)
    // adaptive cycle: a second coarse visit when the first left more than adapt_ratio of the
    // coarse residual it started from; decisions kept in a ring (1 = second visit)
    double adapt_ratio = 0.2;
    long adapt_n = 0;
    std::vector<unsigned char> adapt_log = std::vector<unsigned char>(4096);
    double* nrm = nullptr;                      // device: 128 partial sums and the total
    int sweep_split = 0;                        // evolution sweep: 0 by size, 1 split by coupling class, 2 never
    bool shock = false;                         // pressure-jump collision time at interior faces
    unsigned long long wait_ns = 200000000ull;  // bound of the prediction sweep's device waits
    // timing mode: the finest level's wavefront and line-class sweep launches; totals since the last read
    SweepTimer sweep_timer;
    double t_sweepk[2] = {0, 0}, u_sweepk[2] = {0, 0};
    long n_sweepk[2] = {0, 0};
    bool initialised = false;
    bool timing = false;
    cudaEvent_t ev[6] = {};
    // one outer iteration captured as a CUDA graph (replayed while the launch
    // sequence and its arguments do not change)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool graph_ok = true;
    int eager_done = 0;
    double t_flux = 0, t_sweep = 0, t_total = 0;
    // per-launch events of the finest-level prediction sweep (timing mode only)
    std::vector<cudaEvent_t> ev_macro;
    int n_macro_used = 0;
    double t_macro = 0;
    long n_macro = 0;
    // adjoint work (FP64), allocated on first use
    struct {
        bool alloc = false;
        int m = 0;                          // Krylov basis vectors allocated
        double *f = nullptr, *W = nullptr, *q = nullptr, *itau = nullptr;
        double *recx = nullptr, *recy = nullptr, *crec = nullptr;
        double *b = nullptr, *x = nullptr, *w = nullptr, *z = nullptr, *t = nullptr, *Vb = nullptr;
        double *part = nullptr, *fpart = nullptr;
        int* faces = nullptr;
        // per level: state of the transposed CS cycle (checkpointed W and 1/tau,
        // work vectors, inverse prolongation stencil to the next coarser level)
        struct Lvl {
            double *W = nullptr, *itau = nullptr, *invD = nullptr, *T[6] = {}, *z = nullptr, *o = nullptr;
            int *pptr = nullptr, *pcell = nullptr;
            double* pw = nullptr;
        } lv[kMaxLevels];
        bool lv_alloc = false;
        // macroscopic correction of the preconditioner (transposed prediction step): Gamma at the
        // checkpoint, inverse transposed diagonal blocks of dR_E/dW, 4-vectors and the inner basis
        double *gx = nullptr, *gy = nullptr, *idiag = nullptr, *binv = nullptr;
        double *m4 = nullptr, *w4 = nullptr, *t4 = nullptr, *Vi = nullptr;
        double* Zb = nullptr;                 // flexible-GMRES preconditioned basis
        int mz = 0;
        bool macro = true;                    // apply the macroscopic correction
    } adj;
};

namespace {

miugks_status fail(miugks_solver* s, miugks_status code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (s) s->err = buf;
    return code;
}

#define CK(expr)                                                                                     \
    do {                                                                                             \
        cudaError_t e_ = (expr);                                                                     \
        if (e_ != cudaSuccess) return fail(s, MIUGKS_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)
#define ST(expr)                                  \
    do {                                          \
        miugks_status st_ = (expr);               \
        if (st_ != MIUGKS_OK) return st_;         \
    } while (0)

template <typename T>
miugks_status dalloc(miugks_solver* s, T** p, size_t count)
{
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    void* ptr = nullptr;
    if (s->opts.dev_alloc) {
        ptr = s->opts.dev_alloc(bytes, s->opts.alloc_ctx);
        if (!ptr) return fail(s, MIUGKS_ENOMEM, "device allocation of %zu bytes failed", bytes);
    } else {
        cudaError_t e = cudaMalloc(&ptr, bytes);
        if (e != cudaSuccess) return fail(s, MIUGKS_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    s->allocs.push_back(ptr);
    *p = (T*)ptr;
    return MIUGKS_OK;
}

// Mesh constants of every interior face of one axis of a level for the interface
// flux (layout kFluxGeo), with the arithmetic the flux would otherwise repeat
// per face and iteration: reconstruction distances, face-to-centre distances,
// the local time step dt = CFL min(w_L, w_R) / cmax and reciprocals.
std::vector<double> flux_face_geometry(const HLevel& L, int axis, double cfl, double cmax)
{
    const int nf = axis == 0 ? L.nfx : L.nfy;
    std::vector<double> t((size_t)nf * kFluxGeo, 0.0);
    const int n = axis == 0 ? L.nx : L.ny;                 // cells along the axis
    const std::vector<double>& c = axis == 0 ? L.xc : L.yc;
    const std::vector<double>& e = axis == 0 ? L.xn : L.yn;
    const std::vector<double>& w = axis == 0 ? L.dx : L.dy;
    for (int fi = 0; fi < nf; ++fi) {
        const int p = axis == 0 ? fi % (L.nx + 1) : fi / L.nx;   // face index along the axis
        if (p < 1 || p >= n) continue;
        double* g = &t[(size_t)fi * kFluxGeo];
        g[0] = p >= 2 ? 1.0 / (c[p - 1] - c[p - 2]) : 1.0;
        g[1] = 1.0 / (c[p] - c[p - 1]);
        g[2] = p + 1 < n ? 1.0 / (c[p + 1] - c[p]) : 1.0;
        g[3] = e[p] - c[p - 1];
        g[4] = c[p] - e[p];
        g[5] = cfl * std::fmin(w[p - 1], w[p]) / cmax;
        g[6] = 1.0 / g[5];
        g[7] = 1.0 / g[3];
        g[8] = 1.0 / g[4];
    }
    return t;
}

// per-velocity array of count elements of the solver's storage type
miugks_status falloc(miugks_solver* s, void** p, size_t count)
{
    if (s->mixed) return dalloc(s, (float**)p, count);
    return dalloc(s, (double**)p, count);
}

template <typename T>
miugks_status upload(miugks_solver* s, T** p, const std::vector<T>& h)
{
    ST(dalloc(s, p, h.size()));
    CK(cudaMemcpyAsync(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s->st));
    return MIUGKS_OK;
}

// discrete velocity nodes and weights of one axis (symmetric placement)
bool axis_grid(int n, double a, double b, int rule, std::vector<double>& x, std::vector<double>& w)
{
    if (n < 2 || !(b > a)) return false;
    x.resize(n);
    w.assign(n, 0.0);
    double h = (b - a) / (n - 1), c = 0.5 * (a + b);
    for (int i = 0; i < n; ++i) x[i] = c + (i - 0.5 * (n - 1)) * h;
    if (rule == 0) {
        for (int i = 0; i < n; ++i) w[i] = h;
        w[0] = w[n - 1] = 0.5 * h;
    } else if (rule == 1) {
        if ((n - 1) % 4) return false;
        static const double pan[5] = {7, 32, 12, 32, 7};
        for (int p = 0; p + 4 < n; p += 4)
            for (int q = 0; q < 5; ++q) w[p + q] += pan[q];
        for (int i = 0; i < n; ++i) w[i] *= 2.0 * h / 45.0;
    } else {
        return false;
    }
    return true;
}

double maxwell_unit(double U, double V, double T, double u, double v)
{
    double lam = 1.0 / T;
    return lam / kPi * std::exp(-lam * ((u - U) * (u - U) + (v - V) * (v - V)));
}

// unit-density Maxwellian of BC b at every discrete velocity (wall C_k, Eq. f_on_wall)
void refresh_bc_tables(miugks_solver* s, int b)
{
    const BcDev& B = s->bch[b];
    for (int k = 0; k < s->nv; ++k) s->Cwh[(size_t)b * s->nv + k] = maxwell_unit(B.u, B.v, B.t, s->uh[k], s->vh[k]);
}

// Z[b*4 + axis*2 + (outward normal positive)] = sum over incoming velocities of w u_n C_k,
// followed by the reciprocals (at offset 4 * kMaxBcs)
std::vector<double> wall_norms(miugks_solver* s)
{
    std::vector<double> Zh((size_t)kMaxBcs * 8, 0.0);
    for (int b = 0; b < s->nbc; ++b)
        for (int k = 0; k < s->nv; ++k) {
            double C = s->Cwh[(size_t)b * s->nv + k];
            for (int axis = 0; axis < 2; ++axis)
                for (int pos = 0; pos < 2; ++pos) {
                    double uo = (pos ? 1.0 : -1.0) * (axis == 0 ? s->uh[k] : s->vh[k]);
                    if (uo < 0) Zh[(size_t)b * 4 + axis * 2 + pos] += s->wh[k] * uo * C;
                }
        }
    for (int q = 0; q < 4 * s->nbc; ++q) Zh[4 * kMaxBcs + q] = Zh[q] != 0.0 ? 1.0 / Zh[q] : 0.0;
    return Zh;
}

void level_geometry(HLevel& Lv)
{
    Lv.xc.resize(Lv.nx); Lv.dx.resize(Lv.nx); Lv.yc.resize(Lv.ny); Lv.dy.resize(Lv.ny);
    for (int i = 0; i < Lv.nx; ++i) { Lv.dx[i] = Lv.xn[i + 1] - Lv.xn[i]; Lv.xc[i] = 0.5 * (Lv.xn[i] + Lv.xn[i + 1]); }
    for (int j = 0; j < Lv.ny; ++j) { Lv.dy[j] = Lv.yn[j + 1] - Lv.yn[j]; Lv.yc[j] = 0.5 * (Lv.yn[j] + Lv.yn[j + 1]); }
}

// Prolongation stencil of fine cell (i, j) inside coarse cell (I, J), as
// four coarse cells with weights (Eqs. prolongation, prolongationWeight; on a
// rectilinear mesh the products of 1-D linear weights).  Along each axis the
// second coarse cell is the neighbour on the side of the fine centre, else the
// one on the other side (signed weights: extrapolation), skipping cells
// outside the domain or in a body; with neither the axis is constant.  If the
// corner cell of the two chosen neighbours is in a body, the first
// combination of the axis options (own side first, x outer) whose three cells
// are fluid is used, else the y-axis is dropped.  Fine cells in a body get
// zero weights (a correction), or weight 1 on their own coarse cell with
// inject_solid (a state).
void prolong_stencil(const HLevel& F, const HLevel& C, int i, int j, int idx[4], double w[4], bool inject_solid = false)
{
    const int I = i / 2, J = j / 2;
    auto fluid = [&](int a, int b) { return a >= 0 && a < C.nx && b >= 0 && b < C.ny && !C.solid[b * C.nx + a]; };
    const int own = J * C.nx + I;
    if (F.solid[(size_t)j * F.nx + i]) {
        for (int q = 0; q < 4; ++q) { idx[q] = own; w[q] = 0.0; }
        if (inject_solid) w[0] = 1.0;
        return;
    }
    const double x = F.xc[i], y = F.yc[j];
    const int dx = x < C.xc[I] ? -1 : 1, dy = y < C.yc[J] ? -1 : 1;
    std::vector<int> ox, oy;
    for (int a : {I + dx, I - dx}) if (fluid(a, J)) ox.push_back(a);
    for (int b : {J + dy, J - dy}) if (fluid(I, b)) oy.push_back(b);
    int IN = ox.empty() ? I : ox[0], JN = oy.empty() ? J : oy[0];
    if (!ox.empty() && !oy.empty() && !fluid(IN, JN)) {
        bool found = false;
        for (size_t p = 0; p < ox.size() && !found; ++p)
            for (size_t q = 0; q < oy.size() && !found; ++q)
                if (fluid(ox[p], oy[q])) { IN = ox[p]; JN = oy[q]; found = true; }
        if (!found) JN = J;
    }
    double ax = 1.0, bx = 0.0, ay = 1.0, by = 0.0;
    if (IN != I) { double sp = C.xc[IN] - C.xc[I]; ax = (C.xc[IN] - x) / sp; bx = (x - C.xc[I]) / sp; }
    if (JN != J) { double sp = C.yc[JN] - C.yc[J]; ay = (C.yc[JN] - y) / sp; by = (y - C.yc[J]) / sp; }
    idx[0] = own;               w[0] = ax * ay;
    idx[1] = J * C.nx + IN;     w[1] = bx * ay;
    idx[2] = JN * C.nx + I;     w[2] = ax * by;
    idx[3] = JN * C.nx + IN;    w[3] = bx * by;
}

miugks_status upload_level(miugks_solver* s, HLevel& Lv)
{
    double *xn, *yn, *xc, *yc, *dx, *dy, *rdx, *rdy;
    int *fbx, *fby;
    unsigned char* solid;
    std::vector<double> rdxh(Lv.nx), rdyh(Lv.ny);
    for (int i = 0; i < Lv.nx; ++i) rdxh[i] = 1.0 / Lv.dx[i];
    for (int j = 0; j < Lv.ny; ++j) rdyh[j] = 1.0 / Lv.dy[j];
    ST(upload(s, &xn, Lv.xn)); ST(upload(s, &yn, Lv.yn)); ST(upload(s, &xc, Lv.xc)); ST(upload(s, &yc, Lv.yc));
    ST(upload(s, &dx, Lv.dx)); ST(upload(s, &dy, Lv.dy)); ST(upload(s, &fbx, Lv.fbx)); ST(upload(s, &fby, Lv.fby));
    ST(upload(s, &rdx, rdxh)); ST(upload(s, &rdy, rdyh)); ST(upload(s, &solid, Lv.solid));
    std::vector<int> ubc;   // fluid cells with an east or north boundary face
    for (int j = 0; j < Lv.ny; ++j)
        for (int i = 0; i < Lv.nx; ++i)
            if (!Lv.solid[j * Lv.nx + i] && (Lv.fbx[j * (Lv.nx + 1) + i + 1] >= 0 || Lv.fby[(j + 1) * Lv.nx + i] >= 0))
                ubc.push_back(j * Lv.nx + i);
    int* ubcd;
    ST(upload(s, &ubcd, ubc));
    Lv.dev = LevelDev{Lv.nx, Lv.ny, Lv.nc, Lv.nfx, Lv.nfy, xn, yn, xc, yc, dx, dy, fbx, fby, rdx, rdy, solid,
                      ubcd, (int)ubc.size()};
    size_t n4 = 4 * (size_t)Lv.nc, nf = 2 * (size_t)Lv.nc * s->nv;
    ST(dalloc(s, &Lv.Wn, n4)); ST(dalloc(s, &Lv.Wc, n4)); ST(dalloc(s, &Lv.Rc, n4)); ST(dalloc(s, &Lv.P, n4));
    ST(dalloc(s, &Lv.R, n4)); ST(dalloc(s, &Lv.dW, n4)); ST(dalloc(s, &Lv.Wt, n4));
    ST(dalloc(s, &Lv.gx, (size_t)Lv.nfx)); ST(dalloc(s, &Lv.gy, (size_t)Lv.nfy));
    ST(dalloc(s, &Lv.idiag, (size_t)Lv.nc)); ST(dalloc(s, &Lv.T, (macro_rec_bytes(Lv.nx, Lv.ny, s->mixed) + 7) / 8));
    ST(falloc(s, &Lv.r, nf)); ST(falloc(s, &Lv.df, nf)); ST(falloc(s, &Lv.dl, nf));
    ST(falloc(s, &Lv.invD, (size_t)Lv.nc * s->nv)); ST(dalloc(s, &Lv.inv_tau, (size_t)Lv.nc));
    return MIUGKS_OK;
}

MicroArgs micro_args(miugks_solver* s, int l)
{
    return MicroArgs{s->lev[l].dev, s->vel, s->bc, s->Cw, s->lev[l].inv_tau, s->lev[l].plan};
}

SweepPlanHost sweep_plan(const miugks_solver* s, const HLevel& Lv)
{
    SweepPlanHost h{};
    for (int p = 0; p < 2; ++p) { h.brk[p] = Lv.brk[p].data(); h.nbrk[p] = (int)Lv.brk[p].size(); }
    h.split = s->sweep_split;
    h.timer = s->timing && &Lv == &s->lev[0] ? const_cast<SweepTimer*>(&s->sweep_timer) : nullptr;
    return h;
}

// Sweep order of a level.  Per pass (0 forward: west / south faces on the
// sweep side; 1 backward: east / north), every fluid cell with a boundary
// face on the sweep side is a boundary-line cell: the domain edge's column and
// row (walked from the corner before the wavefront), and runs of cells along
// a body's faces, walked from the fluid cell before the run once the
// wavefront has passed that cell.  Every cell may have at most one such face
// (the two corners of the domain excepted), so the cells of the domain edge
// must be fluid and bodies keep one cell away from the edge.
miugks_status build_sweep_plan(miugks_solver* s, HLevel& Lv)
{
    const int nx = Lv.nx, ny = Lv.ny, nc = Lv.nc, nd = nx + ny - 1;
    auto bx = [&](int p, int i, int j) { return Lv.fbx[j * (nx + 1) + i + p] >= 0; };
    auto by = [&](int p, int i, int j) { return Lv.fby[(j + p) * nx + i] >= 0; };
    int nl_max = 0;
    for (int p = 0; p < 2; ++p) {
        std::vector<int> code(nc, -1);
        std::vector<int> lcell;              // int4 per entry
        for (int c = 0; c < nc; ++c) if (Lv.solid[c]) code[c] = -2;
        const int ie = p == 0 ? 0 : nx - 1, je = p == 0 ? 0 : ny - 1, sg = p == 0 ? 1 : -1;
        // the edge column (e = st) and row (e = ny + st), the corner first
        for (int st = 0; st < ny; ++st) {
            int i = ie, j = je + sg * st, c = j * nx + i;
            if (Lv.solid[c]) return fail(s, MIUGKS_EINVAL, "level with %dx%d cells: the cells on the domain edge must be fluid", nx, ny);
            lcell.insert(lcell.end(), {c, 0, st, st == 0});
            code[c] = (st << 2) | 2 | (st == 0 ? 1 : 0);
        }
        for (int st = 0; st < nx; ++st) {
            int i = ie + sg * st, j = je, c = j * nx + i;
            if (Lv.solid[c]) return fail(s, MIUGKS_EINVAL, "level with %dx%d cells: the cells on the domain edge must be fluid", nx, ny);
            lcell.insert(lcell.end(), {c, 1, kMaxLine + st, st == 0});
            if (st > 0) code[c] = ((ny + st) << 2) | 1;
        }
        Lv.plan.nl[p] = nx + ny;
        // every other fluid cell: at most one sweep-side boundary face
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int c = j * nx + i;
                if (Lv.solid[c] || code[c] != -1) continue;
                if (bx(p, i, j) && by(p, i, j))
                    return fail(s, MIUGKS_EINVAL, "cell (%d,%d) of a %dx%d level has two boundary faces on one sweep side "
                                  "(bodies must keep one cell away from the domain edge and from each other)", i, j, nx, ny);
            }
        // runs along bodies: x-face runs along columns, y-face runs along rows
        struct Run { int i0, j0, di, dj, len, axis, dd; };
        std::vector<Run> runs;
        for (int axis = 0; axis < 2; ++axis) {
            const int nout = axis == 0 ? nx : ny, nin = axis == 0 ? ny : nx;
            for (int a = 0; a < nout; ++a) {
                int b = 0;
                while (b < nin) {
                    auto member = [&](int t) {
                        int i = axis == 0 ? a : t, j = axis == 0 ? t : a, c = j * nx + i;
                        return !Lv.solid[c] && code[c] == -1 && (axis == 0 ? bx(p, i, j) : by(p, i, j));
                    };
                    if (!member(b)) { ++b; continue; }
                    int e = b;
                    while (e + 1 < nin && member(e + 1)) ++e;
                    // walk direction: +j / +i forward, -j / -i backward; cell 0 the fluid cell before the run
                    int first = p == 0 ? b : e, pre = first - sg;
                    int pi = axis == 0 ? a : pre, pj = axis == 0 ? pre : a;
                    if (pre < 0 || pre >= nin || Lv.solid[pj * nx + pi])
                        return fail(s, MIUGKS_EINVAL, "a body line of a %dx%d level has no fluid cell before it", nx, ny);
                    int dpre = pi + pj, ddpre = p == 0 ? dpre : nd - 1 - dpre;
                    runs.push_back({pi, pj, axis == 0 ? 0 : sg, axis == 0 ? sg : 0, e - b + 2, axis, ddpre + 1});
                    b = e + 1;
                }
            }
        }
        std::stable_sort(runs.begin(), runs.end(), [](const Run& x, const Run& y) { return x.dd < y.dd; });
        if ((int)runs.size() > kMaxBodyLines) return fail(s, MIUGKS_EINVAL, "too many body lines (%d > %d)", (int)runs.size(), kMaxBodyLines);
        std::vector<int> lines;
        Lv.brk[p].clear();
        for (int q = 0; q < (int)runs.size(); ++q) {
            const Run& R = runs[q];
            const int slot = (2 + q) * kMaxLine, e0 = (int)lcell.size() / 4;
            lines.insert(lines.end(), {R.i0, R.j0, R.di, R.dj, R.len, R.axis, slot, 0});
            for (int st = 1; st < R.len; ++st) {
                int i = R.i0 + st * R.di, j = R.j0 + st * R.dj, c = j * nx + i;
                code[c] = (((int)lcell.size() / 4) << 2) | (R.axis == 0 ? 2 : 1);
                lcell.insert(lcell.end(), {c, R.axis, slot + st, 0});
            }
            const int ne = (int)lcell.size() / 4 - e0;
            if (!Lv.brk[p].empty() && Lv.brk[p].back().dd == R.dd) {
                Lv.brk[p].back().nq++;
                Lv.brk[p].back().ne += ne;
            } else {
                Lv.brk[p].push_back(SweepBreak{R.dd, q, 1, e0, ne});
            }
        }
        Lv.nlines = std::max(Lv.nlines, (int)runs.size());
        nl_max = std::max(nl_max, (int)lcell.size() / 4);
        int* dcode;
        int4* dl;
        int* dlines = nullptr;
        ST(upload(s, &dcode, code));
        std::vector<int4> l4(lcell.size() / 4);
        for (size_t e = 0; e < l4.size(); ++e) l4[e] = make_int4(lcell[4 * e], lcell[4 * e + 1], lcell[4 * e + 2], lcell[4 * e + 3]);
        ST(upload(s, &dl, l4));
        if (!lines.empty()) ST(upload(s, &dlines, lines));
        Lv.plan.code[p] = dcode;
        Lv.plan.lcell[p] = dl;
        Lv.plan.lines[p] = dlines;
    }
    Lv.plan.nl_max = nl_max;
    Lv.plan.bodies = Lv.nfluid != Lv.nc;
    // The transposed sweep's wavefront covers pass 0 the cells i <= nx - 2, j <= ny - 2 in
    // steps t = i + j, pass 1 the cells i >= 1, j >= 1 in steps t = nd' - 1 - (i - 1 + j - 1),
    // nd' = nx + ny - 3.  A fluid cell there with exactly one wall face of a body on the
    // pass's side (pass 0 east or north, pass 1 west or south) gets its wall coupling after
    // its step; a cell with two such faces (a concave body corner) keeps the wavefront's
    // value (the Krylov solve corrects what the preconditioner leaves out).
    for (int p = 0; p < 2; ++p) {
        Lv.adjstep[p].clear();
        Lv.adjoff[p].assign(1, 0);
        if (nx < 2 || ny < 2 || Lv.nfluid == nc) continue;
        const int ndT = nx + ny - 3;
        std::vector<std::pair<int, int>> ent;   // (step, cell * 4 + face)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const int c = j * nx + i;
                if (Lv.solid[c]) continue;
                if (p == 0 ? (i > nx - 2 || j > ny - 2) : (i < 1 || j < 1)) continue;
                const int fx = Lv.fbx[j * (nx + 1) + i + (p == 0 ? 1 : 0)];
                const int fy = Lv.fby[(j + (p == 0 ? 1 : 0)) * nx + i];
                const bool wx = fx >= 0 && s->bch[fx].type == BC_WALL, wy = fy >= 0 && s->bch[fy].type == BC_WALL;
                if (wx == wy) continue;
                const int t = p == 0 ? i + j : ndT - 1 - (i - 1 + j - 1);
                ent.emplace_back(t, c * 4 + (wx ? (p == 0 ? 1 : 0) : (p == 0 ? 3 : 2)));
            }
        std::stable_sort(ent.begin(), ent.end(),
                         [](const std::pair<int, int>& a, const std::pair<int, int>& b) { return a.first < b.first; });
        std::vector<int> cells(ent.size());
        for (size_t e = 0; e < ent.size(); ++e) {
            cells[e] = ent[e].second;
            if (e == 0 || ent[e].first != ent[e - 1].first) {
                if (e > 0) Lv.adjoff[p].push_back((int)e);
                Lv.adjstep[p].push_back(ent[e].first);
            }
        }
        if (!ent.empty()) {
            Lv.adjoff[p].push_back((int)ent.size());
            ST(upload(s, &Lv.adjb[p], cells));
        }
    }
    return MIUGKS_OK;
}

MacroArgs macro_args(miugks_solver* s, int l, double dtn_inv)
{
    return MacroArgs{s->lev[l].dev, s->gas, s->bc, dtn_inv, s->rms_out + 5, s->wait_ns};
}

double dtn_inv(miugks_solver* s)
{
    if (!(s->opts.dtn_growth > 0.0)) return 0.0;
    return 1.0 / (std::pow(s->opts.dtn_growth, (double)s->iter) * s->dtp_min);
}

// ---------------------------------------------------------------- cycles
cudaError_t macro_sgs(miugks_solver* s, const MacroArgs& ma, HLevel& Lv)
{
    if (s->mixed) return launch_macro_sgs<float>(ma, Lv.Wc, Lv.gx, Lv.gy, Lv.idiag, Lv.T, Lv.R, Lv.dW, s->st);
    return launch_macro_sgs<double>(ma, Lv.Wc, Lv.gx, Lv.gy, Lv.idiag, Lv.T, Lv.R, Lv.dW, s->st);
}

// one prediction sweep; on the finest level, bracketed by events in timing mode
miugks_status timed_macro_sgs(miugks_solver* s, const MacroArgs& ma, HLevel& Lv, int l)
{
    if (!s->timing || l != 0) {
        CK(macro_sgs(s, ma, Lv));
        return MIUGKS_OK;
    }
    while ((int)s->ev_macro.size() < 2 * (s->n_macro_used + 1)) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        s->ev_macro.push_back(e);
    }
    CK(cudaEventRecord(s->ev_macro[2 * s->n_macro_used], s->st));
    CK(macro_sgs(s, ma, Lv));
    CK(cudaEventRecord(s->ev_macro[2 * s->n_macro_used + 1], s->st));
    s->n_macro_used++;
    return MIUGKS_OK;
}

// host value of the sum of squares of n device values (synchronises the stream)
template <typename T>
miugks_status sumsq(miugks_solver* s, const T* a, size_t n, double* h)
{
    CK(launch_sumsq<T>(a, n, s->nrm, s->nrm + 128, s->st));
    CK(cudaMemcpyAsync(h, s->nrm + 128, sizeof(double), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    return MIUGKS_OK;
}

// adaptive cycle: is another coarse visit due (and record the decision)
bool adapt_again(miugks_solver* s, double before, double after)
{
    const bool again = after > s->adapt_ratio * s->adapt_ratio * before;
    s->adapt_log[s->adapt_n++ % s->adapt_log.size()] = again ? 1 : 0;
    return again;
}
constexpr int kAdaptMaxVisits = 2;

// FAS cycle (Eq. FASCYC) of level l: forcing function and frozen Gamma from the
// level's W^n, then one visit.  A visit smooths, corrects from the next level
// (one coarse visit for V; W: two W visits; F: an F visit then a V visit, the
// second starting from the coarse state the first left, with the same forcing)
// and post-smooths.
miugks_status fas_visit(miugks_solver* s, int l, double dti, int type, bool first);

miugks_status fas(miugks_solver* s, int l, double dti, int type)
{
    HLevel& Lv = s->lev[l];
    MacroArgs ma = macro_args(s, l, dti);
    size_t n4 = 4 * (size_t)Lv.nc;
    CK(launch_macro_gamma(ma, Lv.Wn, Lv.gx, Lv.gy, Lv.idiag, s->st));
    CK(launch_macro_resid(ma, Lv.Wn, Lv.gx, Lv.gy, Lv.Rc, Lv.P, 0, s->st));     // forcing function
    CK(cudaMemcpyAsync(Lv.Wc, Lv.Wn, n4 * sizeof(double), cudaMemcpyDeviceToDevice, s->st));
    return fas_visit(s, l, dti, type, true);
}

miugks_status fas_visit(miugks_solver* s, int l, double dti, int type, bool first)
{
    HLevel& Lv = s->lev[l];
    MacroArgs ma = macro_args(s, l, dti);
    size_t n4 = 4 * (size_t)Lv.nc;
    if (first) CK(cudaMemcpyAsync(Lv.R, Lv.Rc, n4 * sizeof(double), cudaMemcpyDeviceToDevice, s->st));
    else CK(launch_macro_resid(ma, Lv.Wc, Lv.gx, Lv.gy, Lv.P, Lv.R, 1, s->st));   // P + R_E(W) of the state left
    const bool coarsest = l == s->L - 1;
    const int npre = coarsest ? (s->L == 1 ? 1 : s->opts.nu_coarse) : s->opts.nu1;
    for (int m = 0; m < npre; ++m) {
        ST(timed_macro_sgs(s, ma, Lv, l));
        if (coarsest && m == npre - 1) break;
        CK(launch_macro_resid(ma, Lv.Wc, Lv.gx, Lv.gy, Lv.P, Lv.R, 1, s->st));  // renewal P + R_E(W)
    }
    if (coarsest) return MIUGKS_OK;
    HLevel& Cv = s->lev[l + 1];
    CK(launch_restrict<double>(Lv.dev, Cv.dev, 4, 1, Lv.Wc, Cv.Wn, s->st));
    CK(launch_restrict<double>(Lv.dev, Cv.dev, 4, 1, Lv.R, Cv.Rc, s->st));
    ST(fas(s, l + 1, dti, type));
    if (type == 1 || type == 2) ST(fas_visit(s, l + 1, dti, type == 1 ? 1 : 0, false));
    if (type == 3) {
        // adaptive: the coarse residual on entry is the restricted R; after a visit, P + R_E(W)
        const size_t c4 = 4 * (size_t)Cv.nc;
        MacroArgs mc = macro_args(s, l + 1, dti);
        double before = 0.0, after = 0.0;
        ST(sumsq<double>(s, Cv.Rc, c4, &before));
        for (int visit = 1; visit < kAdaptMaxVisits; ++visit) {
            CK(launch_macro_resid(mc, Cv.Wc, Cv.gx, Cv.gy, Cv.P, Cv.R, 1, s->st));
            ST(sumsq<double>(s, Cv.R, c4, &after));
            if (!adapt_again(s, before, after)) break;
            before = after;
            ST(fas_visit(s, l + 1, dti, 3, false));
        }
    }
    CK(launch_sub(Cv.dW, Cv.Wc, Cv.Wn, 4 * (size_t)Cv.nc, s->st));
    CK(launch_prolong_state(Lv.dev, Lv.pidx, Lv.pw, Cv.dW, Lv.Wc, s->st));
    for (int m = 0; m < s->opts.nu2; ++m) {
        CK(launch_macro_resid(ma, Lv.Wc, Lv.gx, Lv.gy, Lv.P, Lv.R, 1, s->st));
        ST(timed_macro_sgs(s, ma, Lv, l));
    }
    return MIUGKS_OK;
}

// CS cycle (Eq. CSCYC) of level l.  W and F cycles visit the next level twice:
// the second visit solves for the coarse residual the first correction leaves,
// r_H - A_H df_H, and the corrections add.
template <typename F>
miugks_status cs(miugks_solver* s, int l, int type)
{
    HLevel& Lv = s->lev[l];
    MicroArgs mi = micro_args(s, l);
    size_t n = 2 * (size_t)Lv.nc * s->nv;
    F *r = (F*)Lv.r, *df = (F*)Lv.df, *dl = (F*)Lv.dl, *invD = (F*)Lv.invD, *xc = (F*)s->xcorner;
    CK(cudaMemsetAsync(df, 0, n * sizeof(F), s->st));
    const bool coarsest = l == s->L - 1;
    const int npre = coarsest ? (s->L == 1 ? 1 : s->opts.nu_coarse) : s->opts.nu1;
    for (int m = 0; m < npre; ++m) {
        CK(launch_micro_sgs<F>(mi, sweep_plan(s, Lv), s->Zw, invD, r, dl, xc, s->st));
        bool last = coarsest && m == npre - 1;
        CK(launch_micro_renew<F>(mi, s->Zw, dl, r, df, last ? 0 : 1, s->st));
        if (last) return MIUGKS_OK;
    }
    HLevel& Cv = s->lev[l + 1];
    const size_t nC = 2 * (size_t)Cv.nc * s->nv;
    CK(launch_restrict<F>(Lv.dev, Cv.dev, s->nv, 2, r, (F*)Cv.r, s->st));
    if (type != 0) CK(cudaMemcpyAsync(Cv.r0, Cv.r, nC * sizeof(F), cudaMemcpyDeviceToDevice, s->st));
    ST(cs<F>(s, l + 1, type));
    if (type == 3) {
        // adaptive: another visit for the coarse residual r_H - A_H df_H the corrections so
        // far leave, while a visit leaves more than the ratio of the residual it started from
        MicroArgs mc = micro_args(s, l + 1);
        double before = 0.0, after = 0.0;
        ST(sumsq<F>(s, (const F*)Cv.r0, nC, &before));
        CK(cudaMemcpyAsync(Cv.acc, Cv.df, nC * sizeof(F), cudaMemcpyDeviceToDevice, s->st));
        for (int visit = 1; visit < kAdaptMaxVisits; ++visit) {
            CK(cudaMemcpyAsync(Cv.r, Cv.r0, nC * sizeof(F), cudaMemcpyDeviceToDevice, s->st));
            CK(launch_micro_renew<F>(mc, s->Zw, (F*)Cv.acc, (F*)Cv.r, nullptr, 1, s->st));   // r_H - A_H acc
            ST(sumsq<F>(s, (const F*)Cv.r, nC, &after));
            if (!adapt_again(s, before, after)) break;
            before = after;
            ST(cs<F>(s, l + 1, 3));
            CK(launch_micro_renew<F>(mc, s->Zw, (F*)Cv.df, (F*)Cv.r, (F*)Cv.acc, 0, s->st));  // acc += df_H
        }
        CK(cudaMemcpyAsync(Cv.df, Cv.acc, nC * sizeof(F), cudaMemcpyDeviceToDevice, s->st));
    } else if (type != 0) {
        MicroArgs mc = micro_args(s, l + 1);
        CK(cudaMemcpyAsync(Cv.acc, Cv.df, nC * sizeof(F), cudaMemcpyDeviceToDevice, s->st));
        CK(cudaMemcpyAsync(Cv.r, Cv.r0, nC * sizeof(F), cudaMemcpyDeviceToDevice, s->st));
        CK(launch_micro_renew<F>(mc, s->Zw, (F*)Cv.acc, (F*)Cv.r, nullptr, 1, s->st));   // r_H - A_H df_H
        ST(cs<F>(s, l + 1, type == 1 ? 1 : 0));
        CK(launch_micro_renew<F>(mc, s->Zw, (F*)Cv.acc, (F*)Cv.r, (F*)Cv.df, 0, s->st)); // df_H += first correction
    }
    CK(launch_prolong_add<F>(Lv.dev, Cv.dev, s->nv, 2, Lv.pidx, Lv.pw, (F*)Cv.df, df, dl, s->st));
    for (int m = 0; m < s->opts.nu2; ++m) {
        CK(launch_micro_renew<F>(mi, s->Zw, dl, r, nullptr, 1, s->st));
        CK(launch_micro_sgs<F>(mi, sweep_plan(s, Lv), s->Zw, invD, r, dl, xc, s->st));
        CK(launch_micro_renew<F>(mi, s->Zw, dl, r, df, 0, s->st));
    }
    return MIUGKS_OK;
}

template <typename F>
miugks_status flux_stage_t(miugks_solver* s)
{
    HLevel& L0 = s->lev[0];
    FaceFluxArgs<F> fa{L0.dev, s->vel, s->gas, s->bc, s->Cw, (const F*)s->f, s->W, (F*)s->phx, s->Fx, 0, s->opts.cfl,
                       s->shock ? 1 : 0, s->fgeo[0]};
    CK(launch_face_flux<F>(fa, s->st));
    fa.axis = 1; fa.ph = (F*)s->phy; fa.Fm = s->Fy; fa.geo = s->fgeo[1];
    CK(launch_face_flux<F>(fa, s->st));
    CK(launch_cell_residual(L0.dev, s->Fx, s->Fy, s->R, s->st));
    return MIUGKS_OK;
}

miugks_status flux_stage(miugks_solver* s)
{
    return s->mixed ? flux_stage_t<float>(s) : flux_stage_t<double>(s);
}

template <typename F>
miugks_status one_iteration_t(miugks_solver* s)
{
    HLevel& L0 = s->lev[0];
    const double dti = dtn_inv(s);
    if (s->timing) CK(cudaEventRecord(s->ev[0], s->st));
    ST(flux_stage(s));                                                       // Step 1
    if (s->timing) CK(cudaEventRecord(s->ev[1], s->st));
    CK(launch_rms(s->R, s->W, L0.nc, L0.nfluid, s->rms_part, s->rms_out, s->st));
    size_t n4 = 4 * (size_t)L0.nc;
    CK(cudaMemcpyAsync(L0.Wn, s->W, n4 * sizeof(double), cudaMemcpyDeviceToDevice, s->st));
    CK(cudaMemcpyAsync(L0.Rc, s->R, n4 * sizeof(double), cudaMemcpyDeviceToDevice, s->st));
    ST(fas(s, 0, dti, s->cycle));                                            // Step 2
    CK(launch_predicted_state(L0.nc, L0.Wn, L0.Wc, L0.Wt, s->st));
    MicroArgs m0 = micro_args(s, 0);                                         // Steps 3-4
    CK(launch_micro_residual<F>(m0, s->gas, L0.Wt, s->q, (const F*)s->f, (const F*)s->phx, (const F*)s->phy, dti,
                                L0.inv_tau, (F*)L0.invD, (F*)L0.r, s->st));
    for (int l = 1; l < s->L; ++l) {
        CK(launch_restrict<double>(s->lev[l - 1].dev, s->lev[l].dev, 4, 1, s->lev[l - 1].Wt, s->lev[l].Wt, s->st));
        CK(launch_coarse_coeffs<F>(micro_args(s, l), s->gas, s->lev[l].Wt, dti, s->lev[l].inv_tau,
                                   (F*)s->lev[l].invD, s->st));
    }
    if (s->timing) CK(cudaEventRecord(s->ev[2], s->st));
    ST(cs<F>(s, 0, s->cycle));                                                  // Step 5
    if (s->timing) CK(cudaEventRecord(s->ev[3], s->st));
    CK(launch_update_moments<F>(L0.dev, s->vel, (F*)s->f, (const F*)L0.df, s->W, s->q, s->st));   // Steps 6-7
    if (s->timing) CK(cudaEventRecord(s->ev[4], s->st));
    return MIUGKS_OK;
}

miugks_status one_iteration(miugks_solver* s)
{
    return s->mixed ? one_iteration_t<float>(s) : one_iteration_t<double>(s);
}

miugks_status read_residual(miugks_solver* s, double res_out[4])
{
    double h[6];
    CK(cudaMemcpyAsync(h, s->rms_out, sizeof h, cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    if (res_out) memcpy(res_out, h, 4 * sizeof(double));
    if (h[5] != 0.0) return fail(s, MIUGKS_ETIMEOUT, "a bounded wait of the macro sweep gave up at iteration %d", s->iter);
    bool bad = h[4] > 0;
    for (int m = 0; m < 4; ++m) bad = bad || !std::isfinite(h[m]);
    if (bad) return fail(s, MIUGKS_EDIVERGED, "diverged at iteration %d (%.0f unphysical cells)", s->iter, h[4]);
    return MIUGKS_OK;
}

// copy n per-velocity values between a host double array and a device array of the storage type
miugks_status to_device(miugks_solver* s, void* dst, const double* src, size_t n)
{
    if (!s->mixed) {
        CK(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyHostToDevice, s->st));
        return cudaStreamSynchronize(s->st) == cudaSuccess ? MIUGKS_OK : fail(s, MIUGKS_ECUDA, "to_device");
    }
    std::vector<float> h(n);
    for (size_t q = 0; q < n; ++q) h[q] = (float)src[q];
    CK(cudaMemcpyAsync(dst, h.data(), n * sizeof(float), cudaMemcpyHostToDevice, s->st));
    CK(cudaStreamSynchronize(s->st));
    return MIUGKS_OK;
}

miugks_status to_host(miugks_solver* s, double* dst, const void* src, size_t n)
{
    if (!s->mixed) {
        CK(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToHost, s->st));
        CK(cudaStreamSynchronize(s->st));
        return MIUGKS_OK;
    }
    std::vector<float> h(n);
    CK(cudaMemcpyAsync(h.data(), src, n * sizeof(float), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    for (size_t q = 0; q < n; ++q) dst[q] = h[q];
    return MIUGKS_OK;
}

miugks_status moments_now(miugks_solver* s)
{
    if (s->mixed) CK(launch_moments<float>(s->lev[0].dev, s->vel, (const float*)s->f, s->W, s->q, s->st));
    else CK(launch_moments<double>(s->lev[0].dev, s->vel, (const double*)s->f, s->W, s->q, s->st));
    return MIUGKS_OK;
}

miugks_status check_level(miugks_solver* s, int lev)
{
    if (!s) return MIUGKS_EINVAL;
    if (lev < 0 || lev >= s->L) return fail(s, MIUGKS_EINVAL, "level %d out of range", lev);
    return MIUGKS_OK;
}

} // namespace

namespace {
template <typename F>
__global__ void k_invD_from_itau(LevelDev L, VelDev Vg, const double* it, F* invD)
{
    int c = blockIdx.x, i = c % L.nx, j = c / L.nx;
    for (int k = threadIdx.x; k < Vg.nv; k += blockDim.x) {
        double g = fabs(Vg.u[k]) * L.rdx[i] + fabs(Vg.v[k]) * L.rdy[j];
        invD[(size_t)c * Vg.nv + k] = (F)(1.0 / (it[c] + g));
    }
}
} // namespace

// =========================================================================== C ABI
extern "C" {

static thread_local std::string g_create_err;

// message for miugks_last_error(NULL) from entry points that have no solver
extern "C" void miugks_set_thread_error(const char* msg) { g_create_err = msg; }

const char* miugks_last_error(const miugks_solver* s) { return s ? s->err.c_str() : g_create_err.c_str(); }

void miugks_destroy(miugks_solver* s)
{
    if (!s) return;
    if (s->st) cudaStreamSynchronize(s->st);
    else cudaDeviceSynchronize();
    for (void* p : s->allocs) {
        if (s->opts.dev_free) s->opts.dev_free(p, s->opts.alloc_ctx);
        else cudaFree(p);
    }
    for (auto& e : s->ev)
        if (e) cudaEventDestroy(e);
    for (auto& e : s->ev_macro) cudaEventDestroy(e);
    if (s->gexec) cudaGraphExecDestroy(s->gexec);
    if (s->graph) cudaGraphDestroy(s->graph);
    delete s;
}

miugks_status miugks_create(const miugks_mesh* mesh, const miugks_vgrid* vg, const miugks_gas* gas,
                            const miugks_bc* bcs, int n_bcs, const miugks_opts* opts, miugks_solver** out)
{
    if (!out) return MIUGKS_EINVAL;
    *out = nullptr;
    if (!mesh || !vg || !gas || !bcs || !opts || n_bcs < 1) return MIUGKS_EINVAL;
    miugks_solver* s = new miugks_solver();
    s->opts = *opts;
    s->st = (cudaStream_t)opts->cuda_stream;
    auto bad = [&](const char* fmt, auto... a) {
        fail(s, MIUGKS_EINVAL, fmt, a...);
        return MIUGKS_EINVAL;
    };
    miugks_status st = MIUGKS_OK;
    do {
        if (opts->precision != MIUGKS_FP64 && opts->precision != MIUGKS_MIXED) {
            st = bad("unsupported precision %d", opts->precision);
            break;
        }
        s->mixed = opts->precision == MIUGKS_MIXED;
        s->fsz = s->mixed ? sizeof(float) : sizeof(double);
        if (opts->levels < 1 || opts->levels > kMaxLevels) { st = bad("levels must be 1..%d", kMaxLevels); break; }
        if (opts->nu1 < 1 || opts->nu2 < 1 || opts->nu_coarse < 1) { st = bad("smoothing counts must be >= 1"); break; }
        if (!(opts->cfl > 0.0)) { st = bad("cfl must be positive"); break; }
        if (mesh->nx < 1 || mesh->ny < 1) { st = bad("empty mesh"); break; }
        int div = 1 << (opts->levels - 1);
        if (mesh->nx % div || mesh->ny % div) { st = bad("nx, ny must be divisible by 2^(levels-1) = %d", div); break; }
        s->L = opts->levels;
        std::vector<double> ua, wa, vb, wb;
        if (!axis_grid(vg->nu, vg->umin, vg->umax, vg->rule, ua, wa) ||
            !axis_grid(vg->nv, vg->vmin, vg->vmax, vg->rule, vb, wb)) {
            st = bad("bad velocity grid (n >= 2, max > min, rule 0, or rule 1 with (n-1) %% 4 == 0)");
            break;
        }
        s->nu = vg->nu; s->nvv = vg->nv; s->nv = vg->nu * vg->nv;
        s->uah = ua; s->vbh = vb;
        s->uh.resize(s->nv); s->vh.resize(s->nv); s->wh.resize(s->nv);
        for (int a = 0; a < s->nu; ++a)
            for (int b = 0; b < s->nvv; ++b) {
                int k = a * s->nvv + b;
                s->uh[k] = ua[a]; s->vh[k] = vb[b]; s->wh[k] = wa[a] * wb[b];
            }
        s->umax = std::fmax(std::fabs(vg->umin), std::fabs(vg->umax));
        s->vmax = std::fmax(std::fabs(vg->vmin), std::fabs(vg->vmax));
        bool symgrid = vg->umin == -vg->umax && vg->vmin == -vg->vmax;
        if (!(gas->kn > 0) || !(gas->pr > 0)) { st = bad("Kn and Pr must be positive"); break; }
        s->gas = GasDev{15.0 * std::sqrt(kPi) * gas->kn / (2.0 * (5.0 - 2.0 * gas->omega) * (7.0 - 2.0 * gas->omega)),
                        gas->omega, gas->pr};
        if (n_bcs > kMaxBcs) { st = bad("at most %d boundary conditions", kMaxBcs); break; }
        s->nbc = n_bcs;
        s->bch.resize(n_bcs);
        for (int b = 0; b < n_bcs; ++b) {
            const miugks_bc& B = bcs[b];
            if (B.type < 0 || B.type > 3 || !(B.t > 0)) { st = bad("bad BC %d", b); break; }
            if (B.type == MIUGKS_BC_SYMMETRY && !symgrid) { st = bad("symmetry BC needs a velocity grid symmetric about 0"); break; }
            if (B.type == MIUGKS_BC_FARFIELD && !(B.rho > 0)) { st = bad("farfield BC %d needs rho > 0", b); break; }
            s->bch[b] = BcDev{B.type, B.rho, B.u, B.v, B.t};
        }
        if (st != MIUGKS_OK) break;
        // level 0
        HLevel& L0 = s->lev[0];
        L0.nx = mesh->nx; L0.ny = mesh->ny; L0.nc = L0.nx * L0.ny;
        L0.nfx = (L0.nx + 1) * L0.ny; L0.nfy = L0.nx * (L0.ny + 1);
        L0.xn.assign(mesh->x_nodes, mesh->x_nodes + L0.nx + 1);
        L0.yn.assign(mesh->y_nodes, mesh->y_nodes + L0.ny + 1);
        L0.fbx.assign(mesh->face_bc_x, mesh->face_bc_x + L0.nfx);
        L0.fby.assign(mesh->face_bc_y, mesh->face_bc_y + L0.nfy);
        for (int i = 0; i < L0.nx && st == MIUGKS_OK; ++i)
            if (!(L0.xn[i + 1] > L0.xn[i])) st = bad("x nodes must increase");
        for (int j = 0; j < L0.ny && st == MIUGKS_OK; ++j)
            if (!(L0.yn[j + 1] > L0.yn[j])) st = bad("y nodes must increase");
        L0.solid.assign(L0.nc, 0);
        if (mesh->solid)
            for (int c = 0; c < L0.nc; ++c) L0.solid[c] = mesh->solid[c] != 0;
        L0.nfluid = 0;
        for (int c = 0; c < L0.nc; ++c) L0.nfluid += !L0.solid[c];
        if (L0.nfluid == 0) { st = bad("no fluid cell"); break; }
        // a face joining two fluid cells is interior (-1); a face between a fluid
        // cell and a body or the domain edge needs a BC id; a face with no fluid
        // cell on either side is inactive (stored as -1)
        for (int j = 0; j < L0.ny && st == MIUGKS_OK; ++j)
            for (int i = 0; i <= L0.nx; ++i) {
                int& b = L0.fbx[j * (L0.nx + 1) + i];
                bool fl = i > 0 && !L0.solid[j * L0.nx + i - 1], fr = i < L0.nx && !L0.solid[j * L0.nx + i];
                if (!fl && !fr) { b = -1; continue; }
                if ((fl && fr) ? b != -1 : (b < 0 || b >= n_bcs)) { st = bad("x-face (%d,%d): boundary faces need a BC id, interior faces -1", i, j); break; }
            }
        for (int j = 0; j <= L0.ny && st == MIUGKS_OK; ++j)
            for (int i = 0; i < L0.nx; ++i) {
                int& b = L0.fby[j * L0.nx + i];
                bool fl = j > 0 && !L0.solid[(j - 1) * L0.nx + i], fr = j < L0.ny && !L0.solid[j * L0.nx + i];
                if (!fl && !fr) { b = -1; continue; }
                if ((fl && fr) ? b != -1 : (b < 0 || b >= n_bcs)) { st = bad("y-face (%d,%d): boundary faces need a BC id, interior faces -1", i, j); break; }
            }
        if (st != MIUGKS_OK) break;
        level_geometry(L0);
        for (int l = 1; l < s->L && st == MIUGKS_OK; ++l) {
            HLevel& F = s->lev[l - 1];
            HLevel& C = s->lev[l];
            C.nx = F.nx / 2; C.ny = F.ny / 2; C.nc = C.nx * C.ny;
            C.nfx = (C.nx + 1) * C.ny; C.nfy = C.nx * (C.ny + 1);
            for (int I = 0; I <= C.nx; ++I) C.xn.push_back(F.xn[2 * I]);
            for (int J = 0; J <= C.ny; ++J) C.yn.push_back(F.yn[2 * J]);
            C.fbx.resize(C.nfx); C.fby.resize(C.nfy);
            C.solid.assign(C.nc, 0);
            C.nfluid = 0;
            for (int J = 0; J < C.ny && st == MIUGKS_OK; ++J)
                for (int I = 0; I < C.nx; ++I) {
                    int ns = F.solid[(2 * J) * F.nx + 2 * I] + F.solid[(2 * J) * F.nx + 2 * I + 1] +
                             F.solid[(2 * J + 1) * F.nx + 2 * I] + F.solid[(2 * J + 1) * F.nx + 2 * I + 1];
                    if (ns != 0 && ns != 4) { st = bad("level %d: solid cells must fill whole coarse cells (%d,%d)", l, I, J); break; }
                    C.solid[J * C.nx + I] = ns == 4;
                    C.nfluid += ns == 0;
                }
            for (int J = 0; J < C.ny && st == MIUGKS_OK; ++J)
                for (int I = 0; I <= C.nx; ++I) {
                    int a = F.fbx[(2 * J) * (F.nx + 1) + 2 * I], b = F.fbx[(2 * J + 1) * (F.nx + 1) + 2 * I];
                    if (a != b) { st = bad("level %d x-face (%d,%d) spans two boundary ids", l, I, J); break; }
                    C.fbx[J * (C.nx + 1) + I] = a;
                }
            for (int J = 0; J <= C.ny && st == MIUGKS_OK; ++J)
                for (int I = 0; I < C.nx; ++I) {
                    int a = F.fby[(2 * J) * F.nx + 2 * I], b = F.fby[(2 * J) * F.nx + 2 * I + 1];
                    if (a != b) { st = bad("level %d y-face (%d,%d) spans two boundary ids", l, I, J); break; }
                    C.fby[J * C.nx + I] = a;
                }
            level_geometry(C);
        }
        if (st != MIUGKS_OK) break;
        if (mesh->nx > kMaxLine || mesh->ny > kMaxLine) { st = bad("nx and ny are limited to 512"); break; }
        // chain kernel capacity: velocities per CTA of the 8-CTA cluster
        int nloc = (((s->nu + 1) / 2 + 7) / 8) * 2 * s->nvv;
        if (nloc > 8 * 256) { st = bad("velocity grid too large for the boundary-line kernel (%d local > 2048)", nloc); break; }
        // device data (on the caller's stream, or the legacy default stream when none is given)
        upload_series_coefficients();
        if ((st = upload(s, (double**)&s->vel.u, s->uh)) != MIUGKS_OK) break;
        if ((st = upload(s, (double**)&s->vel.v, s->vh)) != MIUGKS_OK) break;
        if ((st = upload(s, (double**)&s->vel.w, s->wh)) != MIUGKS_OK) break;
        if ((st = upload(s, (double**)&s->vel.ua, s->uah)) != MIUGKS_OK) break;
        if ((st = upload(s, (double**)&s->vel.vb, s->vbh)) != MIUGKS_OK) break;
        s->ufh.assign(s->uh.begin(), s->uh.end());
        s->vfh.assign(s->vh.begin(), s->vh.end());
        s->wfh.assign(s->wh.begin(), s->wh.end());
        if ((st = upload(s, (float**)&s->vel.uf, s->ufh)) != MIUGKS_OK) break;
        if ((st = upload(s, (float**)&s->vel.vf, s->vfh)) != MIUGKS_OK) break;
        if ((st = upload(s, (float**)&s->vel.wf, s->wfh)) != MIUGKS_OK) break;
        s->vel.nu = s->nu; s->vel.nvv = s->nvv; s->vel.nv = s->nv; s->vel.umax = s->umax; s->vel.vmax = s->vmax;
        for (int p = 0; p < 2 && st == MIUGKS_OK; ++p) {
            std::vector<int> wb, lk;
            sweep_classes(s->uh.data(), s->vh.data(), s->nv, p, wb, lk, s->vel.nrow[p], s->vel.ncol[p], s->vel.nelem[p]);
            s->vel.nwblk[p] = (int)wb.size();
            if (wb.empty()) wb.push_back(0);        // keep a valid pointer
            if (lk.empty()) lk.push_back(0);
            if ((st = upload(s, (int**)&s->vel.wblk[p], wb)) != MIUGKS_OK) break;
            st = upload(s, (int**)&s->vel.lk[p], lk);
        }
        if (st != MIUGKS_OK) break;
        if ((st = upload(s, &s->bc, s->bch)) != MIUGKS_OK) break;
        s->Cwh.assign((size_t)n_bcs * s->nv, 0.0);
        for (int b = 0; b < n_bcs; ++b) refresh_bc_tables(s, b);
        if ((st = upload(s, &s->Cw, s->Cwh)) != MIUGKS_OK) break;
        if ((st = upload(s, &s->Zw, wall_norms(s))) != MIUGKS_OK) break;
        for (int l = 0; l < s->L && st == MIUGKS_OK; ++l) st = upload_level(s, s->lev[l]);
        if (st != MIUGKS_OK) break;
        for (int l = 0; l < s->L && st == MIUGKS_OK; ++l) st = build_sweep_plan(s, s->lev[l]);
        if (st != MIUGKS_OK) break;
        for (int l = 0; l + 1 < s->L && st == MIUGKS_OK; ++l) {
            HLevel& F = s->lev[l];
            HLevel& C = s->lev[l + 1];
            std::vector<int> idx(4 * (size_t)F.nc);
            std::vector<double> w(4 * (size_t)F.nc);
            std::vector<int> sidx(4 * (size_t)F.nc);
            std::vector<double> sw(4 * (size_t)F.nc);
            for (int j = 0; j < F.ny; ++j)
                for (int i = 0; i < F.nx; ++i) {
                    size_t c = (size_t)j * F.nx + i;
                    prolong_stencil(F, C, i, j, &idx[4 * c], &w[4 * c]);
                    prolong_stencil(F, C, i, j, &sidx[4 * c], &sw[4 * c], true);
                }
            if ((st = upload(s, &F.pidx, idx)) != MIUGKS_OK) break;
            if ((st = upload(s, &F.sidx, sidx)) != MIUGKS_OK) break;
            if ((st = upload(s, &F.sw, sw)) != MIUGKS_OK) break;
            st = upload(s, &F.pw, w);
        }
        if (st != MIUGKS_OK) break;
        size_t nc = L0.nc, nv = s->nv;
        if ((st = falloc(s, &s->f, 2 * nc * nv)) != MIUGKS_OK) break;
        if ((st = dalloc(s, &s->W, 4 * nc)) != MIUGKS_OK) break;
        if ((st = dalloc(s, &s->q, 2 * nc)) != MIUGKS_OK) break;
        if ((st = dalloc(s, &s->R, 4 * nc)) != MIUGKS_OK) break;
        if ((st = falloc(s, &s->phx, 2 * (size_t)L0.nfx * nv)) != MIUGKS_OK) break;
        if ((st = falloc(s, &s->phy, 2 * (size_t)L0.nfy * nv)) != MIUGKS_OK) break;
        if ((st = upload(s, &s->fgeo[0], flux_face_geometry(L0, 0, opts->cfl, s->umax))) != MIUGKS_OK) break;
        if ((st = upload(s, &s->fgeo[1], flux_face_geometry(L0, 1, opts->cfl, s->vmax))) != MIUGKS_OK) break;
        if ((st = dalloc(s, &s->Fx, 4 * (size_t)L0.nfx)) != MIUGKS_OK) break;
        if ((st = dalloc(s, &s->Fy, 4 * (size_t)L0.nfy)) != MIUGKS_OK) break;
        if ((st = dalloc(s, &s->rms_part, 64 * 5)) != MIUGKS_OK) break;
        if ((st = dalloc(s, &s->rms_out, 8)) != MIUGKS_OK) break;
        if ((st = dalloc(s, &s->nrm, 129)) != MIUGKS_OK) break;
        if (cudaMemset(s->rms_out, 0, 8 * sizeof(double)) != cudaSuccess) { st = fail(s, MIUGKS_ECUDA, "cudaMemset"); break; }
        {
            int nlines = 0, nlm = 0;
            for (int l = 0; l < s->L; ++l) {
                nlines = std::max(nlines, s->lev[l].nlines);
                nlm = std::max(nlm, s->lev[l].plan.nl_max);
            }
            if ((st = falloc(s, &s->xcorner, micro_scratch_elems(nv, nlm, nlines))) != MIUGKS_OK) break;
        }
        // smallest interior physical time step (for the numerical time step)
        s->dtp_min = 1e300;
        for (int i = 1; i < L0.nx; ++i) s->dtp_min = std::fmin(s->dtp_min, opts->cfl * std::fmin(L0.dx[i - 1], L0.dx[i]) / s->umax);
        for (int j = 1; j < L0.ny; ++j) s->dtp_min = std::fmin(s->dtp_min, opts->cfl * std::fmin(L0.dy[j - 1], L0.dy[j]) / s->vmax);
        for (auto& e : s->ev) {
            cudaError_t ce = cudaEventCreate(&e);
            if (ce != cudaSuccess) { st = fail(s, MIUGKS_ECUDA, "cudaEventCreate: %s", cudaGetErrorString(ce)); break; }
        }
        if (st != MIUGKS_OK) break;
        cudaError_t ce = cudaStreamSynchronize(s->st);
        if (ce != cudaSuccess) { st = fail(s, MIUGKS_ECUDA, "create: %s", cudaGetErrorString(ce)); break; }
    } while (0);
    if (st != MIUGKS_OK) {
        g_create_err = s->err;   // readable through miugks_last_error(NULL)
        miugks_destroy(s);
        return st;
    }
    *out = s;
    return MIUGKS_OK;
}

miugks_status miugks_init_fields(miugks_solver* s, const double* rho, const double* u, const double* v, const double* t)
{
    if (!s || !rho || !u || !v || !t) return MIUGKS_EINVAL;
    size_t nc = s->lev[0].nc;
    std::vector<double> prim(4 * nc);
    for (size_t c = 0; c < nc; ++c) {
        if (!(rho[c] > 0) || !(t[c] > 0)) return fail(s, MIUGKS_EINVAL, "initial rho and T must be positive");
        prim[4 * c] = rho[c]; prim[4 * c + 1] = u[c]; prim[4 * c + 2] = v[c]; prim[4 * c + 3] = t[c];
    }
    CK(cudaMemcpyAsync(s->lev[0].Wn, prim.data(), prim.size() * sizeof(double), cudaMemcpyHostToDevice, s->st));
    if (s->mixed) {
        CK(launch_init_maxwell<float>(s->lev[0].dev, s->vel, s->lev[0].Wn, (float*)s->f, s->st));
        CK(launch_moments<float>(s->lev[0].dev, s->vel, (const float*)s->f, s->W, s->q, s->st));
    } else {
        CK(launch_init_maxwell<double>(s->lev[0].dev, s->vel, s->lev[0].Wn, (double*)s->f, s->st));
        CK(launch_moments<double>(s->lev[0].dev, s->vel, (const double*)s->f, s->W, s->q, s->st));
    }
    CK(cudaStreamSynchronize(s->st));
    s->iter = 0;
    s->initialised = true;
    return MIUGKS_OK;
}

miugks_status miugks_init_uniform(miugks_solver* s, double rho, double u, double v, double t)
{
    if (!s) return MIUGKS_EINVAL;
    size_t nc = s->lev[0].nc;
    std::vector<double> a(nc, rho), b(nc, u), c(nc, v), d(nc, t);
    return miugks_init_fields(s, a.data(), b.data(), c.data(), d.data());
}

// Enqueue n outer iterations on the solver's stream without waiting.  After one
// eager iteration (which also performs the one-time kernel attribute set-up)
// an iteration is captured into a CUDA graph and replayed: one graph launch per
// iteration instead of a hundred kernel launches.  Stage timing, the numerical
// time step (whose value changes every iteration) and the legacy default
// stream (which cannot be captured) keep the eager path.
static miugks_status enqueue_iterations(miugks_solver* s, int n_iter)
{
    for (int it = 0; it < n_iter; ++it) {
        bool graphable = s->graph_ok && !s->timing && s->st != nullptr && !(s->opts.dtn_growth > 0.0) &&
                         s->eager_done > 0 && s->cycle != 3;
        if (graphable && !s->gexec) {
            cudaError_t e = cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal);
            miugks_status st = e == cudaSuccess ? one_iteration(s) : MIUGKS_ECUDA;
            cudaGraph_t g = nullptr;
            cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(s->st, &g) : e;
            if (st == MIUGKS_OK && e2 == cudaSuccess && g &&
                cudaGraphInstantiate(&s->gexec, g, 0) == cudaSuccess) {
                s->graph = g;
            } else {
                // capture unsupported here: run eagerly from now on
                if (g) cudaGraphDestroy(g);
                s->gexec = nullptr;
                s->graph_ok = false;
                cudaGetLastError();
                graphable = false;
            }
        }
        if (graphable) {
            CK(cudaGraphLaunch(s->gexec, s->st));
        } else {
            ST(one_iteration(s));
            s->eager_done++;
            if (s->timing) {
                CK(cudaEventSynchronize(s->ev[4]));
                float a = 0, b = 0, c = 0;
                CK(cudaEventElapsedTime(&a, s->ev[0], s->ev[1]));
                CK(cudaEventElapsedTime(&b, s->ev[2], s->ev[3]));
                CK(cudaEventElapsedTime(&c, s->ev[0], s->ev[4]));
                s->t_flux += a; s->t_sweep += b; s->t_total += c;
                for (int q = 0; q < s->n_macro_used; ++q) {
                    float t = 0;
                    CK(cudaEventElapsedTime(&t, s->ev_macro[2 * q], s->ev_macro[2 * q + 1]));
                    s->t_macro += t;
                }
                s->n_macro += s->n_macro_used;
                s->n_macro_used = 0;
                SweepTimer& T = s->sweep_timer;
                for (int q = 0; q < T.used; ++q) {
                    float t = 0;
                    CK(cudaEventElapsedTime(&t, T.ev[2 * q], T.ev[2 * q + 1]));
                    s->t_sweepk[T.kind[q]] += t;
                    s->u_sweepk[T.kind[q]] += T.units[q];
                    s->n_sweepk[T.kind[q]]++;
                }
                T.used = 0;
            }
        }
        s->iter++;
    }
    return MIUGKS_OK;
}

miugks_status miugks_step(miugks_solver* s, int n_iter, double res_out[4])
{
    if (!s) return MIUGKS_EINVAL;
    if (!s->initialised) return fail(s, MIUGKS_ESTATE, "step before init");
    if (n_iter < 0) return fail(s, MIUGKS_EINVAL, "n_iter < 0");
    ST(enqueue_iterations(s, n_iter));
    if (n_iter > 0) return read_residual(s, res_out);
    return MIUGKS_OK;
}

miugks_status miugks_step_async(miugks_solver* s, int n_iter)
{
    if (!s) return MIUGKS_EINVAL;
    if (!s->initialised) return fail(s, MIUGKS_ESTATE, "step before init");
    if (n_iter < 0) return fail(s, MIUGKS_EINVAL, "n_iter < 0");
    return enqueue_iterations(s, n_iter);
}

miugks_status miugks_wait(miugks_solver* s, double res_out[4])
{
    if (!s) return MIUGKS_EINVAL;
    return read_residual(s, res_out);
}

miugks_status miugks_run(miugks_solver* s, double tol, int max_iter, int* iters_out, double res_out[4])
{
    if (!s) return MIUGKS_EINVAL;
    double res[4] = {1e300, 1e300, 1e300, 1e300};
    int it = 0;
    miugks_status st = MIUGKS_OK;
    for (; it < max_iter; ++it) {
        st = miugks_step(s, 1, res);
        if (st != MIUGKS_OK) break;
        if (res[0] < tol && res[1] < tol && res[2] < tol && res[3] < tol) { ++it; break; }
    }
    if (iters_out) *iters_out = it;
    if (res_out) memcpy(res_out, res, sizeof res);
    if (st != MIUGKS_OK) return st;
    if (!(res[0] < tol && res[1] < tol && res[2] < tol && res[3] < tol))
        return fail(s, MIUGKS_ENOTCONVERGED, "not converged after %d iterations", it);
    return MIUGKS_OK;
}

miugks_status miugks_residual(miugks_solver* s, double res_out[4])
{
    if (!s) return MIUGKS_EINVAL;
    if (!s->initialised) return fail(s, MIUGKS_ESTATE, "residual before init");
    ST(flux_stage(s));
    CK(launch_rms(s->R, s->W, s->lev[0].nc, s->lev[0].nfluid, s->rms_part, s->rms_out, s->st));
    return read_residual(s, res_out);
}

int miugks_iterations(const miugks_solver* s) { return s ? s->iter : -1; }

miugks_status miugks_get_macro(miugks_solver* s, double* rho, double* u, double* v, double* t, double* qx, double* qy)
{
    if (!s) return MIUGKS_EINVAL;
    size_t nc = s->lev[0].nc;
    std::vector<double> W(4 * nc), q(2 * nc);
    CK(cudaMemcpyAsync(W.data(), s->W, W.size() * sizeof(double), cudaMemcpyDeviceToHost, s->st));
    CK(cudaMemcpyAsync(q.data(), s->q, q.size() * sizeof(double), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    for (size_t c = 0; c < nc; ++c) {
        double r = W[4 * c], U = W[4 * c + 1] / r, V = W[4 * c + 2] / r;
        double eint = W[4 * c + 3] - 0.5 * r * (U * U + V * V);
        double lam = (kKint + 2) * r / (4.0 * eint);
        if (rho) rho[c] = r;
        if (u) u[c] = U;
        if (v) v[c] = V;
        if (t) t[c] = 1.0 / lam;
        if (qx) qx[c] = q[2 * c];
        if (qy) qy[c] = q[2 * c + 1];
    }
    return MIUGKS_OK;
}

miugks_status miugks_get_f(miugks_solver* s, double* f)
{
    if (!s || !f) return MIUGKS_EINVAL;
    return to_host(s, f, s->f, 2 * (size_t)s->lev[0].nc * s->nv);
}

miugks_status miugks_set_f(miugks_solver* s, const double* f)
{
    if (!s || !f) return MIUGKS_EINVAL;
    ST(to_device(s, s->f, f, 2 * (size_t)s->lev[0].nc * s->nv));
    ST(moments_now(s));
    CK(cudaStreamSynchronize(s->st));
    s->initialised = true;
    return MIUGKS_OK;
}

miugks_status miugks_set_bc(miugks_solver* s, int bc, const miugks_bc* value)
{
    if (!s || !value) return MIUGKS_EINVAL;
    if (bc < 0 || bc >= s->nbc) return fail(s, MIUGKS_EINVAL, "BC id %d out of range", bc);
    if (value->type != s->bch[bc].type) return fail(s, MIUGKS_EINVAL, "BC type cannot change");
    if (!(value->t > 0)) return fail(s, MIUGKS_EINVAL, "BC temperature must be positive");
    s->bch[bc] = BcDev{value->type, value->rho, value->u, value->v, value->t};
    refresh_bc_tables(s, bc);
    std::vector<double> Zh = wall_norms(s);
    CK(cudaMemcpyAsync(s->bc + bc, &s->bch[bc], sizeof(BcDev), cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(s->Cw + (size_t)bc * s->nv, s->Cwh.data() + (size_t)bc * s->nv, s->nv * sizeof(double),
                       cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(s->Zw, Zh.data(), Zh.size() * sizeof(double), cudaMemcpyHostToDevice, s->st));
    CK(cudaStreamSynchronize(s->st));
    return MIUGKS_OK;
}

miugks_status miugks_init_from_coarse(miugks_solver* s, const miugks_solver* c)
{
    if (!s || !c) return MIUGKS_EINVAL;
    if (s->L < 2) return fail(s, MIUGKS_EINVAL, "init_from_coarse: the fine solver needs at least two levels");
    const HLevel& F1 = s->lev[1];
    const HLevel& C0 = c->lev[0];
    if (c->nv != s->nv || c->nu != s->nu || C0.nx != F1.nx || C0.ny != F1.ny)
        return fail(s, MIUGKS_EINVAL, "init_from_coarse: the coarse solver is not on the next coarser mesh");
    if (c->mixed != s->mixed) return fail(s, MIUGKS_EINVAL, "init_from_coarse: the two solvers differ in precision");
    if (C0.solid != F1.solid) return fail(s, MIUGKS_EINVAL, "init_from_coarse: the bodies differ");
    if (!c->initialised) return fail(s, MIUGKS_ESTATE, "init_from_coarse: the coarse solver has no state");
    for (int i = 0; i <= F1.nx; ++i)
        if (std::fabs(C0.xn[i] - F1.xn[i]) > 1e-12 * (1.0 + std::fabs(F1.xn[i])))
            return fail(s, MIUGKS_EINVAL, "init_from_coarse: x nodes differ");
    for (int j = 0; j <= F1.ny; ++j)
        if (std::fabs(C0.yn[j] - F1.yn[j]) > 1e-12 * (1.0 + std::fabs(F1.yn[j])))
            return fail(s, MIUGKS_EINVAL, "init_from_coarse: y nodes differ");
    HLevel& L0 = s->lev[0];
    const size_t n = 2 * (size_t)L0.nc * s->nv;
    CK(cudaStreamSynchronize(c->st));                      // the coarse state is complete
    CK(cudaMemsetAsync(s->f, 0, n * s->fsz, s->st));
    if (s->mixed)
        CK(launch_prolong_add<float>(L0.dev, F1.dev, s->nv, 2, L0.sidx, L0.sw, (const float*)c->f, (float*)s->f,
                                     (float*)nullptr, s->st));
    else
        CK(launch_prolong_add<double>(L0.dev, F1.dev, s->nv, 2, L0.sidx, L0.sw, (const double*)c->f, (double*)s->f,
                                      (double*)nullptr, s->st));
    // cells whose prolonged state is unphysical take their coarse cell's f
    if (s->mixed)
        CK(launch_state_fallback<float>(L0.dev, s->vel, C0.nx, (size_t)C0.nc, (const float*)c->f, (float*)s->f,
                                        s->st));
    else
        CK(launch_state_fallback<double>(L0.dev, s->vel, C0.nx, (size_t)C0.nc, (const double*)c->f, (double*)s->f,
                                         s->st));
    ST(moments_now(s));
    CK(cudaStreamSynchronize(s->st));
    s->initialised = true;
    s->iter = 0;
    return MIUGKS_OK;
}

miugks_status miugks_copy_state(miugks_solver* s, const miugks_solver* src)
{
    if (!s || !src) return MIUGKS_EINVAL;
    const HLevel& A = s->lev[0];
    const HLevel& B = src->lev[0];
    if (src->nv != s->nv || src->nu != s->nu || A.nx != B.nx || A.ny != B.ny || A.solid != B.solid)
        return fail(s, MIUGKS_EINVAL, "copy_state: the solvers differ in mesh, bodies or velocity grid");
    for (int i = 0; i <= A.nx; ++i)
        if (A.xn[i] != B.xn[i]) return fail(s, MIUGKS_EINVAL, "copy_state: x nodes differ");
    for (int j = 0; j <= A.ny; ++j)
        if (A.yn[j] != B.yn[j]) return fail(s, MIUGKS_EINVAL, "copy_state: y nodes differ");
    for (int k = 0; k < s->nv; ++k)
        if (s->uh[k] != src->uh[k] || s->vh[k] != src->vh[k] || s->wh[k] != src->wh[k])
            return fail(s, MIUGKS_EINVAL, "copy_state: velocity grids differ");
    if (!src->initialised) return fail(s, MIUGKS_ESTATE, "copy_state: the source solver has no state");
    const size_t n = 2 * (size_t)A.nc * s->nv;
    CK(cudaStreamSynchronize(src->st));                    // the source state is complete
    if (s->mixed == src->mixed) CK(cudaMemcpyAsync(s->f, src->f, n * s->fsz, cudaMemcpyDeviceToDevice, s->st));
    else if (!s->mixed) CK(launch_to_double<float>((const float*)src->f, (double*)s->f, n, s->st));
    else CK(launch_to_float((const double*)src->f, (float*)s->f, n, s->st));
    ST(moments_now(s));
    CK(cudaStreamSynchronize(s->st));
    s->initialised = true;
    s->iter = src->iter;
    return MIUGKS_OK;
}

miugks_status miugks_set_cycle(miugks_solver* s, int type)
{
    if (!s) return MIUGKS_EINVAL;
    if (type < 0 || type > 3) return fail(s, MIUGKS_EINVAL, "cycle type %d: 0 V, 1 W, 2 F, 3 adaptive", type);
    if (type != 0)
        for (int l = 1; l < s->L; ++l) {
            HLevel& Cv = s->lev[l];
            const size_t n = 2 * (size_t)Cv.nc * s->nv;
            if (!Cv.r0) ST(falloc(s, &Cv.r0, n));
            if (!Cv.acc) ST(falloc(s, &Cv.acc, n));
        }
    if (type != s->cycle && s->gexec) {
        // the captured iteration holds the old launch sequence
        CK(cudaStreamSynchronize(s->st));
        cudaGraphExecDestroy(s->gexec);
        if (s->graph) cudaGraphDestroy(s->graph);
        s->gexec = nullptr;
        s->graph = nullptr;
    }
    s->cycle = type;
    return MIUGKS_OK;
}

miugks_status miugks_set_sweep_split(miugks_solver* s, int mode)
{
    if (!s) return MIUGKS_EINVAL;
    if (mode < 0 || mode > 2) return fail(s, MIUGKS_EINVAL, "sweep split mode %d: 0 by size, 1 always, 2 never", mode);
    if (mode != s->sweep_split && s->gexec) {
        // the captured iteration holds the old launch sequence
        CK(cudaStreamSynchronize(s->st));
        cudaGraphExecDestroy(s->gexec);
        if (s->graph) cudaGraphDestroy(s->graph);
        s->gexec = nullptr;
        s->graph = nullptr;
    }
    s->sweep_split = mode;
    return MIUGKS_OK;
}

miugks_status miugks_set_wait_limit(miugks_solver* s, double seconds)
{
    if (!s) return MIUGKS_EINVAL;
    if (!(seconds >= 0.0 && seconds <= 10.0)) return fail(s, MIUGKS_EINVAL, "wait limit %g s: 0 to 10", seconds);
    s->wait_ns = (unsigned long long)(seconds * 1e9);   // a kernel argument: a captured iteration is re-captured
    if (s->gexec) {
        CK(cudaStreamSynchronize(s->st));
        cudaGraphExecDestroy(s->gexec);
        if (s->graph) cudaGraphDestroy(s->graph);
        s->gexec = nullptr;
        s->graph = nullptr;
    }
    return MIUGKS_OK;
}

miugks_status miugks_set_shock_capturing(miugks_solver* s, int on)
{
    if (!s) return MIUGKS_EINVAL;
    s->shock = on != 0;            // a kernel argument: a captured iteration is re-captured
    if (s->gexec) {
        CK(cudaStreamSynchronize(s->st));
        cudaGraphExecDestroy(s->gexec);
        if (s->graph) cudaGraphDestroy(s->graph);
        s->gexec = nullptr;
        s->graph = nullptr;
    }
    return MIUGKS_OK;
}

miugks_status miugks_set_adaptive_ratio(miugks_solver* s, double ratio)
{
    if (!s) return MIUGKS_EINVAL;
    if (!(ratio >= 0.0)) return fail(s, MIUGKS_EINVAL, "adaptive ratio %g must be >= 0", ratio);
    s->adapt_ratio = ratio;
    return MIUGKS_OK;
}

int miugks_adaptive_decisions(const miugks_solver* s, unsigned char* out, int cap)
{
    if (!s) return -1;
    const long n = s->adapt_n, ring = (long)s->adapt_log.size();
    long m = n < cap ? n : cap;
    if (m > ring) m = ring;
    for (long q = 0; q < m && out; ++q) out[q] = s->adapt_log[(n - m + q) % ring];
    return (int)n;
}

miugks_status miugks_get_wall(miugks_solver* s, int bc, int* n_faces, double* p, double* tau, double* q)
{
    if (!s || !n_faces) return MIUGKS_EINVAL;
    if (bc < 0 || bc >= s->nbc) return fail(s, MIUGKS_EINVAL, "BC id %d out of range", bc);
    if (s->bch[bc].type != MIUGKS_BC_WALL) return fail(s, MIUGKS_EINVAL, "BC %d is not a wall", bc);
    HLevel& L0 = s->lev[0];
    std::vector<int> faces;
    for (int fi = 0; fi < L0.nfx; ++fi) if (L0.fbx[fi] == bc) faces.push_back(fi);
    for (int fi = 0; fi < L0.nfy; ++fi) if (L0.fby[fi] == bc) faces.push_back((1 << 30) | fi);
    int cap = *n_faces, n = (int)faces.size();
    *n_faces = n;
    if (cap == 0) return MIUGKS_OK;
    if (cap < n) return fail(s, MIUGKS_EINVAL, "capacity %d < %d faces", cap, n);
    int* dfaces;
    double* dout;
    cudaError_t e = cudaMalloc(&dfaces, n * sizeof(int));
    if (e != cudaSuccess) return fail(s, MIUGKS_ENOMEM, "cudaMalloc: %s", cudaGetErrorString(e));
    e = cudaMalloc(&dout, 3 * n * sizeof(double));
    if (e != cudaSuccess) { cudaFree(dfaces); return fail(s, MIUGKS_ENOMEM, "cudaMalloc: %s", cudaGetErrorString(e)); }
    std::vector<double> h(3 * (size_t)n);
    e = cudaMemcpyAsync(dfaces, faces.data(), n * sizeof(int), cudaMemcpyHostToDevice, s->st);
    if (e == cudaSuccess)
        e = s->mixed ? launch_wall_quantities<float>(L0.dev, s->vel, s->bc, s->Cw, (const float*)s->f, bc, dfaces, n,
                                                      dout, s->st)
                     : launch_wall_quantities<double>(L0.dev, s->vel, s->bc, s->Cw, (const double*)s->f, bc, dfaces, n,
                                                       dout, s->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), dout, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    cudaFree(dfaces);
    cudaFree(dout);
    if (e != cudaSuccess) return fail(s, MIUGKS_ECUDA, "get_wall: %s", cudaGetErrorString(e));
    for (int m = 0; m < n; ++m) {
        if (p) p[m] = h[3 * m];
        if (tau) tau[m] = h[3 * m + 1];
        if (q) q[m] = h[3 * m + 2];
    }
    return MIUGKS_OK;
}

miugks_status miugks_sizes(const miugks_solver* s, int* nx, int* ny, int* nv, int* levels)
{
    if (!s) return MIUGKS_EINVAL;
    if (nx) *nx = s->lev[0].nx;
    if (ny) *ny = s->lev[0].ny;
    if (nv) *nv = s->nv;
    if (levels) *levels = s->L;
    return MIUGKS_OK;
}

miugks_status miugks_set_timing(miugks_solver* s, int on)
{
    if (!s) return MIUGKS_EINVAL;
    s->timing = on != 0;
    s->t_flux = s->t_sweep = s->t_total = 0;
    return MIUGKS_OK;
}

miugks_status miugks_macro_sweep_times(miugks_solver* s, double* ms, int* launches)
{
    if (!s) return MIUGKS_EINVAL;
    if (ms) *ms = s->timing ? s->t_macro : -1.0;
    if (launches) *launches = s->timing ? (int)s->n_macro : 0;
    s->t_macro = 0;
    s->n_macro = 0;
    return MIUGKS_OK;
}

miugks_status miugks_sweep_kernel_times(miugks_solver* s, double out[6])
{
    if (!s || !out) return MIUGKS_EINVAL;
    for (int k = 0; k < 2; ++k) {
        out[3 * k] = s->timing ? s->t_sweepk[k] : -1.0;
        out[3 * k + 1] = s->timing ? (double)s->n_sweepk[k] : 0.0;
        out[3 * k + 2] = s->timing ? s->u_sweepk[k] : 0.0;
        s->t_sweepk[k] = s->u_sweepk[k] = 0.0;
        s->n_sweepk[k] = 0;
    }
    return MIUGKS_OK;
}

miugks_status miugks_kernel_times(miugks_solver* s, double* flux_ms, double* sweep_ms, double* total_ms)
{
    if (!s) return MIUGKS_EINVAL;
    if (flux_ms) *flux_ms = s->timing ? s->t_flux : -1.0;
    if (sweep_ms) *sweep_ms = s->timing ? s->t_sweep : -1.0;
    if (total_ms) *total_ms = s->timing ? s->t_total : -1.0;
    s->t_flux = s->t_sweep = s->t_total = 0;
    return MIUGKS_OK;
}

// ---------------------------------------------------------------- stages
miugks_status miugks_stage_flux(miugks_solver* s, double* R, double* phx, double* phy)
{
    if (!s) return MIUGKS_EINVAL;
    if (!s->initialised) return fail(s, MIUGKS_ESTATE, "stage before init");
    ST(flux_stage(s));
    HLevel& L0 = s->lev[0];
    if (R) CK(cudaMemcpyAsync(R, s->R, 4 * (size_t)L0.nc * sizeof(double), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    if (phx) ST(to_host(s, phx, s->phx, 2 * (size_t)L0.nfx * s->nv));
    if (phy) ST(to_host(s, phy, s->phy, 2 * (size_t)L0.nfy * s->nv));
    return MIUGKS_OK;
}


miugks_status miugks_stage_sgs_micro(miugks_solver* s, int lev, const double* inv_tau, const double* r, double* x)
{
    ST(check_level(s, lev));
    HLevel& Lv = s->lev[lev];
    size_t n = 2 * (size_t)Lv.nc * s->nv;
    CK(cudaMemcpyAsync(Lv.inv_tau, inv_tau, Lv.nc * sizeof(double), cudaMemcpyHostToDevice, s->st));
    ST(to_device(s, Lv.r, r, n));
    MicroArgs mi = micro_args(s, lev);
    if (s->mixed) {
        k_invD_from_itau<float><<<Lv.nc, 128, 0, s->st>>>(Lv.dev, s->vel, Lv.inv_tau, (float*)Lv.invD);
        CK(cudaGetLastError());
        CK(launch_micro_sgs<float>(mi, sweep_plan(s, Lv), s->Zw, (float*)Lv.invD, (float*)Lv.r, (float*)Lv.dl, (float*)s->xcorner, s->st));
    } else {
        k_invD_from_itau<double><<<Lv.nc, 128, 0, s->st>>>(Lv.dev, s->vel, Lv.inv_tau, (double*)Lv.invD);
        CK(cudaGetLastError());
        CK(launch_micro_sgs<double>(mi, sweep_plan(s, Lv), s->Zw, (double*)Lv.invD, (double*)Lv.r, (double*)Lv.dl, (double*)s->xcorner,
                                    s->st));
    }
    return to_host(s, x, Lv.dl, n);
}

miugks_status miugks_stage_apply_micro(miugks_solver* s, int lev, const double* inv_tau, const double* x, double* y)
{
    ST(check_level(s, lev));
    HLevel& Lv = s->lev[lev];
    size_t n = 2 * (size_t)Lv.nc * s->nv;
    CK(cudaMemcpyAsync(Lv.inv_tau, inv_tau, Lv.nc * sizeof(double), cudaMemcpyHostToDevice, s->st));
    ST(to_device(s, Lv.dl, x, n));
    CK(cudaMemsetAsync(Lv.r, 0, n * s->fsz, s->st));
    MicroArgs mi = micro_args(s, lev);
    if (s->mixed) CK(launch_micro_renew<float>(mi, s->Zw, (float*)Lv.dl, (float*)Lv.r, nullptr, 1, s->st));
    else CK(launch_micro_renew<double>(mi, s->Zw, (double*)Lv.dl, (double*)Lv.r, nullptr, 1, s->st));
    std::vector<double> h(n);
    ST(to_host(s, h.data(), Lv.r, n));
    for (size_t q = 0; q < n; ++q) y[q] = -h[q];
    return MIUGKS_OK;
}

miugks_status miugks_stage_sgs_macro(miugks_solver* s, int lev, const double* W, const double* Wg, const double* R,
                                     double* dW)
{
    ST(check_level(s, lev));
    HLevel& Lv = s->lev[lev];
    size_t n4 = 4 * (size_t)Lv.nc;
    CK(cudaMemcpyAsync(Lv.Wc, W, n4 * sizeof(double), cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(Lv.Wn, Wg, n4 * sizeof(double), cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(Lv.R, R, n4 * sizeof(double), cudaMemcpyHostToDevice, s->st));
    MacroArgs ma = macro_args(s, lev, dtn_inv(s));   // the diagonal of the current iteration
    CK(launch_macro_gamma(ma, Lv.Wn, Lv.gx, Lv.gy, Lv.idiag, s->st));
    CK(macro_sgs(s, ma, Lv));
    CK(cudaMemcpyAsync(dW, Lv.dW, n4 * sizeof(double), cudaMemcpyDeviceToHost, s->st));
    double flag = 0.0;
    CK(cudaMemcpyAsync(&flag, s->rms_out + 5, sizeof flag, cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    if (flag != 0.0) return fail(s, MIUGKS_ETIMEOUT, "a bounded wait of the macro sweep gave up");
    return MIUGKS_OK;
}

miugks_status miugks_stage_resid_macro(miugks_solver* s, int lev, const double* W, const double* Wg, double* RE)
{
    ST(check_level(s, lev));
    HLevel& Lv = s->lev[lev];
    size_t n4 = 4 * (size_t)Lv.nc;
    CK(cudaMemcpyAsync(Lv.Wc, W, n4 * sizeof(double), cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(Lv.Wn, Wg, n4 * sizeof(double), cudaMemcpyHostToDevice, s->st));
    CK(cudaMemsetAsync(Lv.P, 0, n4 * sizeof(double), s->st));
    MacroArgs ma = macro_args(s, lev, 0.0);
    CK(launch_macro_gamma(ma, Lv.Wn, Lv.gx, Lv.gy, Lv.idiag, s->st));
    CK(launch_macro_resid(ma, Lv.Wc, Lv.gx, Lv.gy, Lv.P, Lv.R, 1, s->st));
    CK(cudaMemcpyAsync(RE, Lv.R, n4 * sizeof(double), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    return MIUGKS_OK;
}

static miugks_status transfer(miugks_solver* s, int lev, int m, const double* in, double* out, bool up)
{
    ST(check_level(s, lev));
    if (lev + 1 >= s->L) return fail(s, MIUGKS_EINVAL, "no coarser level below %d", lev);
    if (m < 1) return fail(s, MIUGKS_EINVAL, "m must be positive");
    HLevel& F = s->lev[lev];
    HLevel& C = s->lev[lev + 1];
    size_t nin = (size_t)(up ? F.nc : C.nc) * m, nout = (size_t)(up ? C.nc : F.nc) * m;
    double *din, *dout;
    cudaError_t e = cudaMalloc(&din, nin * sizeof(double));
    if (e != cudaSuccess) return fail(s, MIUGKS_ENOMEM, "cudaMalloc: %s", cudaGetErrorString(e));
    e = cudaMalloc(&dout, nout * sizeof(double));
    if (e != cudaSuccess) { cudaFree(din); return fail(s, MIUGKS_ENOMEM, "cudaMalloc: %s", cudaGetErrorString(e)); }
    e = cudaMemcpyAsync(din, in, nin * sizeof(double), cudaMemcpyHostToDevice, s->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dout, 0, nout * sizeof(double), s->st);
    if (e == cudaSuccess)
        e = up ? launch_restrict<double>(F.dev, C.dev, m, 1, din, dout, s->st)
               : launch_prolong_add<double>(F.dev, C.dev, m, 1, F.pidx, F.pw, din, dout, nullptr, s->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, nout * sizeof(double), cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    cudaFree(din);
    cudaFree(dout);
    if (e != cudaSuccess) return fail(s, MIUGKS_ECUDA, "transfer: %s", cudaGetErrorString(e));
    return MIUGKS_OK;
}

miugks_status miugks_stage_restrict(miugks_solver* s, int lev, int m, const double* fine, double* coarse)
{
    return transfer(s, lev, m, fine, coarse, true);
}

miugks_status miugks_stage_prolong(miugks_solver* s, int lev, int m, const double* coarse, double* fine)
{
    return transfer(s, lev, m, coarse, fine, false);
}

} // extern "C"

// =========================================================================== adjoint (differentiation form)
namespace {

constexpr int kDotBlocks = 608;
constexpr int kInnerRestart = 20;           // basis of the inner (macroscopic) Krylov solve of the adjoint
constexpr int kInnerIters = 40;
constexpr double kInnerTol = 1e-2;

bool closed_domain(const miugks_solver* s)
{
    for (const BcDev& b : s->bch)
        if (b.type != BC_WALL && b.type != BC_SYMMETRY) return false;
    return true;
}

miugks_status adj_prepare_levels(miugks_solver* s);
miugks_status refresh_invD(miugks_solver* s);

// allocate the adjoint work (basis of m + 1 vectors) and take the FP64 checkpoint of f
miugks_status adj_prepare(miugks_solver* s, int m)
{
    HLevel& L0 = s->lev[0];
    if (s->shock) return fail(s, MIUGKS_EINVAL, "adjoint: the pressure-jump collision time is not differentiated");
    const size_t n = 2 * (size_t)L0.nc * s->nv;
    auto& A = s->adj;
    if (!A.alloc) {
        ST(dalloc(s, &A.f, n)); ST(dalloc(s, &A.W, 4 * (size_t)L0.nc)); ST(dalloc(s, &A.q, 2 * (size_t)L0.nc));
        ST(dalloc(s, &A.itau, (size_t)L0.nc));
        ST(dalloc(s, &A.recx, (size_t)kFaceRec * L0.nfx)); ST(dalloc(s, &A.recy, (size_t)kFaceRec * L0.nfy));
        ST(dalloc(s, &A.crec, (size_t)kCellRec * L0.nc));
        ST(dalloc(s, &A.b, n)); ST(dalloc(s, &A.x, n)); ST(dalloc(s, &A.w, n)); ST(dalloc(s, &A.z, n));
        ST(dalloc(s, &A.t, n));
        ST(dalloc(s, &A.part, (size_t)kDotBlocks * 33 + L0.nc));
        ST(dalloc(s, &A.fpart, 4 * (size_t)(L0.nfx + L0.nfy)));
        ST(dalloc(s, &A.faces, (size_t)(L0.nfx + L0.nfy)));
        ST(dalloc(s, &A.gx, (size_t)L0.nfx)); ST(dalloc(s, &A.gy, (size_t)L0.nfy));
        ST(dalloc(s, &A.idiag, (size_t)L0.nc)); ST(dalloc(s, &A.binv, 16 * (size_t)L0.nc));
        ST(dalloc(s, &A.m4, 4 * (size_t)L0.nc)); ST(dalloc(s, &A.w4, 8 * (size_t)L0.nc));
        ST(dalloc(s, &A.t4, 4 * (size_t)L0.nc));
        ST(dalloc(s, &A.Vi, (size_t)(kInnerRestart + 1) * 4 * L0.nc));
        A.alloc = true;
    }
    if (m > A.m) {
        ST(dalloc(s, &A.Vb, (size_t)(m + 1) * n));
        ST(dalloc(s, &A.Zb, (size_t)m * n));
        A.m = m;
    }
    if (s->mixed) CK(launch_to_double<float>((const float*)s->f, A.f, n, s->st));
    else CK(cudaMemcpyAsync(A.f, s->f, n * sizeof(double), cudaMemcpyDeviceToDevice, s->st));
    CK(launch_moments<double>(L0.dev, s->vel, A.f, A.W, A.q, s->st));
    CK(launch_inv_tau(s->gas, A.W, L0.nc, A.itau, s->st));
    MacroArgs ma = macro_args(s, 0, 0.0);
    CK(launch_macro_gamma(ma, A.W, A.gx, A.gy, A.idiag, s->st));
    CK(launch_macro_jacT(ma, A.W, A.gx, A.gy, nullptr, nullptr, A.binv, s->st));
    return adj_prepare_levels(s);
}

// per-level work of the transposed CS cycle; W and 1/tau of every level from
// the volume-restricted checkpoint (the coarse collision time of the forward cycle)
miugks_status adj_prepare_levels(miugks_solver* s)
{
    auto& A = s->adj;
    if (!A.lv_alloc) {
        for (int l = 0; l < s->L; ++l) {
            HLevel& Lv = s->lev[l];
            auto& V = A.lv[l];
            const size_t n = 2 * (size_t)Lv.nc * s->nv;
            if (l > 0) {
                ST(dalloc(s, &V.W, 4 * (size_t)Lv.nc)); ST(dalloc(s, &V.itau, (size_t)Lv.nc));
                ST(dalloc(s, &V.z, n)); ST(dalloc(s, &V.o, n));
            }
            for (int q = 0; q < 6; ++q) ST(dalloc(s, &V.T[q], n));
            ST(dalloc(s, &V.invD, (size_t)Lv.nc * s->nv));
            if (l + 1 < s->L) {
                // inverse of the bilinear prolongation stencil (same weights as the forward cycle)
                HLevel& C = s->lev[l + 1];
                std::vector<std::vector<std::pair<int, double>>> inv((size_t)C.nc);
                for (int j = 0; j < Lv.ny; ++j)
                    for (int i = 0; i < Lv.nx; ++i) {
                        int idx[4];
                        double pw[4];
                        prolong_stencil(Lv, C, i, j, idx, pw);
                        int c = j * Lv.nx + i;
                        for (int q = 0; q < 4; ++q) inv[(size_t)idx[q]].push_back({c, pw[q]});
                    }
                std::vector<int> ptr(1, 0), cell;
                std::vector<double> w;
                for (auto& v : inv) {
                    for (auto& e : v) { cell.push_back(e.first); w.push_back(e.second); }
                    ptr.push_back((int)cell.size());
                }
                ST(upload(s, &V.pptr, ptr)); ST(upload(s, &V.pcell, cell)); ST(upload(s, &V.pw, w));
            }
        }
        A.lv_alloc = true;
    }
    A.lv[0].W = A.W;
    A.lv[0].itau = A.itau;
    for (int l = 1; l < s->L; ++l) {
        CK(launch_restrict<double>(s->lev[l - 1].dev, s->lev[l].dev, 4, 1, A.lv[l - 1].W, A.lv[l].W, s->st));
        CK(launch_inv_tau(s->gas, A.lv[l].W, s->lev[l].nc, A.lv[l].itau, s->st));
    }
    return refresh_invD(s);
}

// inverse diagonals of every level from the current collision frequencies
miugks_status refresh_invD(miugks_solver* s)
{
    for (int l = 0; l < s->L; ++l)
        CK(launch_adjoint_invD(s->lev[l].dev, s->vel, s->adj.lv[l].itau, s->adj.lv[l].invD, s->st));
    return MIUGKS_OK;
}

AdjSweepArgs lvl_args(miugks_solver* s, int l, const double* r, double* out)
{
    auto& V = s->adj.lv[l];
    return AdjSweepArgs{s->lev[l].dev, s->vel, s->bc, s->Cw, s->Zw, V.itau, V.invD, r, V.T[5], out};
}

// out = S^T r and y = A^T x on level l
miugks_status sweep_T(miugks_solver* s, int l, const double* r, double* out)
{
    const HLevel& Lv = s->lev[l];
    AdjBodyPlan P{};
    for (int p = 0; p < 2; ++p) {
        P.cells[p] = Lv.adjb[p];
        P.step[p] = Lv.adjstep[p].data();
        P.off[p] = Lv.adjoff[p].data();
        P.ngroups[p] = (int)Lv.adjstep[p].size();
    }
    CK(launch_adjoint_sgs(lvl_args(s, l, r, out), P, s->st));
    return MIUGKS_OK;
}
miugks_status apply_AT(miugks_solver* s, int l, const double* x, double* y)
{
    CK(launch_adjoint_apply(lvl_args(s, l, nullptr, nullptr), x, y, s->st));
    return MIUGKS_OK;
}
// t <- E^T t = t - S^T (A^T t), with work vectors a, b
miugks_status step_ET(miugks_solver* s, int l, double* t, double* a, double* b)
{
    const size_t n = 2 * (size_t)s->lev[l].nc * s->nv;
    ST(apply_AT(s, l, t, a));
    ST(sweep_T(s, l, a, b));
    CK(launch_axpy(t, b, -1.0, n, s->st));
    return MIUGKS_OK;
}

// out = M_l^T z, M_l the CS cycle of level l (Eq. CSCYC) as a linear map of its
// residual: M_l = sum_{m<nu1} S E^m + P M_{l+1} R E^nu1 + sum_{m<nu2} S E^m G E^nu1
// with E = I - A S and G = I - A P M_{l+1} R; on the coarsest level
// M = sum_{m<nc} S E^m.  Transposed with E^T = I - S^T A^T:
//   M_l^T z = sum_{m<nu1} (E^T)^m S^T z + (E^T)^nu1 [u + R^T M_{l+1}^T P^T (z - A^T u)],
//   u = sum_{m<nu2} (E^T)^m S^T z.
miugks_status cs_T(miugks_solver* s, int l, const double* z, double* out)
{
    auto& V = s->adj.lv[l];
    const size_t n = 2 * (size_t)s->lev[l].nc * s->nv, nb = n * sizeof(double);
    double **T = V.T;
    const bool coarsest = l == s->L - 1;
    if (coarsest) {
        const int nsm = s->L == 1 ? 1 : s->opts.nu_coarse;
        ST(sweep_T(s, l, z, T[0]));
        CK(cudaMemcpyAsync(out, T[0], nb, cudaMemcpyDeviceToDevice, s->st));
        for (int m = 1; m < nsm; ++m) {
            ST(step_ET(s, l, T[0], T[2], T[3]));
            CK(launch_axpy(out, T[0], 1.0, n, s->st));
        }
        return MIUGKS_OK;
    }
    HLevel& F = s->lev[l];
    HLevel& C = s->lev[l + 1];
    auto& Vc = s->adj.lv[l + 1];
    ST(sweep_T(s, l, z, T[0]));                                   // s0 = S^T z
    CK(cudaMemcpyAsync(T[1], T[0], nb, cudaMemcpyDeviceToDevice, s->st));
    CK(cudaMemcpyAsync(T[2], T[0], nb, cudaMemcpyDeviceToDevice, s->st));
    for (int m = 1; m < s->opts.nu2; ++m) {                        // u = sum_{m<nu2} (E^T)^m s0
        ST(step_ET(s, l, T[2], T[3], T[4]));
        CK(launch_axpy(T[1], T[2], 1.0, n, s->st));
    }
    ST(apply_AT(s, l, T[1], T[2]));                               // w = z - A^T u
    CK(launch_sub(T[2], z, T[2], n, s->st));
    CK(launch_adjoint_prolong_t(F.dev, C.dev, s->nv, V.pptr, V.pcell, V.pw, T[2], Vc.z, s->st));
    ST(cs_T(s, l + 1, Vc.z, Vc.o));
    CK(launch_adjoint_restrict_t(F.dev, C.dev, s->nv, Vc.o, T[3], s->st));
    CK(launch_axpy(T[1], T[3], 1.0, n, s->st));                   // v = u + R^T M^T P^T w
    CK(cudaMemcpyAsync(out, T[0], nb, cudaMemcpyDeviceToDevice, s->st));
    CK(cudaMemcpyAsync(T[2], T[0], nb, cudaMemcpyDeviceToDevice, s->st));
    for (int m = 1; m < s->opts.nu1; ++m) {                        // sum_{m<nu1} (E^T)^m s0
        ST(step_ET(s, l, T[2], T[3], T[4]));
        CK(launch_axpy(out, T[2], 1.0, n, s->st));
    }
    for (int m = 0; m < s->opts.nu1; ++m) ST(step_ET(s, l, T[1], T[3], T[4]));   // (E^T)^nu1 v
    CK(launch_axpy(out, T[1], 1.0, n, s->st));
    return MIUGKS_OK;
}

AdjDev adj_dev(miugks_solver* s)
{
    return AdjDev{s->lev[0].dev, s->vel, s->gas, s->bc, s->Cw, s->adj.f, s->adj.W, s->adj.q, s->opts.cfl};
}

// host sum (fixed order) of nblk x m partials -> out[m]
miugks_status sum_parts(miugks_solver* s, int nblk, int m, double* out)
{
    std::vector<double> h((size_t)nblk * m);
    CK(cudaMemcpyAsync(h.data(), s->adj.part, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    for (int q = 0; q < m; ++q) {
        double a = 0.0;
        for (int b = 0; b < nblk; ++b) a += h[(size_t)b * m + q];
        out[q] = a;
    }
    return MIUGKS_OK;
}

miugks_status vdots_n(miugks_solver* s, const double* Vb, int m, size_t n, const double* w, double* out)
{
    CK(launch_multi_dot(Vb, m, n, w, s->adj.part, kDotBlocks, s->st));
    return sum_parts(s, kDotBlocks, m, out);
}

miugks_status vdots(miugks_solver* s, const double* Vb, int m, const double* w, double* out)
{
    return vdots_n(s, Vb, m, 2 * (size_t)s->lev[0].nc * s->nv, w, out);
}


// w ~ J^{-T} m with J = dR_E/dW at the checkpoint (Gamma frozen there): restarted GMRES,
// right-preconditioned by the inverse transposed diagonal blocks, to kInnerTol
miugks_status macro_solve_T(miugks_solver* s, const double* m, double* w)
{
    auto& A = s->adj;
    HLevel& L0 = s->lev[0];
    const size_t n = 4 * (size_t)L0.nc, nb = n * sizeof(double);
    const int mi = kInnerRestart;
    MacroArgs ma = macro_args(s, 0, 0.0);
    CK(cudaMemsetAsync(w, 0, nb, s->st));
    double bn;
    ST(vdots_n(s, m, 1, n, m, &bn));
    bn = std::sqrt(bn);
    if (!(bn > 0)) return MIUGKS_OK;
    std::vector<double> H((size_t)(mi + 1) * mi), cs(mi), sn(mi), g(mi + 1), y(mi), h(mi + 1), h2(mi + 1);
    int it = 0;
    double rel = 1.0;
    while (it < kInnerIters && rel > kInnerTol) {
        double* V0 = A.Vi;
        CK(launch_macro_jacT(ma, A.W, A.gx, A.gy, w, A.t4, nullptr, s->st));
        CK(cudaMemcpyAsync(V0, m, nb, cudaMemcpyDeviceToDevice, s->st));
        CK(launch_axpy(V0, A.t4, -1.0, n, s->st));
        double beta;
        ST(vdots_n(s, V0, 1, n, V0, &beta));
        beta = std::sqrt(beta);
        rel = beta / bn;
        if (rel <= kInnerTol) break;
        CK(launch_multi_axpy(nullptr, 0, n, nullptr, 1.0 / beta, V0, s->st));
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int jdone = 0;
        for (int j = 0; j < mi && it < kInnerIters; ++j) {
            double* Vj = A.Vi + (size_t)j * n;
            double* Vn = A.Vi + (size_t)(j + 1) * n;
            CK(launch_block_apply(L0.nc, A.binv, Vj, A.w4, s->st));
            CK(launch_macro_jacT(ma, A.W, A.gx, A.gy, A.w4, Vn, nullptr, s->st));
            ST(vdots_n(s, A.Vi, j + 1, n, Vn, h.data()));
            for (int q = 0; q <= j; ++q) h2[q] = -h[q];
            CK(launch_multi_axpy(A.Vi, j + 1, n, h2.data(), 1.0, Vn, s->st));
            ST(vdots_n(s, A.Vi, j + 1, n, Vn, h2.data()));
            for (int q = 0; q <= j; ++q) { h[q] += h2[q]; h2[q] = -h2[q]; }
            CK(launch_multi_axpy(A.Vi, j + 1, n, h2.data(), 1.0, Vn, s->st));
            double hn;
            ST(vdots_n(s, Vn, 1, n, Vn, &hn));
            hn = std::sqrt(hn);
            h[j + 1] = hn;
            if (hn > 0) CK(launch_multi_axpy(nullptr, 0, n, nullptr, 1.0 / hn, Vn, s->st));
            for (int q = 0; q < j; ++q) {
                double a = cs[q] * h[q] + sn[q] * h[q + 1];
                h[q + 1] = -sn[q] * h[q] + cs[q] * h[q + 1];
                h[q] = a;
            }
            double rr = std::hypot(h[j], h[j + 1]);
            cs[j] = rr > 0 ? h[j] / rr : 1.0;
            sn[j] = rr > 0 ? h[j + 1] / rr : 0.0;
            h[j] = rr;
            h[j + 1] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            for (int q = 0; q <= j; ++q) H[(size_t)q * mi + j] = h[q];
            ++it;
            jdone = j + 1;
            rel = std::fabs(g[j + 1]) / bn;
            if (rel <= kInnerTol || hn == 0.0) break;
        }
        for (int q = jdone - 1; q >= 0; --q) {
            double a = g[q];
            for (int p2 = q + 1; p2 < jdone; ++p2) a -= H[(size_t)q * mi + p2] * y[p2];
            y[q] = a / H[(size_t)q * mi + q];
        }
        CK(launch_multi_axpy(A.Vi, jdone, n, y.data(), 0.0, A.t4, s->st));
        CK(launch_block_apply(L0.nc, A.binv, A.t4, A.w4, s->st));
        CK(launch_axpy(w, A.w4, 1.0, n, s->st));
    }
    return MIUGKS_OK;
}

// out = B v = -((dN/df)^T v - m (m . v)/|m|^2 in a closed domain)
miugks_status apply_B(miugks_solver* s, const double* v, double* out, double mm)
{
    HLevel& L0 = s->lev[0];
    const size_t n = 2 * (size_t)L0.nc * s->nv;
    double pen = 0.0;
    if (mm > 0.0) {
        CK(launch_mass_dot(L0.dev, s->vel, v, s->adj.part, s->st));
        double mv;
        ST(sum_parts(s, L0.nc, 1, &mv));
        pen = -mv / mm;
    }
    CK(launch_adjoint_residual(adj_dev(s), v, s->adj.recx, s->adj.recy, s->adj.crec, pen, out, s->st));
    CK(launch_multi_axpy(nullptr, 0, n, nullptr, -1.0, out, s->st));
    return MIUGKS_OK;
}

// preconditioner of the adjoint solve: the transposed CS cycle of the solver's
// own multigrid (one transposed LU-SGS pass on a single grid)
//
// With the macroscopic correction the preconditioner is the transpose of the
// forward iteration's linearisation, prediction included: the forward step is
// df = M r with r = N + (dr/dW~) dW~ and dW~ = -J^{-1} R, R ~ Pi N (the moments of
// the residual), so P = M (I - (dr/dW~) J^{-1} Pi) and
//   P^T z = y - Pi^T J^{-T} (dr/dW~)^T y,   y = M^T z.
// The inner solve with J^T is inexact, so the outer Krylov method is flexible GMRES.
miugks_status apply_PT_cycle(miugks_solver* s, const double* r, double* out)
{
    ST(cs_T(s, 0, r, out));
    if (!s->adj.macro) return MIUGKS_OK;
    auto& A = s->adj;
    HLevel& L0 = s->lev[0];
    double* w = A.w4 + 4 * (size_t)L0.nc;
    CK(launch_adjoint_macro_m(adj_dev(s), out, A.m4, s->st));
    ST(macro_solve_T(s, A.m4, w));
    if (closed_domain(s)) {
        // the total mass is a null direction of J^T there (V_c in the density of every cell):
        // keep w orthogonal to it, or the inexact inner solve can drift along it
        CK(launch_macro_null_dot(L0.dev, w, A.part, 64, s->st));
        double wn, nn = 0.0;
        ST(sum_parts(s, 64, 1, &wn));
        for (int j = 0; j < L0.ny; ++j)
            for (int i = 0; i < L0.nx; ++i) nn += (L0.dx[i] * L0.dy[j]) * (L0.dx[i] * L0.dy[j]);
        CK(launch_macro_null_sub(L0.dev, wn / nn, w, s->st));
    }
    CK(launch_adjoint_macro_spread(L0.dev, s->vel, w, out, s->st));
    return MIUGKS_OK;
}

// On a mesh with bodies the transposed cycle carries the wall coupling of the bodies' faces (the
// sweep adds it after the wavefront step that reaches each such cell; AdjBodyPlan), and its
// values in the cells of bodies, which hold no state, are zeroed.
miugks_status apply_PT(miugks_solver* s, const double* r, double* out)
{
    ST(apply_PT_cycle(s, r, out));
    HLevel& L0 = s->lev[0];
    if (L0.nfluid != L0.nc) CK(launch_zero_solid(L0.dev, s->nv, out, s->st));
    return MIUGKS_OK;
}

miugks_status wall_face_list(miugks_solver* s, int bc, int* nfaces)
{
    HLevel& L0 = s->lev[0];
    std::vector<int> faces;
    for (int fi = 0; fi < L0.nfx; ++fi) if (L0.fbx[fi] == bc) faces.push_back(fi);
    for (int fi = 0; fi < L0.nfy; ++fi) if (L0.fby[fi] == bc) faces.push_back((1 << 30) | fi);
    *nfaces = (int)faces.size();
    if (!faces.empty())
        CK(cudaMemcpyAsync(s->adj.faces, faces.data(), faces.size() * sizeof(int), cudaMemcpyHostToDevice, s->st));
    return MIUGKS_OK;
}

// J, dJ/dtheta at fixed f (and dJ/df into dJdf_dev when not null) from the checkpoint
miugks_status objective_dev(miugks_solver* s, int obj, int bc, double* dJdf_dev, double out[4])
{
    int nf = 0;
    ST(wall_face_list(s, bc, &nf));
    if (dJdf_dev) CK(cudaMemsetAsync(dJdf_dev, 0, 2 * (size_t)s->lev[0].nc * s->nv * sizeof(double), s->st));
    CK(launch_adjoint_objective(adj_dev(s), obj, bc, s->adj.faces, nf, s->adj.fpart, dJdf_dev, s->st));
    std::vector<double> h(4 * (size_t)nf);
    if (nf) CK(cudaMemcpyAsync(h.data(), s->adj.fpart, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    for (int p = 0; p < 4; ++p) {
        out[p] = 0.0;
        for (int f = 0; f < nf; ++f) out[p] += h[4 * (size_t)f + p];
    }
    return MIUGKS_OK;
}

miugks_status check_wall_args(miugks_solver* s, int obj, int bc)
{
    if (!s->initialised) return fail(s, MIUGKS_ESTATE, "adjoint before init");
    if (bc < 0 || bc >= s->nbc || s->bch[bc].type != BC_WALL) return fail(s, MIUGKS_EINVAL, "BC %d is not a wall", bc);
    if (obj < 0 || obj > 2) return fail(s, MIUGKS_EINVAL, "unknown objective %d", obj);
    if (s->nv > kMaxAdjNv) return fail(s, MIUGKS_EINVAL, "adjoint supports at most %d velocities", kMaxAdjNv);
    return MIUGKS_OK;
}

} // namespace

extern "C" {

miugks_status miugks_stage_adjoint_residual(miugks_solver* s, const double* mu, double* out)
{
    if (!s || !mu || !out) return MIUGKS_EINVAL;
    if (!s->initialised) return fail(s, MIUGKS_ESTATE, "stage before init");
    if (s->nv > kMaxAdjNv) return fail(s, MIUGKS_EINVAL, "adjoint supports at most %d velocities", kMaxAdjNv);
    ST(adj_prepare(s, 0));
    const size_t n = 2 * (size_t)s->lev[0].nc * s->nv;
    CK(cudaMemcpyAsync(s->adj.b, mu, n * sizeof(double), cudaMemcpyHostToDevice, s->st));
    CK(launch_adjoint_residual(adj_dev(s), s->adj.b, s->adj.recx, s->adj.recy, s->adj.crec, 0.0, s->adj.w, s->st));
    CK(cudaMemcpyAsync(out, s->adj.w, n * sizeof(double), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    return MIUGKS_OK;
}

miugks_status miugks_stage_sgs_micro_transposed(miugks_solver* s, const double* inv_tau, const double* r, double* x)
{
    if (!s || !inv_tau || !r || !x) return MIUGKS_EINVAL;
    if (!s->initialised) return fail(s, MIUGKS_ESTATE, "stage before init");
    if (s->nv > kMaxAdjNv) return fail(s, MIUGKS_EINVAL, "adjoint supports at most %d velocities", kMaxAdjNv);
    ST(adj_prepare(s, 0));
    HLevel& L0 = s->lev[0];
    const size_t n = 2 * (size_t)L0.nc * s->nv;
    CK(cudaMemcpyAsync(s->adj.itau, inv_tau, L0.nc * sizeof(double), cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(s->adj.b, r, n * sizeof(double), cudaMemcpyHostToDevice, s->st));
    ST(refresh_invD(s));
    ST(sweep_T(s, 0, s->adj.b, s->adj.x));
    CK(cudaMemcpyAsync(x, s->adj.x, n * sizeof(double), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    return MIUGKS_OK;
}

miugks_status miugks_set_adjoint_options(miugks_solver* s, int macro_correction)
{
    if (!s) return MIUGKS_EINVAL;
    s->adj.macro = macro_correction != 0;
    return MIUGKS_OK;
}

miugks_status miugks_stage_macro_jacobian_transposed(miugks_solver* s, const double* W, const double* x, double* y)
{
    if (!s || !W || !x || !y) return MIUGKS_EINVAL;
    HLevel& L0 = s->lev[0];
    if (L0.nfluid != L0.nc) return fail(s, MIUGKS_EINVAL, "adjoint: meshes with bodies (solid cells) are not supported");
    const size_t n4 = 4 * (size_t)L0.nc;
    // scratch for this test stage only, released before returning
    const size_t tot = 3 * n4 + (size_t)L0.nfx + L0.nfy + L0.nc;
    double* buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, tot * sizeof(double));
    if (e != cudaSuccess) return fail(s, MIUGKS_ENOMEM, "cudaMalloc: %s", cudaGetErrorString(e));
    double *dW = buf, *dx = dW + n4, *dy = dx + n4, *gx = dy + n4, *gy = gx + L0.nfx, *id = gy + L0.nfy;
    MacroArgs ma = macro_args(s, 0, 0.0);
    e = cudaMemcpyAsync(dW, W, n4 * sizeof(double), cudaMemcpyHostToDevice, s->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dx, x, n4 * sizeof(double), cudaMemcpyHostToDevice, s->st);
    if (e == cudaSuccess) e = launch_macro_gamma(ma, dW, gx, gy, id, s->st);
    if (e == cudaSuccess) e = launch_macro_jacT(ma, dW, gx, gy, dx, dy, nullptr, s->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(y, dy, n4 * sizeof(double), cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    cudaFree(buf);
    if (e != cudaSuccess) return fail(s, MIUGKS_ECUDA, "macro_jacobian_transposed: %s", cudaGetErrorString(e));
    return MIUGKS_OK;
}

miugks_status miugks_stage_cs_transposed(miugks_solver* s, const double* inv_tau, const double* z, double* out)
{
    if (!s || !inv_tau || !z || !out) return MIUGKS_EINVAL;
    if (!s->initialised) return fail(s, MIUGKS_ESTATE, "stage before init");
    if (s->nv > kMaxAdjNv) return fail(s, MIUGKS_EINVAL, "adjoint supports at most %d velocities", kMaxAdjNv);
    ST(adj_prepare(s, 0));
    size_t off = 0;
    for (int l = 0; l < s->L; ++l) {
        CK(cudaMemcpyAsync(s->adj.lv[l].itau, inv_tau + off, s->lev[l].nc * sizeof(double), cudaMemcpyHostToDevice,
                           s->st));
        off += s->lev[l].nc;
    }
    ST(refresh_invD(s));
    const size_t n = 2 * (size_t)s->lev[0].nc * s->nv;
    CK(cudaMemcpyAsync(s->adj.b, z, n * sizeof(double), cudaMemcpyHostToDevice, s->st));
    ST(cs_T(s, 0, s->adj.b, s->adj.x));
    CK(cudaMemcpyAsync(out, s->adj.x, n * sizeof(double), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    return MIUGKS_OK;
}

miugks_status miugks_objective(miugks_solver* s, int obj, int bc, double* J, double* dJdf, double dJdtheta[3])
{
    if (!s) return MIUGKS_EINVAL;
    ST(check_wall_args(s, obj, bc));
    ST(adj_prepare(s, 0));
    double o[4];
    ST(objective_dev(s, obj, bc, dJdf ? s->adj.b : nullptr, o));
    if (J) *J = o[0];
    if (dJdtheta) for (int p = 0; p < 3; ++p) dJdtheta[p] = o[1 + p];
    if (dJdf) {
        CK(cudaMemcpyAsync(dJdf, s->adj.b, 2 * (size_t)s->lev[0].nc * s->nv * sizeof(double), cudaMemcpyDeviceToHost,
                           s->st));
        CK(cudaStreamSynchronize(s->st));
    }
    return MIUGKS_OK;
}

miugks_status miugks_adjoint(miugks_solver* s, int obj, int bc, int param, double tol, int max_iter, int restart,
                             double* grad, double info[3])
{
    if (!s || !grad) return MIUGKS_EINVAL;
    ST(check_wall_args(s, obj, bc));
    if (param < 0 || param > 2) return fail(s, MIUGKS_EINVAL, "unknown parameter %d", param);
    if (restart < 1 || restart > 32) return fail(s, MIUGKS_EINVAL, "restart length must be in 1..32");
    if (!(tol > 0) || max_iter < 1) return fail(s, MIUGKS_EINVAL, "need tol > 0 and max_iter >= 1");
    const int m = restart;
    ST(adj_prepare(s, m));
    HLevel& L0 = s->lev[0];
    const size_t n = 2 * (size_t)L0.nc * s->nv;
    auto& A = s->adj;
    double mm = 0.0;
    if (closed_domain(s)) {
        // |m|^2 = sum_c V_c^2 sum_k w_k^2 (G component)
        double w2 = 0.0;
        for (int k = 0; k < s->nv; ++k) w2 += s->wh[k] * s->wh[k];
        for (int j = 0; j < L0.ny; ++j)
            for (int i = 0; i < L0.nx; ++i) mm += (L0.dx[i] * L0.dy[j]) * (L0.dx[i] * L0.dy[j]) * w2;
    }
    double o[4];
    ST(objective_dev(s, obj, bc, A.b, o));           // b = dJ/df
    double bnorm;
    ST(vdots(s, A.b, 1, A.b, &bnorm));
    bnorm = std::sqrt(bnorm);
    CK(cudaMemsetAsync(A.x, 0, n * sizeof(double), s->st));
    int it = 0;
    double rel = bnorm > 0 ? 1.0 : 0.0;
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m), h(m + 1), h2(m + 1);
    while (bnorm > 0 && it < max_iter && rel > tol) {
        // r = b - B x into V_0
        double* V0 = A.Vb;
        ST(apply_B(s, A.x, A.w, mm));
        CK(cudaMemcpyAsync(V0, A.b, n * sizeof(double), cudaMemcpyDeviceToDevice, s->st));
        CK(launch_axpy(V0, A.w, -1.0, n, s->st));
        double beta;
        ST(vdots(s, V0, 1, V0, &beta));
        beta = std::sqrt(beta);
        rel = beta / bnorm;
        if (rel <= tol) break;
        double sc = 1.0 / beta;
        CK(launch_multi_axpy(nullptr, 0, n, nullptr, sc, V0, s->st));
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int jdone = 0;
        for (int j = 0; j < m && it < max_iter; ++j) {
            double* Vj = A.Vb + (size_t)j * n;
            double* Vn = A.Vb + (size_t)(j + 1) * n;
            double* Zj = A.Zb + (size_t)j * n;       // flexible GMRES: keep the preconditioned vector
            ST(apply_PT(s, Vj, Zj));
            ST(apply_B(s, Zj, Vn, mm));
            // classical Gram-Schmidt, twice
            ST(vdots(s, A.Vb, j + 1, Vn, h.data()));
            for (int q = 0; q <= j; ++q) h2[q] = -h[q];
            CK(launch_multi_axpy(A.Vb, j + 1, n, h2.data(), 1.0, Vn, s->st));
            ST(vdots(s, A.Vb, j + 1, Vn, h2.data()));
            for (int q = 0; q <= j; ++q) { h[q] += h2[q]; h2[q] = -h2[q]; }
            CK(launch_multi_axpy(A.Vb, j + 1, n, h2.data(), 1.0, Vn, s->st));
            double hn;
            ST(vdots(s, Vn, 1, Vn, &hn));
            hn = std::sqrt(hn);
            h[j + 1] = hn;
            if (hn > 0) CK(launch_multi_axpy(nullptr, 0, n, nullptr, 1.0 / hn, Vn, s->st));
            // Givens rotations
            for (int q = 0; q < j; ++q) {
                double a = cs[q] * h[q] + sn[q] * h[q + 1];
                h[q + 1] = -sn[q] * h[q] + cs[q] * h[q + 1];
                h[q] = a;
            }
            double rr = std::hypot(h[j], h[j + 1]);
            cs[j] = rr > 0 ? h[j] / rr : 1.0;
            sn[j] = rr > 0 ? h[j + 1] / rr : 0.0;
            h[j] = rr;
            h[j + 1] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            for (int q = 0; q <= j; ++q) H[(size_t)q * m + j] = h[q];
            ++it;
            jdone = j + 1;
            rel = std::fabs(g[j + 1]) / bnorm;
            if (rel <= tol || hn == 0.0) break;
        }
        // y from the triangular system, x += P^T (V y)
        for (int q = jdone - 1; q >= 0; --q) {
            double a = g[q];
            for (int p2 = q + 1; p2 < jdone; ++p2) a -= H[(size_t)q * m + p2] * y[p2];
            y[q] = a / H[(size_t)q * m + q];
        }
        CK(launch_multi_axpy(A.Zb, jdone, n, y.data(), 0.0, A.w, s->st));
        CK(launch_axpy(A.x, A.w, 1.0, n, s->st));
    }
    // true relative residual of the final iterate
    if (bnorm > 0) {
        ST(apply_B(s, A.x, A.w, mm));
        CK(launch_axpy(A.w, A.b, -1.0, n, s->st));
        double rn;
        ST(vdots(s, A.w, 1, A.w, &rn));
        rel = std::sqrt(rn) / bnorm;
    }
    // gradient: dJ/dtheta|_f + lambda . dN/dtheta|_f with lambda = -x ... sign: B = -(dN/df)^T, B x = dJ/df
    // gives (dN/df)^T x = -dJ/df, so lambda = x
    int nf = 0;
    ST(wall_face_list(s, bc, &nf));
    CK(launch_adjoint_dtheta(adj_dev(s), bc, A.faces, nf, A.x, A.fpart, s->st));
    std::vector<double> hp(3 * (size_t)nf);
    if (nf) CK(cudaMemcpyAsync(hp.data(), A.fpart, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    double ln = 0.0;
    for (int f = 0; f < nf; ++f) ln += hp[3 * (size_t)f + param];
    *grad = o[1 + param] + ln;
    if (info) { info[0] = o[0]; info[1] = it; info[2] = rel; }
    if (!(rel <= tol)) return fail(s, MIUGKS_ENOTCONVERGED, "adjoint GMRES reached %d iterations at relative residual %.3e",
                                   it, rel);
    return MIUGKS_OK;
}

} // extern "C"

// =========================================================================== checkpoint / resume
extern "C" {

// File layout (native byte order): 8-byte magic "MIUGKSv1", int32 nx, ny, nu, nvv, nbc, iter,
// then nbc x {int32 type, 4 doubles rho, u, v, T}, then f as FP64 [2][nc][nv].
miugks_status miugks_save(miugks_solver* s, const char* path)
{
    if (!s || !path) return MIUGKS_EINVAL;
    if (!s->initialised) return fail(s, MIUGKS_ESTATE, "save before init");
    const size_t n = 2 * (size_t)s->lev[0].nc * s->nv;
    std::vector<double> f(n);
    ST(to_host(s, f.data(), s->f, n));
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return fail(s, MIUGKS_EINVAL, "cannot open %s for writing", path);
    const char magic[8] = {'M', 'I', 'U', 'G', 'K', 'S', 'v', '1'};
    int32_t hdr[6] = {s->lev[0].nx, s->lev[0].ny, s->nu, s->nvv, s->nbc, s->iter};
    bool ok = std::fwrite(magic, 1, 8, fp) == 8 && std::fwrite(hdr, sizeof hdr, 1, fp) == 1;
    for (int b = 0; ok && b < s->nbc; ++b) {
        int32_t t = s->bch[b].type;
        double v[4] = {s->bch[b].rho, s->bch[b].u, s->bch[b].v, s->bch[b].t};
        ok = std::fwrite(&t, sizeof t, 1, fp) == 1 && std::fwrite(v, sizeof v, 1, fp) == 1;
    }
    ok = ok && std::fwrite(f.data(), sizeof(double), n, fp) == n;
    ok = (std::fclose(fp) == 0) && ok;
    return ok ? MIUGKS_OK : fail(s, MIUGKS_EINVAL, "write to %s failed", path);
}

miugks_status miugks_load(miugks_solver* s, const char* path)
{
    if (!s || !path) return MIUGKS_EINVAL;
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return fail(s, MIUGKS_EINVAL, "cannot open %s", path);
    char magic[8];
    int32_t hdr[6];
    bool ok = std::fread(magic, 1, 8, fp) == 8 && std::memcmp(magic, "MIUGKSv1", 8) == 0 &&
              std::fread(hdr, sizeof hdr, 1, fp) == 1;
    if (!ok || hdr[0] != s->lev[0].nx || hdr[1] != s->lev[0].ny || hdr[2] != s->nu || hdr[3] != s->nvv ||
        hdr[4] != s->nbc) {
        std::fclose(fp);
        return fail(s, MIUGKS_EINVAL, "%s is not a checkpoint of this mesh, velocity grid and BC table", path);
    }
    std::vector<BcDev> bcs(s->nbc);
    for (int b = 0; ok && b < s->nbc; ++b) {
        int32_t t;
        double v[4];
        ok = std::fread(&t, sizeof t, 1, fp) == 1 && std::fread(v, sizeof v, 1, fp) == 1 && t == s->bch[b].type;
        bcs[b] = BcDev{t, v[0], v[1], v[2], v[3]};
    }
    const size_t n = 2 * (size_t)s->lev[0].nc * s->nv;
    std::vector<double> f(n);
    ok = ok && std::fread(f.data(), sizeof(double), n, fp) == n;
    std::fclose(fp);
    if (!ok) return fail(s, MIUGKS_EINVAL, "%s is truncated or its BC types differ", path);
    for (int b = 0; b < s->nbc; ++b) {
        miugks_bc v{(miugks_bc_type)bcs[b].type, bcs[b].rho, bcs[b].u, bcs[b].v, bcs[b].t};
        ST(miugks_set_bc(s, b, &v));
    }
    ST(miugks_set_f(s, f.data()));
    s->iter = hdr[5];
    return MIUGKS_OK;
}

} // extern "C"
