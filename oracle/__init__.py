"""Plain FP64 CPU oracle of MIUGKS (arXiv 1704.03151) -- test infrastructure.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It compiles ``oracle.c`` with the host C
compiler (no fast-math) and wraps it with ctypes.  It shares no code with the
CUDA library in ``paper_1704_03151_gb300``.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_LIB_OMP = os.path.join(_BUILD, "liboracle_omp.so")
_lib = None
_lib_omp = None

WALL, SYMMETRY, FARFIELD, OUTFLOW = 0, 1, 2, 3


def build(force=False, omp=False):
    """Compile the oracle into oracle/_build/liboracle.so (gcc, -O2, no fast-math);
    omp=True builds liboracle_omp.so from the same source with -fopenmp (faces,
    cells and the cells of each sweep diagonal over threads, the same bits)."""
    src = os.path.join(_HERE, "oracle.c")
    out = _LIB_OMP if omp else _LIB
    if not force and os.path.exists(out) and os.path.getmtime(out) >= max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fno-fast-math",
                           "-ffp-contract=off"] + (["-fopenmp"] if omp else []) + ["-o", tmp, src, "-lm"])
    os.replace(tmp, out)
    return out


def lib(omp=False):
    global _lib, _lib_omp
    if omp:
        if _lib_omp is None:
            _lib_omp = _declare(ctypes.CDLL(build(omp=True)))
        return _lib_omp
    if _lib is None:
        _lib = _declare(ctypes.CDLL(build()))
    return _lib


def _declare(L):
    """argument and result types of the exported functions"""
    if True:
        P = ctypes.POINTER
        d, i, vp = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        L.oracle_create.restype = vp
        L.oracle_create.argtypes = [i, i, vp, vp, vp, vp, vp, i, vp, vp, i, i, d, d, d, d, i,
                                    d, d, d, i, i, i, i, d, d]
        L.oracle_last_error.restype = ctypes.c_char_p
        L.oracle_destroy.argtypes = [vp]
        L.oracle_init_uniform.argtypes = [vp, d, d, d, d]
        L.oracle_init_fields.argtypes = [vp, vp, vp, vp, vp]
        L.oracle_step.argtypes = [vp, i, vp]
        L.oracle_get_macro.argtypes = [vp] + [vp] * 6
        L.oracle_get_f.argtypes = [vp, vp]
        L.oracle_set_f.argtypes = [vp, vp]
        L.oracle_get_wall.argtypes = [vp, i, P(i), vp, vp, vp]
        L.oracle_set_bc.argtypes = [vp, i, d, d, d, d]
        L.oracle_residual.argtypes = [vp, vp]
        L.oracle_iterations.argtypes = [vp]
        L.oracle_vgrid.argtypes = [i, d, d, i, vp, vp]
        L.oracle_time_coeffs.argtypes = [d, d, vp]
        L.oracle_time_coeffs.restype = None
        L.oracle_micro_slope.argtypes = [vp, d, d, d, vp]
        L.oracle_micro_slope.restype = None
        L.oracle_shakhov.argtypes = [d, d, d, d, d, d, d, i, vp, vp, vp, vp]
        L.oracle_shakhov.restype = None
        L.oracle_vanleer.argtypes = [d, d]
        L.oracle_vanleer.restype = d
        L.oracle_mu_ref.argtypes = [d, d]
        L.oracle_mu_ref.restype = d
        L.oracle_wall_jacobian.argtypes = [vp, d, d, d, vp]
        L.oracle_wall_jacobian.restype = None
        L.oracle_wall_ghost.argtypes = [vp, d, d, d, vp]
        L.oracle_wall_ghost.restype = None
        L.oracle_stage_flux.argtypes = [vp, vp, vp, vp]
        L.oracle_stage_sgs_micro.argtypes = [vp, i, vp, vp, vp, i]
        L.oracle_stage_apply_micro.argtypes = [vp, i, vp, vp, vp]
        L.oracle_stage_sgs_macro.argtypes = [vp, i, vp, vp, vp, vp, i]
        L.oracle_stage_resid_macro.argtypes = [vp, i, vp, vp, vp]
        L.oracle_stage_restrict.argtypes = [vp, i, i, vp, vp]
        L.oracle_stage_prolong.argtypes = [vp, i, i, vp, vp]
        L.oracle_level_size.argtypes = [vp, i, P(i), P(i)]
        L.oracle_nv.argtypes = [vp]
        L.oracle_time_coeffs_dtau.argtypes = [d, d, vp]
        L.oracle_time_coeffs_dtau.restype = None
        L.oracle_micro_slope_adj.argtypes = [vp, d, d, d, vp, vp, vp]
        L.oracle_micro_slope_adj.restype = None
        L.oracle_steady_residual.argtypes = [vp, vp]
        L.oracle_adjoint_residual.argtypes = [vp, vp, vp]
        L.oracle_objective.argtypes = [vp, i, i, vp, vp, vp]
        L.oracle_residual_dtheta.argtypes = [vp, i, i, vp]
        L.oracle_stage_cs.argtypes = [vp, vp, vp, vp]
        L.oracle_set_cycle.argtypes = [vp, i]
        L.oracle_adapt_log.argtypes = [vp, vp, i]
        L.oracle_set_adapt_ratio.argtypes = [vp, d]
        L.oracle_set_shock_capturing.argtypes = [vp, i]
        L.oracle_init_from_coarse.argtypes = [vp, vp]
    return L


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(st):
    if st:
        raise RuntimeError("oracle: " + lib().oracle_last_error().decode())


class Oracle:
    """One MIUGKS problem on the oracle.  ``case`` is a dict from
    ``paper_1704_03151_gb300.workloads`` (mesh nodes, face BC ids, BC table,
    velocity grid, gas and multigrid options)."""

    def __init__(self, case, omp=False):
        """omp=True: the OpenMP build of the same source (same results bit for bit)."""
        self._L = L = lib(omp)
        self.case = case
        self.nx, self.ny = case["nx"], case["ny"]
        self.nc = self.nx * self.ny
        self._keep = [np.ascontiguousarray(case[k], dtype=np.float64) for k in ("x_nodes", "y_nodes")]
        self._keep += [np.ascontiguousarray(case[k], dtype=np.int32) for k in ("face_bc_x", "face_bc_y")]
        solid = case.get("solid")
        self.solid = None if solid is None else np.ascontiguousarray(solid, dtype=np.uint8).reshape(-1)
        bt = np.ascontiguousarray([b["type"] for b in case["bcs"]], dtype=np.int32)
        bv = np.ascontiguousarray([[b["rho"], b["u"], b["v"], b["t"]] for b in case["bcs"]], dtype=np.float64)
        self._keep += [bt, bv]
        vg, gas, mg = case["vgrid"], case["gas"], case["mg"]
        self.h = L.oracle_create(self.nx, self.ny, _p(self._keep[0]), _p(self._keep[1]), _p(self._keep[2]),
                                 _p(self._keep[3]), None if self.solid is None else _p(self.solid),
                                 len(bt), _p(bt), _p(bv),
                                 vg["nu"], vg["nv"], vg["umin"], vg["umax"], vg["vmin"], vg["vmax"], vg["rule"],
                                 gas["kn"], gas["omega"], gas["pr"],
                                 mg["levels"], mg["nu1"], mg["nu2"], mg["nuc"], mg["cfl"], mg["dtn_growth"])
        if not self.h:
            raise RuntimeError("oracle_create: " + L.oracle_last_error().decode())
        self.nv = L.oracle_nv(self.h)

    def _check(self, st):
        if st:
            raise RuntimeError("oracle: " + self._L.oracle_last_error().decode())

    def close(self):
        if self.h:
            self._L.oracle_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_from_coarse(self, coarse):
        """Initial state by bilinear prolongation of f from an oracle on the next coarser mesh."""
        self._check(self._L.oracle_init_from_coarse(self.h, coarse.h))

    def set_cycle(self, cycle):
        """Multigrid cycle type of both cycles: "V", "W", "F" or "A" (adaptive)."""
        self._check(self._L.oracle_set_cycle(self.h, {"V": 0, "W": 1, "F": 2, "A": 3}[cycle]))

    def set_shock_capturing(self, on):
        self._check(self._L.oracle_set_shock_capturing(self.h, 1 if on else 0))

    def set_adapt_ratio(self, ratio):
        self._check(self._L.oracle_set_adapt_ratio(self.h, ratio))

    def adapt_log(self, cap=4096):
        """Decisions of the adaptive cycle so far, oldest first (1 = a second coarse visit)."""
        out = np.zeros(cap, dtype=np.uint8)
        n = self._L.oracle_adapt_log(self.h, _p(out), cap)
        return out[:min(n, cap)].copy()

    def init_uniform(self, rho, u, v, t):
        self._check(self._L.oracle_init_uniform(self.h, rho, u, v, t))

    def init_fields(self, rho, u, v, t):
        arrs = [np.ascontiguousarray(a, dtype=np.float64).ravel() for a in (rho, u, v, t)]
        self._check(self._L.oracle_init_fields(self.h, *[_p(a) for a in arrs]))

    def step(self, n=1):
        res = np.zeros(4)
        self._check(self._L.oracle_step(self.h, n, _p(res)))
        return res

    def residual(self):
        R = np.zeros((self.nc, 4))
        self._check(self._L.oracle_residual(self.h, _p(R)))
        return R

    def macro(self):
        out = [np.zeros(self.nc) for _ in range(6)]
        self._check(self._L.oracle_get_macro(self.h, *[_p(a) for a in out]))
        return dict(zip(("rho", "u", "v", "t", "qx", "qy"), out))

    def get_f(self):
        f = np.zeros((2, self.nc, self.nv))
        self._check(self._L.oracle_get_f(self.h, _p(f)))
        return f

    def set_f(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        self._check(self._L.oracle_set_f(self.h, _p(f)))

    def set_bc(self, b, rho, u, v, t):
        self._check(self._L.oracle_set_bc(self.h, b, rho, u, v, t))

    def wall(self, bc):
        n = ctypes.c_int(0)
        self._L.oracle_get_wall(self.h, bc, ctypes.byref(n), None, None, None)
        cap = n.value
        p, tau, q = np.zeros(cap), np.zeros(cap), np.zeros(cap)
        n = ctypes.c_int(cap)
        self._check(self._L.oracle_get_wall(self.h, bc, ctypes.byref(n), _p(p), _p(tau), _p(q)))
        return p, tau, q

    def iterations(self):
        return self._L.oracle_iterations(self.h)

    # ---- steady equations and their adjoint ----
    def steady_residual(self):
        """N(f) of the steady equations at the current f (Eq. microResidualDef
        with the predicted state equal to the moments of f)."""
        N = np.zeros((2, self.nc, self.nv))
        self._check(self._L.oracle_steady_residual(self.h, _p(N)))
        return N

    def adjoint_residual(self, mu):
        """(dN/df)^T mu at the current f."""
        mu = np.ascontiguousarray(mu, dtype=np.float64).reshape(2, self.nc, self.nv)
        out = np.zeros_like(mu)
        self._check(self._L.oracle_adjoint_residual(self.h, _p(mu), _p(out)))
        return out

    def objective(self, obj, bc):
        """J = sum over the faces of wall `bc` of face length x (shear, heat
        flux, pressure)[obj]; returns J, dJ/df and dJ/d(T, u, v) of that wall."""
        J = np.zeros(1)
        dJdf = np.zeros((2, self.nc, self.nv))
        dJdth = np.zeros(3)
        self._check(self._L.oracle_objective(self.h, obj, bc, _p(J), _p(dJdf), _p(dJdth)))
        return float(J[0]), dJdf, dJdth

    def residual_dtheta(self, bc, param):
        """dN/dtheta at fixed f, theta = (T, u, v)[param] of wall `bc`."""
        dN = np.zeros((2, self.nc, self.nv))
        self._check(self._L.oracle_residual_dtheta(self.h, bc, param, _p(dN)))
        return dN

    # ---- stages for the pins ----
    def level_size(self, lev):
        nx, ny = ctypes.c_int(), ctypes.c_int()
        self._check(self._L.oracle_level_size(self.h, lev, ctypes.byref(nx), ctypes.byref(ny)))
        return nx.value, ny.value

    def stage_flux(self):
        nfx, nfy = (self.nx + 1) * self.ny, self.nx * (self.ny + 1)
        R = np.zeros((self.nc, 4))
        px, py = np.zeros((2, nfx, self.nv)), np.zeros((2, nfy, self.nv))
        self._check(self._L.oracle_stage_flux(self.h, _p(R), _p(px), _p(py)))
        return R, px, py

    def sgs_micro(self, lev, inv_tau, r, order=0):
        r = np.ascontiguousarray(r, dtype=np.float64)
        it = np.ascontiguousarray(inv_tau, dtype=np.float64)
        x = np.zeros_like(r)
        self._check(self._L.oracle_stage_sgs_micro(self.h, lev, _p(it), _p(r), _p(x), order))
        return x

    def cs_cycle(self, inv_tau_levels, r):
        """One CS cycle (frozen coefficients) applied to the level-0 residual r."""
        it = np.ascontiguousarray(np.concatenate([np.ravel(a) for a in inv_tau_levels]), dtype=np.float64)
        r = np.ascontiguousarray(r, dtype=np.float64)
        df = np.zeros_like(r)
        self._check(self._L.oracle_stage_cs(self.h, _p(it), _p(r), _p(df)))
        return df

    def apply_micro(self, lev, inv_tau, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        it = np.ascontiguousarray(inv_tau, dtype=np.float64)
        y = np.zeros_like(x)
        self._check(self._L.oracle_stage_apply_micro(self.h, lev, _p(it), _p(x), _p(y)))
        return y

    def sgs_macro(self, lev, W, Wg, R, order=0):
        W, Wg, R = (np.ascontiguousarray(a, dtype=np.float64) for a in (W, Wg, R))
        dW = np.zeros_like(W)
        self._check(self._L.oracle_stage_sgs_macro(self.h, lev, _p(W), _p(Wg), _p(R), _p(dW), order))
        return dW

    def resid_macro(self, lev, W, Wg):
        W, Wg = (np.ascontiguousarray(a, dtype=np.float64) for a in (W, Wg))
        RE = np.zeros_like(W)
        self._check(self._L.oracle_stage_resid_macro(self.h, lev, _p(W), _p(Wg), _p(RE)))
        return RE

    def restrict(self, lev, fine):
        fine = np.ascontiguousarray(fine, dtype=np.float64)
        nx, ny = self.level_size(lev + 1)
        m = fine.shape[-1]
        coarse = np.zeros((nx * ny, m))
        self._check(self._L.oracle_stage_restrict(self.h, lev, m, _p(fine), _p(coarse)))
        return coarse

    def prolong(self, lev, coarse):
        coarse = np.ascontiguousarray(coarse, dtype=np.float64)
        nx, ny = self.level_size(lev)
        m = coarse.shape[-1]
        fine = np.zeros((nx * ny, m))
        self._check(self._L.oracle_stage_prolong(self.h, lev, m, _p(coarse), _p(fine)))
        return fine


def vgrid(n, a, b, rule):
    x, w = np.zeros(n), np.zeros(n)
    _check(lib().oracle_vgrid(n, a, b, rule, _p(x), _p(w)))
    return x, w


def time_coeffs(dt, tau):
    q = np.zeros(5)
    lib().oracle_time_coeffs(dt, tau, _p(q))
    return q


def micro_slope(dw, U, V, lam):
    dw = np.ascontiguousarray(dw, dtype=np.float64)
    a = np.zeros(4)
    lib().oracle_micro_slope(_p(dw), U, V, lam, _p(a))
    return a


def shakhov(rho, U, V, lam, qx, qy, pr, u, v):
    """Shakhov equilibrium (G+, H+) at the nodes (u, v) (Sec. 2.1)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    G, H = np.empty_like(u), np.empty_like(u)
    lib().oracle_shakhov(rho, U, V, lam, qx, qy, pr, u.size, _p(u), _p(v), _p(G), _p(H))
    return G, H


def vanleer(s1, s2):
    return lib().oracle_vanleer(s1, s2)


def mu_ref(kn, omega):
    return lib().oracle_mu_ref(kn, omega)


def wall_jacobian(W, Uw, Vw, Tw):
    W = np.ascontiguousarray(W, dtype=np.float64)
    M = np.zeros(16)
    lib().oracle_wall_jacobian(_p(W), Uw, Vw, Tw, _p(M))
    return M.reshape(4, 4)


def wall_ghost(W, Uw, Vw, Tw):
    W = np.ascontiguousarray(W, dtype=np.float64)
    G = np.zeros(4)
    lib().oracle_wall_ghost(_p(W), Uw, Vw, Tw, _p(G))
    return G


def time_coeffs_dtau(dt, tau):
    q = np.zeros(5)
    lib().oracle_time_coeffs_dtau(dt, tau, _p(q))
    return q


def micro_slope_adj(dw, U, V, lam, abar):
    """Reverse of micro_slope: returns (dL/d dw, dL/d(U, V, lam)) for dL/da = abar."""
    dw = np.ascontiguousarray(dw, dtype=np.float64)
    ab = np.ascontiguousarray(abar, dtype=np.float64)
    dwb, pb = np.zeros(4), np.zeros(3)
    lib().oracle_micro_slope_adj(_p(dw), U, V, lam, _p(ab), _p(dwb), _p(pb))
    return dwb, pb


def closed_domain(case):
    """True when every boundary is a wall or a symmetry plane: the steady
    equations then fix the state only up to its total mass."""
    return all(b["type"] in (WALL, SYMMETRY) for b in case["bcs"])


def mass_weights(o):
    """dM/df of the total mass M = sum_i V_i sum_k w_k G_i,k (2 x nc x nv)."""
    c = o.case
    vg = c["vgrid"]
    _, wu = vgrid(vg["nu"], vg["umin"], vg["umax"], vg["rule"])
    _, wv = vgrid(vg["nv"], vg["vmin"], vg["vmax"], vg["rule"])
    V = np.outer(np.diff(c["y_nodes"]), np.diff(c["x_nodes"])).ravel()
    m = np.zeros((2, o.nc, o.nv))
    m[0] = V[:, None] * np.outer(wu, wv).ravel()[None, :]
    return m


def adjoint_matrix(o):
    """Dense (dN/df)^T at the current f, column by column from adjoint_residual
    (tiny problems only)."""
    n = 2 * o.nc * o.nv
    A = np.zeros((n, n))
    e = np.zeros(n)
    for i in range(n):
        e[i] = 1.0
        A[:, i] = o.adjoint_residual(e).ravel()
        e[i] = 0.0
    return A


def adjoint_gradient(o, obj, bc, param, A=None):
    """Gradient of the wall objective J with respect to theta = (T, u, v)[param]
    of wall `bc` at the current (converged) f of oracle `o`: dense solve of
    (dN/df)^T lambda = -(dJ/df)^T, then dJ/dtheta = dJ/dtheta|_f + lambda .
    dN/dtheta|_f.  In a closed domain the total mass is held fixed: the
    transposed Jacobian gets the rank-one term -m m^T/|m|^2 (m = dM/df), which
    leaves the fixed-mass derivative unchanged.  Returns (gradient, lambda)."""
    if A is None:
        A = adjoint_matrix(o)
    if closed_domain(o.case):
        m = mass_weights(o).ravel()
        A = A - np.outer(m, m) / np.dot(m, m)
    J, dJdf, dJdth = o.objective(obj, bc)
    lam = np.linalg.solve(A, -dJdf.ravel())
    dN = o.residual_dtheta(bc, param)
    return float(dJdth[param] + np.dot(lam, dN.ravel())), lam.reshape(2, o.nc, o.nv)
