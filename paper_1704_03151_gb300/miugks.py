"""Python binding of the MIUGKS CUDA library (include/miugks.h).

Argument marshalling only: every step of the method runs in the CUDA kernels
of libmiugks.so.  PyTorch provides the device memory (through the library's
allocator callbacks, backed by PyTorch's caching allocator) and the CUDA
stream.  There is no CPU fallback: without the built library, or without a
CUDA device, creating a solver raises.
"""
import ctypes
import os

import numpy as np

from . import build as _build

MIUGKS_OK, MIUGKS_EINVAL, MIUGKS_ENOMEM, MIUGKS_ECUDA, MIUGKS_EDIVERGED, MIUGKS_ETIMEOUT, \
    MIUGKS_ENOTCONVERGED, MIUGKS_ESTATE = range(8)
WALL, SYMMETRY, FARFIELD, OUTFLOW = 0, 1, 2, 3
PRECISIONS = {"fp64": 0, "mixed": 1}

_d, _i, _vp, _P = ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.POINTER


class miugks_mesh(ctypes.Structure):
    _fields_ = [("nx", _i), ("ny", _i), ("x_nodes", _vp), ("y_nodes", _vp), ("face_bc_x", _vp), ("face_bc_y", _vp),
                ("solid", _vp)]


class miugks_vgrid(ctypes.Structure):
    _fields_ = [("nu", _i), ("nv", _i), ("umin", _d), ("umax", _d), ("vmin", _d), ("vmax", _d), ("rule", _i)]


class miugks_gas(ctypes.Structure):
    _fields_ = [("kn", _d), ("omega", _d), ("pr", _d)]


class miugks_bc(ctypes.Structure):
    _fields_ = [("type", _i), ("rho", _d), ("u", _d), ("v", _d), ("t", _d)]


ALLOC_FN = ctypes.CFUNCTYPE(_vp, ctypes.c_size_t, _vp)
FREE_FN = ctypes.CFUNCTYPE(None, _vp, _vp)


class miugks_opts(ctypes.Structure):
    _fields_ = [("levels", _i), ("nu1", _i), ("nu2", _i), ("nu_coarse", _i), ("cfl", _d), ("dtn_growth", _d),
                ("precision", _i), ("cuda_stream", _vp), ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN),
                ("alloc_ctx", _vp)]


class MiugksError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("miugks status %d: %s" % (status, msg))
        self.status = status


_lib = None


def library_path():
    return _build.LIB


def load():
    """Load libmiugks.so (it must have been built; see __graft_entry__.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        raise ImportError("libmiugks.so is not built (%s); run __graft_entry__.build()" % _build.LIB)
    L = ctypes.CDLL(_build.LIB)
    vp = _vp
    sig = {
        "miugks_create": [_P(miugks_mesh), _P(miugks_vgrid), _P(miugks_gas), _P(miugks_bc), _i, _P(miugks_opts),
                          _P(vp)],
        "miugks_destroy": [vp], "miugks_last_error": [vp],
        "miugks_init_uniform": [vp, _d, _d, _d, _d], "miugks_init_fields": [vp, vp, vp, vp, vp],
        "miugks_step": [vp, _i, vp], "miugks_run": [vp, _d, _i, _P(_i), vp], "miugks_residual": [vp, vp],
        "miugks_iterations": [vp], "miugks_get_macro": [vp] + [vp] * 6, "miugks_get_f": [vp, vp],
        "miugks_set_f": [vp, vp], "miugks_get_wall": [vp, _i, _P(_i), vp, vp, vp],
        "miugks_set_bc": [vp, _i, _P(miugks_bc)],
        "miugks_stage_flux": [vp, vp, vp, vp], "miugks_stage_sgs_micro": [vp, _i, vp, vp, vp],
        "miugks_stage_apply_micro": [vp, _i, vp, vp, vp], "miugks_stage_sgs_macro": [vp, _i, vp, vp, vp, vp],
        "miugks_stage_resid_macro": [vp, _i, vp, vp, vp], "miugks_stage_restrict": [vp, _i, _i, vp, vp],
        "miugks_stage_prolong": [vp, _i, _i, vp, vp], "miugks_sizes": [vp, _P(_i), _P(_i), _P(_i), _P(_i)],
        "miugks_set_timing": [vp, _i], "miugks_kernel_times": [vp, _P(_d), _P(_d), _P(_d)],
        "miugks_step_async": [vp, _i], "miugks_wait": [vp, vp],
        "miugks_stage_adjoint_residual": [vp, vp, vp], "miugks_stage_sgs_micro_transposed": [vp, vp, vp, vp],
        "miugks_stage_cs_transposed": [vp, vp, vp, vp],
        "miugks_objective": [vp, _i, _i, vp, vp, vp],
        "miugks_adjoint": [vp, _i, _i, _i, _d, _i, _i, vp, vp],
        "miugks_save": [vp, ctypes.c_char_p], "miugks_load": [vp, ctypes.c_char_p],
        "miugks_macro_sweep_times": [vp, _P(_d), _P(_i)], "miugks_set_cycle": [vp, _i],
        "miugks_init_from_coarse": [vp, vp],
        "miugks_set_adjoint_options": [vp, _i], "miugks_stage_macro_jacobian_transposed": [vp, vp, vp, vp],
        "miugks_set_adaptive_ratio": [vp, _d], "miugks_adaptive_decisions": [vp, vp, _i],
        "miugks_set_sweep_split": [vp, _i], "miugks_sweep_kernel_times": [vp, vp],
        "miugks_copy_state": [vp, vp], "miugks_set_shock_capturing": [vp, _i],
        "miugks_set_wait_limit": [vp, _d],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = _i
    L.miugks_destroy.restype = None
    L.miugks_last_error.restype = ctypes.c_char_p
    L.miugks_residual_rms_noalloc.argtypes = [vp, vp, vp, _i, vp, vp]
    L.miugks_residual_rms_noalloc.restype = _i
    _lib = L
    return L


def exported_symbols():
    return ["miugks_create", "miugks_destroy", "miugks_last_error", "miugks_init_uniform", "miugks_init_fields",
            "miugks_step", "miugks_run", "miugks_residual", "miugks_iterations", "miugks_get_macro",
            "miugks_get_f", "miugks_set_f", "miugks_get_wall", "miugks_set_bc", "miugks_stage_flux",
            "miugks_stage_sgs_micro", "miugks_stage_apply_micro", "miugks_stage_sgs_macro",
            "miugks_stage_resid_macro", "miugks_stage_restrict", "miugks_stage_prolong", "miugks_sizes",
            "miugks_set_timing", "miugks_kernel_times", "miugks_step_async", "miugks_wait",
            "miugks_stage_adjoint_residual", "miugks_stage_sgs_micro_transposed", "miugks_stage_cs_transposed",
            "miugks_objective",
            "miugks_adjoint", "miugks_residual_rms_noalloc", "miugks_save", "miugks_load",
            "miugks_macro_sweep_times", "miugks_set_cycle", "miugks_init_from_coarse",
            "miugks_set_adjoint_options", "miugks_stage_macro_jacobian_transposed", "miugks_set_adaptive_ratio",
            "miugks_adaptive_decisions", "miugks_set_sweep_split", "miugks_sweep_kernel_times",
            "miugks_copy_state", "miugks_set_shock_capturing", "miugks_set_wait_limit"]


def _ptr(a):
    return a.ctypes.data_as(_vp)


class _TorchAllocator:
    """Device memory for the library from PyTorch's caching allocator."""

    def __init__(self, torch, device):
        self.torch, self.device, self.live = torch, device, {}
        self.alloc_fn = ALLOC_FN(self._alloc)
        self.free_fn = FREE_FN(self._free)

    def _alloc(self, nbytes, ctx):
        try:
            t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device=self.device)
        except Exception:
            return None
        p = t.data_ptr()
        self.live[p] = t
        return p

    def _free(self, ptr, ctx):
        self.live.pop(ptr, None)


class Solver:
    """One MIUGKS problem.  ``case`` is a dict as produced by
    ``paper_1704_03151_gb300.workloads`` (mesh nodes, face BC ids, BC table,
    velocity grid, gas, multigrid options)."""

    def __init__(self, case, use_torch=True, stream=None, precision=None):
        import torch
        if not torch.cuda.is_available():
            raise MiugksError(MIUGKS_ECUDA, "no CUDA device: the MIUGKS library has no CPU path")
        self._lib = L = load()
        self.case = case
        self.nx, self.ny = int(case["nx"]), int(case["ny"])
        self.nc = self.nx * self.ny
        self._arrays = [np.ascontiguousarray(case["x_nodes"], dtype=np.float64),
                        np.ascontiguousarray(case["y_nodes"], dtype=np.float64),
                        np.ascontiguousarray(case["face_bc_x"], dtype=np.int32),
                        np.ascontiguousarray(case["face_bc_y"], dtype=np.int32)]
        solid = case.get("solid")
        if solid is not None:
            self._arrays.append(np.ascontiguousarray(solid, dtype=np.uint8).reshape(-1))
        mesh = miugks_mesh(self.nx, self.ny, *[_ptr(a) for a in self._arrays[:4]],
                           _ptr(self._arrays[4]) if solid is not None else None)
        vg = case["vgrid"]
        vgrid = miugks_vgrid(vg["nu"], vg["nv"], vg["umin"], vg["umax"], vg["vmin"], vg["vmax"], vg["rule"])
        gas = miugks_gas(case["gas"]["kn"], case["gas"]["omega"], case["gas"]["pr"])
        bcs = (miugks_bc * len(case["bcs"]))(*[miugks_bc(b["type"], b["rho"], b["u"], b["v"], b["t"])
                                               for b in case["bcs"]])
        mg = case["mg"]
        dev = torch.device("cuda", torch.cuda.current_device())
        self._stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self._alloc = _TorchAllocator(torch, dev) if use_torch else None
        precision = precision or mg.get("precision", "fp64")
        if precision not in PRECISIONS:
            raise MiugksError(MIUGKS_EINVAL, "precision must be one of %s" % sorted(PRECISIONS))
        self.precision = precision
        opts = miugks_opts(mg["levels"], mg["nu1"], mg["nu2"], mg["nuc"], mg["cfl"], mg["dtn_growth"],
                           PRECISIONS[precision],
                           _vp(self._stream.cuda_stream),
                           self._alloc.alloc_fn if self._alloc else ALLOC_FN(),
                           self._alloc.free_fn if self._alloc else FREE_FN(), None)
        h = _vp()
        st = L.miugks_create(ctypes.byref(mesh), ctypes.byref(vgrid), ctypes.byref(gas), bcs, len(case["bcs"]),
                             ctypes.byref(opts), ctypes.byref(h))
        if st != MIUGKS_OK:
            raise MiugksError(st, L.miugks_last_error(None).decode())
        self.h = h
        nx, ny, nv, lv = _i(), _i(), _i(), _i()
        L.miugks_sizes(h, ctypes.byref(nx), ctypes.byref(ny), ctypes.byref(nv), ctypes.byref(lv))
        self.nv, self.levels = nv.value, lv.value

    def _check(self, st):
        if st != MIUGKS_OK:
            raise MiugksError(st, self._lib.miugks_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self._lib.miugks_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- C ABI, same names without the prefix
    def init_uniform(self, rho, u, v, t):
        self._check(self._lib.miugks_init_uniform(self.h, rho, u, v, t))

    def init_fields(self, rho, u, v, t):
        a = [np.ascontiguousarray(x, dtype=np.float64).ravel() for x in (rho, u, v, t)]
        self._check(self._lib.miugks_init_fields(self.h, *[_ptr(x) for x in a]))

    def step(self, n=1):
        res = np.zeros(4)
        self._check(self._lib.miugks_step(self.h, n, _ptr(res)))
        return res

    def step_async(self, n=1):
        self._check(self._lib.miugks_step_async(self.h, n))

    def wait(self):
        res = np.zeros(4)
        self._check(self._lib.miugks_wait(self.h, _ptr(res)))
        return res

    def run(self, tol, max_iter):
        res = np.zeros(4)
        it = _i()
        st = self._lib.miugks_run(self.h, tol, max_iter, ctypes.byref(it), _ptr(res))
        if st not in (MIUGKS_OK, MIUGKS_ENOTCONVERGED):
            self._check(st)
        return it.value, res, st == MIUGKS_OK

    def residual(self):
        res = np.zeros(4)
        self._check(self._lib.miugks_residual(self.h, _ptr(res)))
        return res

    def iterations(self):
        return self._lib.miugks_iterations(self.h)

    def macro(self):
        out = [np.zeros(self.nc) for _ in range(6)]
        self._check(self._lib.miugks_get_macro(self.h, *[_ptr(a) for a in out]))
        return dict(zip(("rho", "u", "v", "t", "qx", "qy"), out))

    def get_f(self):
        f = np.zeros((2, self.nc, self.nv))
        self._check(self._lib.miugks_get_f(self.h, _ptr(f)))
        return f

    def set_f(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        self._check(self._lib.miugks_set_f(self.h, _ptr(f)))

    def set_bc(self, b, type_, rho, u, v, t):
        self._check(self._lib.miugks_set_bc(self.h, b, ctypes.byref(miugks_bc(type_, rho, u, v, t))))

    def init_from_coarse(self, coarse):
        """Initial state by bilinear prolongation of f from a solver on the next coarser mesh."""
        self._check(self._lib.miugks_init_from_coarse(self.h, coarse.h))

    def copy_state(self, src):
        """f (converted to this solver's precision) and the iteration count of src."""
        self._check(self._lib.miugks_copy_state(self.h, src.h))

    def set_cycle(self, cycle):
        """Multigrid cycle type of both cycles: "V", "W", "F" or "A" (adaptive)."""
        self._check(self._lib.miugks_set_cycle(self.h, {"V": 0, "W": 1, "F": 2, "A": 3}[cycle]))

    def set_wait_limit(self, seconds):
        """Bound of the prediction sweep's device waits (0.2 s by default)."""
        self._check(self._lib.miugks_set_wait_limit(self.h, float(seconds)))

    def set_shock_capturing(self, on):
        """Pressure-jump term of the interface collision time (off by default)."""
        self._check(self._lib.miugks_set_shock_capturing(self.h, 1 if on else 0))

    def set_sweep_split(self, mode):
        """Evolution-sweep layout: "auto" (by level size), "split" or "wave" (same results)."""
        self._check(self._lib.miugks_set_sweep_split(self.h, {"auto": 0, "split": 1, "wave": 2}[mode]))

    def set_adaptive_ratio(self, ratio):
        self._check(self._lib.miugks_set_adaptive_ratio(self.h, float(ratio)))

    def adaptive_decisions(self, cap=4096):
        """Decisions of the adaptive cycle so far, oldest first (1 = a second coarse visit)."""
        out = np.zeros(cap, dtype=np.uint8)
        n = self._lib.miugks_adaptive_decisions(self.h, _ptr(out), cap)
        return out[:min(n, cap)].copy()

    def wall(self, bc):
        n = _i(0)
        self._check(self._lib.miugks_get_wall(self.h, bc, ctypes.byref(n), None, None, None))
        p, tau, q = np.zeros(n.value), np.zeros(n.value), np.zeros(n.value)
        self._check(self._lib.miugks_get_wall(self.h, bc, ctypes.byref(n), _ptr(p), _ptr(tau), _ptr(q)))
        return p, tau, q

    def set_timing(self, on):
        self._check(self._lib.miugks_set_timing(self.h, 1 if on else 0))

    def kernel_times(self):
        a, b, c = _d(), _d(), _d()
        self._check(self._lib.miugks_kernel_times(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def sweep_kernel_times(self):
        """Finest-level evolution-sweep kernels since the last call (timing mode):
        {"wave": (ms, launches, cell-velocity pairs), "lines": (...)}."""
        out = np.zeros(6)
        self._check(self._lib.miugks_sweep_kernel_times(self.h, _ptr(out)))
        return {"wave": (out[0], int(out[1]), out[2]), "lines": (out[3], int(out[4]), out[5])}

    def macro_sweep_times(self):
        """(total ms, launches) of the finest-level prediction sweeps since the last call."""
        ms, n = _d(), _i()
        self._check(self._lib.miugks_macro_sweep_times(self.h, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    # ---- stages
    def stage_flux(self):
        nfx, nfy = (self.nx + 1) * self.ny, self.nx * (self.ny + 1)
        R = np.zeros((self.nc, 4))
        px, py = np.zeros((2, nfx, self.nv)), np.zeros((2, nfy, self.nv))
        self._check(self._lib.miugks_stage_flux(self.h, _ptr(R), _ptr(px), _ptr(py)))
        return R, px, py

    def sgs_micro(self, lev, inv_tau, r):
        r = np.ascontiguousarray(r, dtype=np.float64)
        it = np.ascontiguousarray(inv_tau, dtype=np.float64)
        x = np.zeros_like(r)
        self._check(self._lib.miugks_stage_sgs_micro(self.h, lev, _ptr(it), _ptr(r), _ptr(x)))
        return x

    def apply_micro(self, lev, inv_tau, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        it = np.ascontiguousarray(inv_tau, dtype=np.float64)
        y = np.zeros_like(x)
        self._check(self._lib.miugks_stage_apply_micro(self.h, lev, _ptr(it), _ptr(x), _ptr(y)))
        return y

    def sgs_macro(self, lev, W, Wg, R):
        W, Wg, R = (np.ascontiguousarray(a, dtype=np.float64) for a in (W, Wg, R))
        dW = np.zeros_like(W)
        self._check(self._lib.miugks_stage_sgs_macro(self.h, lev, _ptr(W), _ptr(Wg), _ptr(R), _ptr(dW)))
        return dW

    def resid_macro(self, lev, W, Wg):
        W, Wg = (np.ascontiguousarray(a, dtype=np.float64) for a in (W, Wg))
        RE = np.zeros_like(W)
        self._check(self._lib.miugks_stage_resid_macro(self.h, lev, _ptr(W), _ptr(Wg), _ptr(RE)))
        return RE

    def restrict(self, lev, fine):
        fine = np.ascontiguousarray(fine, dtype=np.float64)
        m = fine.shape[-1]
        coarse = np.zeros((self.nc // 4 ** (lev + 1), m))
        self._check(self._lib.miugks_stage_restrict(self.h, lev, m, _ptr(fine), _ptr(coarse)))
        return coarse

    def prolong(self, lev, coarse):
        coarse = np.ascontiguousarray(coarse, dtype=np.float64)
        m = coarse.shape[-1]
        fine = np.zeros((self.nc // 4 ** lev, m))
        self._check(self._lib.miugks_stage_prolong(self.h, lev, m, _ptr(coarse), _ptr(fine)))
        return fine

    def save(self, path):
        self._check(self._lib.miugks_save(self.h, os.fsencode(path)))

    def load(self, path):
        self._check(self._lib.miugks_load(self.h, os.fsencode(path)))

    # ---- differentiation form (adjoint of the steady equations)
    def adjoint_residual(self, mu):
        """(dN/df)^T mu at the current f (host arrays, 2 x nc x nv)."""
        mu = np.ascontiguousarray(mu, dtype=np.float64).reshape(2, self.nc, self.nv)
        out = np.zeros_like(mu)
        self._check(self._lib.miugks_stage_adjoint_residual(self.h, _ptr(mu), _ptr(out)))
        return out

    def sgs_micro_transposed(self, inv_tau, r):
        """P^T r, P one LU-SGS pass of the evolution smoother on level 0."""
        r = np.ascontiguousarray(r, dtype=np.float64)
        it = np.ascontiguousarray(inv_tau, dtype=np.float64)
        x = np.zeros_like(r)
        self._check(self._lib.miugks_stage_sgs_micro_transposed(self.h, _ptr(it), _ptr(r), _ptr(x)))
        return x

    def cs_cycle_transposed(self, inv_tau_levels, z):
        """M^T z, M one CS cycle with frozen per-level collision frequencies."""
        it = np.ascontiguousarray(np.concatenate([np.ravel(a) for a in inv_tau_levels]), dtype=np.float64)
        z = np.ascontiguousarray(z, dtype=np.float64)
        out = np.zeros_like(z)
        self._check(self._lib.miugks_stage_cs_transposed(self.h, _ptr(it), _ptr(z), _ptr(out)))
        return out

    def macro_jacobian_transposed(self, W, x):
        """J^T x, J the Jacobian of the split Euler residual at W (Gamma frozen at W)."""
        W = np.ascontiguousarray(W, dtype=np.float64)
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.zeros_like(x)
        self._check(self._lib.miugks_stage_macro_jacobian_transposed(self.h, _ptr(W), _ptr(x), _ptr(y)))
        return y

    def set_adjoint_options(self, macro_correction=True):
        self._check(self._lib.miugks_set_adjoint_options(self.h, 1 if macro_correction else 0))

    def objective(self, obj, bc):
        """J, dJ/df and dJ/d(T, u, v) of wall `bc` at the current f."""
        J = np.zeros(1)
        dJdf = np.zeros((2, self.nc, self.nv))
        dth = np.zeros(3)
        self._check(self._lib.miugks_objective(self.h, obj, bc, _ptr(J), _ptr(dJdf), _ptr(dth)))
        return float(J[0]), dJdf, dth

    def adjoint(self, obj, bc, param, tol=1e-10, max_iter=2000, restart=30):
        """dJ/dtheta at the current (converged) state by the adjoint solve;
        returns (gradient, {"J", "iterations", "residual"}).  At a state
        converged in the mixed form, polish it in FP64 first
        (refine.polish): the Krylov solve then needs several times fewer
        iterations."""
        g = np.zeros(1)
        info = np.zeros(3)
        st = self._lib.miugks_adjoint(self.h, obj, bc, param, tol, max_iter, restart, _ptr(g), _ptr(info))
        if st not in (MIUGKS_OK, MIUGKS_ENOTCONVERGED):
            self._check(st)
        return float(g[0]), {"J": float(info[0]), "iterations": int(info[1]), "residual": float(info[2]),
                             "converged": st == MIUGKS_OK}


OBJECTIVES = {"shear": 0, "heat_flux": 1, "pressure": 2}
PARAMS = {"t": 0, "u": 1, "v": 2}
_WallObjective = None


def wall_objective(solver, theta, obj="shear", bc=0, param="t", tol=1e-10, max_iter=5000, adj_tol=1e-10,
                   adj_max_iter=2000):
    """J(theta): a wall objective at the converged state, as a differentiable
    torch function of one wall parameter (temperature or velocity component of
    wall `bc`).  Forward: set the parameter, run the solver to RMS residual
    `tol`, evaluate J and keep a checkpoint of the converged f.  Backward:
    restore the checkpoint and return the adjoint gradient times the incoming
    gradient.  theta is a 0-d (or 1-element) float64 tensor."""
    global _WallObjective
    import torch
    if _WallObjective is None:
        class _WO(torch.autograd.Function):
            @staticmethod
            def forward(ctx, th, s, o, b, p, tl, mi, atl, ami):
                B = s.case["bcs"][b]
                vals = {"t": B["t"], "u": B["u"], "v": B["v"]}
                vals[p] = float(th.detach().cpu().reshape(-1)[0])
                s.set_bc(b, B["type"], B["rho"], vals["u"], vals["v"], vals["t"])
                s.init_uniform(s.case["init"]["rho"], s.case["init"]["u"], s.case["init"]["v"], s.case["init"]["t"])
                it, res, ok = s.run(tl, mi)
                if not ok:
                    raise MiugksError(MIUGKS_ENOTCONVERGED, "forward solve not converged (%s)" % res)
                J = s.objective(OBJECTIVES[o], b)[0]
                ctx.solver, ctx.args = s, (OBJECTIVES[o], b, PARAMS[p], atl, ami)
                ctx.f_ckpt = s.get_f()
                return th.new_tensor(J)

            @staticmethod
            def backward(ctx, gJ):
                s = ctx.solver
                s.set_f(ctx.f_ckpt)
                obj_, b, p, atl, ami = ctx.args
                g, info = s.adjoint(obj_, b, p, tol=atl, max_iter=ami)
                if not info["converged"]:
                    raise MiugksError(MIUGKS_ENOTCONVERGED, "adjoint not converged (%s)" % info)
                return (gJ * g,) + (None,) * 8

        _WallObjective = _WO
    return _WallObjective.apply(theta, solver, obj, bc, param, tol, max_iter, adj_tol, adj_max_iter)
