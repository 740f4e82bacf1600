"""Parity of the differentiation form (adjoint of the steady equations) of the
CUDA library with the FP64 oracle, through the C ABI: the transposed Jacobian
(dN/df)^T mu element by element on seeded states for every boundary type and
a stretched mesh, the transposed LU-SGS pass against the transpose of the
oracle's assembled smoother, the wall objectives, and the adjoint gradient
against the oracle's dense adjoint gradient and against central differences of
converged GPU forward solves; plus the torch.autograd entry point."""
import numpy as np
import pytest

import oracle
from paper_1704_03151_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03151_gb300 import miugks
    miugks.load()
    return miugks


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _stretched_cavity():
    case = wl.cavity(nx=9, ny=7, nvel=10, kn=0.7, lid=0.3, levels=1)
    case["x_nodes"] = wl.geometric_nodes(0.0, 1.0, 9, 0.05)
    return case


def _open_box():
    nx, ny = 7, 6
    fbx, fby = wl.edge_face_ids(nx, ny, 2, 3, 0, 1)
    case = wl.couette(n=ny, nx=nx, nvel=12, kn=0.4)
    case["face_bc_x"], case["face_bc_y"] = fbx, fby
    case["y_nodes"] = wl.geometric_nodes(0.0, 1.0, ny, 0.1)
    case["bcs"] = [wl.bc(wl.WALL, u=0.2, t=1.1), wl.bc(wl.FARFIELD, rho=1.0, u=0.3, v=-0.1, t=1.0),
                   wl.bc(wl.SYMMETRY), wl.bc(wl.OUTFLOW)]
    case["init"] = {"rho": 1.0, "u": 0.2, "v": 0.0, "t": 1.0}
    return case


def _odd_grid():
    """Odd velocity count (a zero normal velocity at every face), Boole rule."""
    return wl.cavity(n=6, nvel=9, kn=0.4, lid=0.15, levels=1, rule=wl.BOOLE, vmax=4.0)


def _couette_corners():
    """Symmetry-wall corners on both sides of both walls."""
    return wl.couette(n=6, nvel=10, kn=0.3, t_bottom=1.0, t_top=1.3, u_top=0.2, nx=5)


CASES = {"stretched_cavity": _stretched_cavity, "open_box": _open_box, "odd_grid": _odd_grid,
         "couette_corners": _couette_corners}


def _pair(lib, case, seed):
    o, g = oracle.Oracle(case), lib.Solver(case)
    fields = wl.random_fields(case, seed, amp=0.1)
    o.init_fields(*fields)
    g.init_fields(*fields)
    rng = np.random.default_rng(seed)
    f = o.get_f() * (1 + 0.03 * rng.uniform(-1, 1, size=(2, o.nc, o.nv)))
    o.set_f(f)
    g.set_f(f)
    return o, g, rng


@pytest.mark.parametrize("name", sorted(CASES))
def test_adjoint_residual_matches_oracle(lib, name):
    o, g, rng = _pair(lib, CASES[name](), 11)
    for _ in range(2):
        mu = rng.normal(size=(2, o.nc, o.nv))
        assert rel(g.adjoint_residual(mu), o.adjoint_residual(mu)) < TOL, name


def test_adjoint_residual_with_slopes_near_underflow_matches_oracle(lib):
    """One velocity at values of 1e-158 (van Leer slopes whose product is
    subnormal, as in the far tails of the 89^2 grid at Ma 5): the limiter's
    derivative stays finite and matches the oracle."""
    o, g, rng = _pair(lib, _stretched_cavity(), 13)
    f = o.get_f()
    nvv = int(round(np.sqrt(o.nv)))
    k0 = (nvv - 1) * nvv + nvv // 2                 # the largest u > 0
    ix = np.arange(o.nc) % o.nx
    for cp in range(2):
        f[cp, :, k0] = 1e-158 * (1.0 + 0.2 * ix) * (1 + cp)
    o.set_f(f)
    g.set_f(f)
    mu = rng.normal(size=(2, o.nc, o.nv))
    out = g.adjoint_residual(mu)
    assert np.all(np.isfinite(out))
    assert rel(out, o.adjoint_residual(mu)) < TOL


def _dense_sgs(o, inv_tau):
    n = 2 * o.nc * o.nv
    S = np.zeros((n, n))
    e = np.zeros(n)
    for i in range(n):
        e[i] = 1.0
        S[:, i] = o.sgs_micro(0, inv_tau, e.reshape(2, o.nc, o.nv)).ravel()
        e[i] = 0.0
    return S


@pytest.mark.parametrize("name", ["cavity", "open_box", "couette_corners", "odd_grid"])
def test_transposed_sgs_is_the_transpose_of_the_oracle_smoother(lib, name):
    if name == "cavity":
        case = wl.cavity(nx=4, ny=3, nvel=6, kn=0.5, lid=0.2, levels=1)
    elif name == "open_box":
        case = _open_box()
        case["nx"], case["ny"] = 4, 3
        case["x_nodes"], case["y_nodes"] = np.linspace(0, 1, 5), wl.geometric_nodes(0.0, 1.0, 3, 0.2)
        case["face_bc_x"], case["face_bc_y"] = wl.edge_face_ids(4, 3, 2, 3, 0, 1)
        case["vgrid"].update(nu=6, nv=6)
    elif name == "couette_corners":
        case = wl.couette(n=3, nvel=6, kn=0.3, nx=4)
    else:
        case = wl.cavity(n=3, nvel=5, kn=0.4, lid=0.15, levels=1, rule=wl.BOOLE, vmax=4.0)
    o, g, rng = _pair(lib, case, 5)
    inv_tau = rng.uniform(0.5, 3.0, size=o.nc)
    ST = _dense_sgs(o, inv_tau).T
    for _ in range(2):
        r = rng.normal(size=(2, o.nc, o.nv))
        assert rel(g.sgs_micro_transposed(inv_tau, r), (ST @ r.ravel()).reshape(r.shape)) < TOL, name


def test_transposed_sgs_dot_product_on_a_larger_grid(lib):
    case = wl.cavity(nx=24, ny=17, nvel=16, kn=0.3, lid=0.2, levels=1)
    o, g, rng = _pair(lib, case, 3)
    inv_tau = rng.uniform(0.5, 3.0, size=o.nc)
    for _ in range(2):
        r, x = rng.normal(size=(2, 2, o.nc, o.nv))
        lhs = np.sum(g.sgs_micro_transposed(inv_tau, r) * x)
        rhs = np.sum(r * o.sgs_micro(0, inv_tau, x))
        assert abs(lhs - rhs) < 1e-11 * np.sqrt(np.sum(r * r) * np.sum(x * x))


@pytest.mark.parametrize("obj", [0, 1, 2])
def test_objective_matches_oracle(lib, obj):
    o, g, _ = _pair(lib, _stretched_cavity(), 2)
    Jo, dfo, dto = o.objective(obj, 2)
    Jg, dfg, dtg = g.objective(obj, 2)
    assert Jg == pytest.approx(Jo, rel=TOL, abs=1e-14)
    assert rel(dfg, dfo) < TOL
    assert np.allclose(dtg, dto, rtol=TOL, atol=1e-13)


def _channel(dt=0.0, du=0.0, n=3, nvel=16):
    c = wl.couette(n=n, nx=n, nvel=nvel, kn=1.0, vmax=5.0, t_bottom=1.0 + dt, t_top=1.0, u_top=0.0)
    c["bcs"][0]["u"] = 0.2 + du
    c["bcs"][1] = wl.bc(wl.FARFIELD, rho=1.0, u=0.0, v=0.0, t=1.2)
    return c


def _closed(dt=0.0, du=0.0):
    c = wl.cavity(nx=3, ny=3, nvel=16, kn=1.0, lid=0.2 + du, levels=1, vmax=5.0)
    c["bcs"][2]["t"] = 1.0 + dt
    return c


@pytest.mark.parametrize("which", ["open", "closed"])
def test_adjoint_gradient_matches_oracle_dense_adjoint(lib, which):
    case, bc = (_channel(), 0) if which == "open" else (_closed(), 2)
    o = oracle.Oracle(case)
    o.init_uniform(1.0, 0.0, 0.0, 1.0)
    o.step(300)
    g = lib.Solver(case)
    g.init_uniform(1.0, 0.0, 0.0, 1.0)
    g.set_f(o.get_f())                       # the same linearisation point
    A = oracle.adjoint_matrix(o)
    for obj, param in ((0, 1), (1, 0), (2, 0)):
        go, _ = oracle.adjoint_gradient(o, obj, bc, param, A=A)
        gg, info = g.adjoint(obj, bc, param, tol=1e-13, max_iter=3000)
        assert info["converged"], info
        assert gg == pytest.approx(go, rel=1e-8, abs=1e-12), (which, obj, param, info)


def test_adjoint_gradient_matches_gpu_converged_differences(lib):
    """Central differences of the GPU forward solve (8x8 channel cells) against
    the GPU adjoint gradient at the converged state."""
    def solve(**kw):
        s = lib.Solver(_channel(n=8, **kw))
        s.init_uniform(1.0, 0.0, 0.0, 1.0)
        s.step(600)
        return s

    s0 = solve()
    for obj, param, h in ((0, 1, 1e-4), (1, 0, 1e-5)):
        gg, info = s0.adjoint(obj, 0, param, tol=1e-12, max_iter=3000)
        assert info["converged"], info
        kw = (lambda sg: {"dt": sg * h}) if param == 0 else (lambda sg: {"du": sg * h})
        fd = (solve(**kw(1)).objective(obj, 0)[0] - solve(**kw(-1)).objective(obj, 0)[0]) / (2 * h)
        assert gg == pytest.approx(fd, rel=1e-5), (obj, param)


def test_mixed_precision_state_gives_the_fp64_gradient_to_its_accuracy(lib):
    case = _channel(n=8)
    grads = {}
    for prec in ("fp64", "mixed"):
        s = lib.Solver(case, precision=prec)
        s.init_uniform(1.0, 0.0, 0.0, 1.0)
        s.step(600)
        grads[prec], info = s.adjoint(0, 0, 1, tol=1e-12, max_iter=3000)
        assert info["converged"], info
    assert grads["mixed"] == pytest.approx(grads["fp64"], rel=1e-4)


def test_torch_autograd_wall_objective(lib):
    import torch
    case = _channel(n=6)
    s = lib.Solver(case)
    theta = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    J = lib.wall_objective(s, theta, obj="heat_flux", bc=0, param="t", tol=1e-8, max_iter=4000)
    J.backward()
    ref, _ = s.adjoint(1, 0, 0, tol=1e-12, max_iter=3000)
    assert float(theta.grad) == pytest.approx(ref, rel=1e-8)
    assert float(J) == pytest.approx(s.objective(1, 0)[0], rel=1e-12)


@pytest.mark.parametrize("levels", [2, 3])
def test_transposed_cs_cycle_is_the_transpose_of_the_oracle_cycle(lib, levels):
    """The adjoint's preconditioner is the exact transpose of one CS cycle
    (frozen coefficients) of the forward solve."""
    n = 4 if levels == 2 else 8
    nvel = 6 if levels == 2 else 4
    case = wl.cavity(n=n, nvel=nvel, kn=0.5, lid=0.2, levels=levels, nx=n, ny=n)
    o, g, rng = _pair(lib, case, 9)
    its = [rng.uniform(0.5, 3.0, size=(n // 2 ** l) ** 2) for l in range(levels)]
    N = 2 * o.nc * o.nv
    M = np.zeros((N, N))
    e = np.zeros(N)
    for i in range(N):
        e[i] = 1.0
        M[:, i] = o.cs_cycle(its, e.reshape(2, o.nc, o.nv)).ravel()
        e[i] = 0.0
    for _ in range(2):
        z = rng.normal(size=(2, o.nc, o.nv))
        assert rel(g.cs_cycle_transposed(its, z), (M.T @ z.ravel()).reshape(z.shape)) < TOL, levels


def test_flat_plate_drag_gradient_matches_oracle(lib):
    """Half-domain flat plate (wall on part of the lower edge, symmetry on the
    rest, farfield elsewhere; stretched mesh): d(drag)/d(plate wall
    temperature) and d(drag)/d(plate velocity) at the converged state."""
    case = wl.flat_plate(kn=0.5, ma=0.2, nvel=16, vmax=5.0, levels=1, n_up=1, n_plate=2, n_down=1, ny=3,
                         growth=1.3)
    o = oracle.Oracle(case)
    o.init_uniform(case["init"]["rho"], case["init"]["u"], case["init"]["v"], case["init"]["t"])
    o.step(300)
    g = lib.Solver(case)
    g.init_uniform(case["init"]["rho"], case["init"]["u"], case["init"]["v"], case["init"]["t"])
    g.set_f(o.get_f())
    A = oracle.adjoint_matrix(o)
    for obj, param in ((0, 0), (0, 1), (1, 0)):
        go, _ = oracle.adjoint_gradient(o, obj, 0, param, A=A)
        gg, info = g.adjoint(obj, 0, param, tol=1e-13, max_iter=3000)
        assert info["converged"], info
        assert gg == pytest.approx(go, rel=1e-8, abs=1e-12), (obj, param, info)


@pytest.mark.parametrize("name", ["stretched_cavity", "open_box", "couette_corners"])
def test_macro_jacobian_transpose_dot_product(lib, name):
    """J^T of the split Euler residual (the prediction step's operator, used by
    the adjoint's macroscopic correction) against central differences of the
    oracle's residual R_E(W) with Gamma frozen: <x, J v> = <J^T x, v>."""
    case = CASES[name]()
    o, g, rng = _pair(lib, case, 13)
    W = np.column_stack([o.macro()[k] for k in ("rho",)])          # shape check only
    m = o.macro()
    rho, u, v, t = m["rho"], m["u"], m["v"], m["t"]
    W = np.column_stack([rho, rho * u, rho * v, 0.5 * rho * (u * u + v * v) + 0.75 * rho * t])
    for _ in range(3):
        x = rng.normal(size=W.shape)
        d = rng.normal(size=W.shape) * np.abs(W)
        h = 1e-6
        fd = (o.resid_macro(0, W + h * d, W) - o.resid_macro(0, W - h * d, W)) / (2 * h)
        lhs = np.sum(x * fd)
        rhs = np.sum(g.macro_jacobian_transposed(W, x) * d)
        assert abs(lhs - rhs) < 1e-7 * max(1.0, abs(lhs)), (name, lhs, rhs)


def test_macro_correction_keeps_the_gradient(lib):
    """The preconditioner changes the Krylov path only: with and without the
    macroscopic correction the adjoint gradient agrees with the oracle's."""
    case, bc = _closed(), 2
    o = oracle.Oracle(case)
    o.init_uniform(1.0, 0.0, 0.0, 1.0)
    o.step(300)
    A = oracle.adjoint_matrix(o)
    go, _ = oracle.adjoint_gradient(o, 0, bc, 1, A=A)
    for corr in (True, False):
        g = lib.Solver(case)
        g.init_uniform(1.0, 0.0, 0.0, 1.0)
        g.set_f(o.get_f())
        g.set_adjoint_options(corr)
        gg, info = g.adjoint(0, bc, 1, tol=1e-13, max_iter=3000)
        assert info["converged"], (corr, info)
        assert gg == pytest.approx(go, rel=1e-8), corr


# ---------------------------------------------------------------- bodies (the square cylinder of Sec. 4.3)
def _body_box(dt=0.0, n_side=1, n_sq=1, half=1.5, nvel=16, levels=1):
    """A box with a body at its centre: isothermal wall on the body (BC 0,
    T_w = 1 + dt), farfield inflow, top and bottom (BC 1), zero-gradient
    outflow (BC 2); Ma 0.5, Kn 1."""
    c = wl.square_cylinder(ma=0.5, kn=1.0, nvel=nvel, vmax=5.0, levels=levels, nx_side=n_side, nx_sq=n_sq,
                           ny_side=n_side, ny_sq=n_sq, half=half, dtn_growth=0.0)
    c["bcs"][0]["t"] = 1.0 + dt
    c.pop("rear")
    return c


def test_adjoint_residual_and_objective_with_bodies_match_oracle(lib):
    """(dN/df)^T mu element by element and the wall objectives of the body
    (face sides found by face id, as in the forward flux; N = -f in the body)."""
    for case in (_body_box(), _body_box(n_side=4, n_sq=2, half=3.0, nvel=10, levels=2)):
        o, g, rng = _pair(lib, case, 13)
        for _ in range(2):
            mu = rng.normal(size=(2, o.nc, o.nv))
            assert rel(g.adjoint_residual(mu), o.adjoint_residual(mu)) < TOL
        for obj in (0, 1, 2):
            Jo, dfo, dto = o.objective(obj, 0)
            Jg, dfg, dtg = g.objective(obj, 0)
            assert Jg == pytest.approx(Jo, rel=TOL, abs=1e-14)
            assert rel(dfg, dfo) < TOL
            assert np.allclose(dtg, dto, rtol=TOL, atol=1e-13)


@pytest.mark.parametrize("levels", [1, 2])
def test_transposed_cs_cycle_around_a_body_is_the_transpose_of_the_oracle_cycle(lib, levels):
    """With a body: the transposed sweep adds the wall coupling of each cell
    with a body face on the pass's side after the wavefront step that reaches
    it, so the preconditioner is again the exact transpose of one CS cycle of
    the forward solve, on the fluid cells (a body's cells hold no unknowns)."""
    case = _body_box(n_side=2, n_sq=2, half=3.0, nvel=4, levels=levels)
    o, g, rng = _pair(lib, case, 21)
    its = [rng.uniform(0.5, 3.0, size=(case["nx"] // 2 ** l) * (case["ny"] // 2 ** l)) for l in range(levels)]
    solid = np.asarray(case["solid"]).astype(bool)
    N = 2 * o.nc * o.nv
    M = np.zeros((N, N))
    e = np.zeros(N)
    for i in range(N):
        e[i] = 1.0
        M[:, i] = o.cs_cycle(its, e.reshape(2, o.nc, o.nv)).ravel()
        e[i] = 0.0
    for _ in range(2):
        z = rng.normal(size=(2, o.nc, o.nv))
        z[:, solid, :] = 0.0
        got = g.cs_cycle_transposed(its, z)
        ref = (M.T @ z.ravel()).reshape(z.shape)
        assert rel(got[:, ~solid], ref[:, ~solid]) < TOL, levels


def test_adjoint_gradient_with_a_body_matches_oracle_dense_adjoint(lib):
    """d(heat flux, shear, pressure on the body)/d(body wall temperature) on
    the 3x3 box with a one-cell body: the GPU adjoint against the oracle's
    dense adjoint gradient."""
    case = _body_box()
    o = oracle.Oracle(case)
    o.init_uniform(1.0, case["init"]["u"], 0.0, 1.0)
    o.step(300)
    g = lib.Solver(case)
    g.init_uniform(1.0, case["init"]["u"], 0.0, 1.0)
    g.set_f(o.get_f())
    A = oracle.adjoint_matrix(o)
    for obj in (1, 0, 2):
        go, _ = oracle.adjoint_gradient(o, obj, 0, 0, A=A)
        gg, info = g.adjoint(obj, 0, 0, tol=1e-13, max_iter=3000)
        assert info["converged"], info
        assert gg == pytest.approx(go, rel=1e-8, abs=1e-12), (obj, info)


def test_body_heat_flux_gradient_matches_gpu_converged_differences(lib):
    """The square cylinder's objective on a 12x12 mesh with a 4x4 body and two
    levels: d(heat flux into the body)/d(T_w) by the adjoint against central
    differences of converged GPU forward solves."""
    def solve(dt):
        c = _body_box(dt, n_side=4, n_sq=4, half=3.0, nvel=16, levels=2)
        s = lib.Solver(c)
        s.init_uniform(1.0, c["init"]["u"], 0.0, 1.0)
        s.step(400)
        return s

    s0 = solve(0.0)
    gg, info = s0.adjoint(1, 0, 0, tol=1e-12, max_iter=3000)
    assert info["converged"], info
    h = 1e-5
    fd = (solve(h).objective(1, 0)[0] - solve(-h).objective(1, 0)[0]) / (2 * h)
    assert gg == pytest.approx(fd, rel=1e-5), (gg, fd, info)
