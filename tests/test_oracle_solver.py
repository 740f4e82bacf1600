"""Pins of the oracle's assembled steps against invariants the method fixes:
conservation, equilibrium fixed points, mirror/transpose symmetry, the LU-SGS
factorisation identities, the collisionless and continuum limits, and the
independence of the converged state from the multigrid cycle."""
import math

import numpy as np
import pytest

import oracle
from paper_1704_03151_gb300 import workloads as wl


def _maxwell(case, rho, U, V, T):
    vg = case["vgrid"]
    u1, _ = oracle.vgrid(vg["nu"], vg["umin"], vg["umax"], vg["rule"])
    v1, _ = oracle.vgrid(vg["nv"], vg["vmin"], vg["vmax"], vg["rule"])
    u, v = np.meshgrid(u1, v1, indexing="ij")
    g = rho / (math.pi * T) * np.exp(-((u - U) ** 2 + (v - V) ** 2) / T)
    return u.ravel(), v.ravel(), g.ravel()


def _weights(case):
    vg = case["vgrid"]
    _, wu = oracle.vgrid(vg["nu"], vg["umin"], vg["umax"], vg["rule"])
    _, wv = oracle.vgrid(vg["nv"], vg["vmin"], vg["vmax"], vg["rule"])
    return np.outer(wu, wv).ravel()


# ------------------------------------------------------------ I1 conservation
def test_closed_cavity_mass_conservation_every_iteration():
    case = wl.cavity(n=12, nvel=12, kn=0.5, lid=0.3, levels=2)
    o = oracle.Oracle(case)
    o.init_fields(*wl.random_fields(case, 11))
    V = np.full(case["nx"] * case["ny"], 1.0 / (case["nx"] * case["ny"]))
    for _ in range(3):
        R = o.residual()
        assert abs(np.dot(V, R[:, 0])) < 1e-14 * np.abs(R[:, 0]).max() * len(V) + 1e-16
        o.step(1)


# ------------------------------------------------------------ I2 equilibrium
def test_uniform_rest_maxwellian_is_a_fixed_point():
    case = wl.cavity(n=8, nvel=28, kn=0.3, lid=0.0, levels=2, vmax=7.0)
    o = oracle.Oracle(case)
    o.init_uniform(1.0, 0.0, 0.0, 1.0)
    f0 = o.get_f()
    res = o.step(2)
    assert np.all(res < 1e-13), res
    f1 = o.get_f()
    assert np.max(np.abs(f1 - f0)) < 1e-13 * np.max(np.abs(f0))


# ------------------------------------------------------------ symmetry of Step 1
def _mirror_f_x(case, f):
    nx, ny, nu, nv = case["nx"], case["ny"], case["vgrid"]["nu"], case["vgrid"]["nv"]
    g = f.reshape(2, ny, nx, nu, nv)
    return g[:, :, ::-1, ::-1, :].reshape(f.shape)


def test_step1_mirror_symmetry():
    case = wl.cavity(n=10, nvel=10, kn=0.2, lid=0.0, levels=1)
    o = oracle.Oracle(case)
    o.init_fields(*wl.random_fields(case, 4, amp=0.1))
    f = o.get_f()
    R1 = o.residual()
    o.set_f(_mirror_f_x(case, f))
    R2 = o.residual()
    nx, ny = case["nx"], case["ny"]
    R1m = R1.reshape(ny, nx, 4)[:, ::-1, :].copy()
    R1m[..., 1] *= -1
    assert np.allclose(R2.reshape(ny, nx, 4), R1m, rtol=1e-11, atol=1e-13 * np.abs(R1).max())


def test_step1_transpose_symmetry():
    case = wl.cavity(n=10, nvel=10, kn=0.2, lid=0.0, levels=1)
    o = oracle.Oracle(case)
    o.init_fields(*wl.random_fields(case, 8, amp=0.1))
    f = o.get_f()
    R1 = o.residual()
    n, nu = 10, 10
    ft = f.reshape(2, n, n, nu, nu).transpose(0, 2, 1, 4, 3).reshape(f.shape)
    o.set_f(ft)
    R2 = o.residual().reshape(n, n, 4)
    R1t = R1.reshape(n, n, 4).transpose(1, 0, 2)[..., [0, 2, 1, 3]]
    assert np.allclose(R2, R1t, rtol=1e-11, atol=1e-13 * np.abs(R1).max())


# ------------------------------------------------------------ flux limits
def test_continuum_limit_flux_is_euler_flux():
    case = wl.cavity(n=6, nvel=44, kn=1e-9, lid=0.0, levels=1, vmax=8.0)
    o = oracle.Oracle(case)
    rho, U, V, T = 1.3, 0.4, -0.2, 1.1
    o.init_uniform(rho, U, V, T)
    _, px, _ = o.stage_flux()
    w = _weights(case)
    u, v, _ = _maxwell(case, 1, 0, 0, 1)
    p = rho * T / 2
    E = 0.5 * rho * (U * U + V * V) + 1.5 * p
    euler = np.array([rho * U, rho * U * U + p, rho * U * V, (E + p) * U])
    nx = case["nx"]
    for fi in [2 * (nx + 1) + 3, 4 * (nx + 1) + 2]:  # interior x-faces
        G, H = px[0, fi], px[1, fi]
        F = np.array([np.dot(w, G), np.dot(w, u * G), np.dot(w, v * G), np.dot(w, 0.5 * (u * u + v * v) * G + H)])
        assert np.allclose(F, euler, rtol=1e-9, atol=1e-10), (F, euler)


def test_free_molecular_flux_of_linear_field():
    case = wl.cavity(n=8, nvel=12, kn=1e9, lid=0.0, levels=1)
    nx, ny = case["nx"], case["ny"]
    o = oracle.Oracle(case)
    u, v, g = _maxwell(case, 1.0, 0.1, 0.0, 1.0)
    xc = 0.5 * (case["x_nodes"][1:] + case["x_nodes"][:-1])
    beta = 0.3 * g * (1 + 0.5 * np.sin(np.arange(len(g))))
    f = np.zeros((2, nx * ny, len(g)))
    for j in range(ny):
        for i in range(nx):
            f[0, j * nx + i] = g + beta * xc[i]
            f[1, j * nx + i] = 0.5 * (g + beta * xc[i])
    o.set_f(f)
    _, px, _ = o.stage_flux()
    h = 1.0 / nx
    dt = case["mg"]["cfl"] * h / case["vgrid"]["umax"]  # physical time step rule of the solver
    for i in range(2, nx - 1):  # faces whose both neighbours have two-sided slopes
        fi = 3 * (nx + 1) + i
        xf = case["x_nodes"][i]
        expect = u * (g + beta * xf) - 0.5 * dt * u * u * beta
        assert np.allclose(px[0, fi], expect, rtol=1e-8, atol=1e-12), i


# ------------------------------------------------------------ micro LU-SGS identities
def _dense(apply, n):
    A = np.zeros((n, n))
    for q in range(n):
        e = np.zeros(n)
        e[q] = 1.0
        A[:, q] = apply(e)
    return A


def _one_cell_case(types, nvel=6):
    """1 x 1 cell with BC types (west, east, south, north)."""
    W, E, S, N = types
    fbx, fby = wl.edge_face_ids(1, 1, 0, 1, 2, 3)
    bcs = [wl.bc(t, u=0.1 * q, t=1.0 + 0.1 * q) for q, t in enumerate(types)]
    return {
        "nx": 1, "ny": 1, "x_nodes": np.array([0.0, 0.7]), "y_nodes": np.array([0.0, 0.4]),
        "face_bc_x": fbx, "face_bc_y": fby, "bcs": bcs,
        "vgrid": {"nu": nvel, "nv": nvel, "umin": -3.0, "umax": 3.0, "vmin": -3.0, "vmax": 3.0, "rule": 0},
        "gas": {"kn": 0.5, "omega": 0.81, "pr": 2 / 3},
        "mg": {"levels": 1, "nu1": 2, "nu2": 1, "nuc": 4, "cfl": 0.8, "dtn_growth": 0.0},
    }


@pytest.mark.parametrize("lower", [(0, 0), (1, 0), (0, 1), (1, 1), (3, 0), (2, 1)])
def test_sgs_boundary_block_is_exact(lower):
    """One cell: the forward sweep solves (D + B_lower) x* = r and the backward
    sweep (D + B_upper) x = D x* exactly, B the ghost couplings of the faces
    on each side (walls, symmetry, farfield, outflow; corners included)."""
    F = wl.FARFIELD
    types = (lower[0], 0, lower[1], 0)  # upper faces: walls
    full, lo, up, none = (oracle.Oracle(_one_cell_case(t)) for t in
                          (types, (types[0], F, types[2], F), (F, types[1], F, types[3]), (F, F, F, F)))
    nv = full.nv
    inv_tau = np.array([0.8])
    n = 2 * nv
    A_lo = _dense(lambda x: lo.apply_micro(0, inv_tau, x.reshape(2, 1, nv)).ravel(), n)
    A_up = _dense(lambda x: up.apply_micro(0, inv_tau, x.reshape(2, 1, nv)).ravel(), n)
    Dm = _dense(lambda x: none.apply_micro(0, inv_tau, x.reshape(2, 1, nv)).ravel(), n)
    assert np.allclose(Dm, np.diag(np.diag(Dm)))
    r = np.random.default_rng(1).normal(size=n)
    x = full.sgs_micro(0, inv_tau, r.reshape(2, 1, nv)).ravel()
    ref = np.linalg.solve(A_up, Dm @ np.linalg.solve(A_lo, r))
    assert np.allclose(x, ref, rtol=1e-11, atol=1e-12 * np.abs(ref).max())


def test_sgs_is_lusgs_factorisation_interior():
    """Farfield box: one SGS pass from zero is (D + U)^-1 D (D + L)^-1 r."""
    case = wl.cavity(n=3, nvel=4, levels=1)
    case["nx"], case["ny"] = 3, 4
    case["y_nodes"] = np.array([0.0, 0.2, 0.5, 0.7, 1.0])
    case["face_bc_x"], case["face_bc_y"] = wl.edge_face_ids(3, 4, 0, 0, 0, 0)
    case["bcs"] = [wl.bc(wl.FARFIELD)]
    o = oracle.Oracle(case)
    nc, nv = 12, o.nv
    inv_tau = np.linspace(0.5, 1.5, nc)
    n = 2 * nc * nv
    A = _dense(lambda x: o.apply_micro(0, inv_tau, x.reshape(2, nc, nv)).ravel(), n)
    cell = (np.arange(n) // nv) % nc
    same = cell[:, None] == cell[None, :]
    D = np.where(same, A, 0.0)
    assert np.allclose(D, np.diag(np.diag(D)))
    L = np.where(cell[:, None] > cell[None, :], A, 0.0)
    U = np.where(cell[:, None] < cell[None, :], A, 0.0)
    r = np.random.default_rng(2).normal(size=n)
    x = o.sgs_micro(0, inv_tau, r.reshape(2, nc, nv)).ravel()
    ref = np.linalg.solve(D + U, D @ np.linalg.solve(D + L, r))
    assert np.allclose(x, ref, rtol=1e-11, atol=1e-12 * np.abs(ref).max())


def test_sgs_wavefront_equals_serial_bitwise():
    for case in (wl.cavity(n=7, nvel=6, levels=1), wl.couette(n=6, nvel=6, nx=5)):
        o = oracle.Oracle(case)
        nc, nv = case["nx"] * case["ny"], o.nv
        rng = np.random.default_rng(3)
        r = rng.normal(size=(2, nc, nv))
        it = rng.uniform(0.3, 2.0, nc)
        assert np.array_equal(o.sgs_micro(0, it, r, order=0), o.sgs_micro(0, it, r, order=1))
        o.init_fields(*wl.random_fields(case, 2))
        W = np.zeros((nc, 4))
        m = o.macro()
        W[:, 0] = m["rho"]
        W[:, 1] = m["rho"] * m["u"]
        W[:, 2] = m["rho"] * m["v"]
        W[:, 3] = 0.5 * m["rho"] * (m["u"] ** 2 + m["v"] ** 2) + 0.75 * m["rho"] * m["t"]
        R = 1e-3 * rng.normal(size=(nc, 4))
        assert np.array_equal(o.sgs_macro(0, W, W, R, order=0), o.sgs_macro(0, W, W, R, order=1))


def test_upwind_operator_conserves_mass_with_walls():
    """Without collisions, sum_i V_i sum_k w_k (A x)_ik,G = net wall mass flux = 0."""
    case = wl.cavity(n=5, nvel=8, lid=0.2, levels=1)
    case["x_nodes"] = np.array([0.0, 0.1, 0.35, 0.5, 0.8, 1.0])
    o = oracle.Oracle(case)
    nc, nv = 25, o.nv
    x = np.random.default_rng(4).normal(size=(2, nc, nv))
    y = o.apply_micro(0, np.zeros(nc), x)
    w = _weights(case)
    V = np.outer(np.diff(case["y_nodes"]), np.diff(case["x_nodes"])).ravel()
    tot = np.dot(V, y[0] @ w)
    assert abs(tot) < 1e-13 * np.dot(V, np.abs(y[0]) @ w)


def test_upwind_operator_annihilates_wall_equilibrium():
    """Walls (and symmetry planes) at rest, one temperature: the wall Maxwellian
    C_k, uniform in space, is a null vector of the collisionless operator."""
    for case in (wl.cavity(n=4, nvel=8, lid=0.0, levels=1, t_wall=1.3),
                 wl.couette(n=4, nvel=8, t_bottom=1.3, t_top=1.3, u_top=0.0)):
        o = oracle.Oracle(case)
        nc = case["nx"] * case["ny"]
        _, _, C = _maxwell(case, 1.0, 0.0, 0.0, 1.3)
        x = np.stack([np.tile(C, (nc, 1)), np.tile(C * 1.3 / 4, (nc, 1))])
        y = o.apply_micro(0, np.zeros(nc), x)
        assert np.max(np.abs(y)) < 1e-12 * np.max(np.abs(x)) * 10


def test_sgs_exact_for_one_sided_velocities():
    """All discrete velocities in one quadrant: the upwind system is triangular
    in sweep order, so one SGS pass is the exact solve."""
    case = wl.cavity(n=4, nvel=4, levels=1)
    case["vgrid"].update(umin=0.5, umax=3.5, vmin=0.25, vmax=2.0)
    o = oracle.Oracle(case)
    nc, nv = 16, o.nv
    it = np.linspace(0.2, 1.0, nc)
    n = 2 * nc * nv
    A = _dense(lambda x: o.apply_micro(0, it, x.reshape(2, nc, nv)).ravel(), n)
    r = np.random.default_rng(6).normal(size=n)
    x = o.sgs_micro(0, it, r.reshape(2, nc, nv)).ravel()
    assert np.allclose(x, np.linalg.solve(A, r), rtol=1e-11, atol=1e-12)


# ------------------------------------------------------------ macro smoother
def test_macro_residual_equilibrium_and_conservation():
    case = wl.cavity(n=6, nvel=4, lid=0.0, levels=1, t_wall=1.0)
    o = oracle.Oracle(case)
    nc = 36
    W = np.tile([1.0, 0.0, 0.0, 0.75], (nc, 1))
    assert np.max(np.abs(o.resid_macro(0, W, W))) < 1e-14
    rng = np.random.default_rng(7)
    W2 = W * (1 + 0.05 * rng.uniform(-1, 1, (nc, 4)))
    W2[:, 1:3] = 0.05 * rng.uniform(-1, 1, (nc, 2))
    RE = o.resid_macro(0, W2, W)
    assert abs(RE[:, 0].sum()) < 1e-14 * nc  # walls carry no mass in the split flux


def test_macro_smoother_converges_to_split_residual_root():
    case = wl.cavity(n=6, nvel=4, lid=0.2, levels=1)
    o = oracle.Oracle(case)
    nc = 36
    rng = np.random.default_rng(8)
    Wn = np.tile([1.0, 0.0, 0.0, 0.75], (nc, 1)) + 0.01 * rng.uniform(-1, 1, (nc, 4))
    P = 1e-2 * rng.normal(size=(nc, 4))
    P[:, 0] -= P[:, 0].mean()  # a closed box exchanges no mass: a root needs zero net mass forcing
    P -= o.resid_macro(0, Wn, Wn)
    W = Wn.copy()
    for _ in range(200):
        R = P + o.resid_macro(0, W, Wn)
        W += o.sgs_macro(0, W, Wn, R)
    assert np.max(np.abs(P + o.resid_macro(0, W, Wn))) < 1e-12


# ------------------------------------------------------------ I3 free-molecular limit
def test_free_molecular_fourier_half_range_solution():
    """Collisionless heat conduction between two diffuse plates at rest (bottom
    T_b, top T_t) with specular planes on the sides: every cell holds the
    bottom wall's Maxwellian for v > 0 and the top wall's for v < 0, with
    densities fixed by the discrete zero-mass-flux balance."""
    Tb, Tt = 1.0, 1.4
    case = wl.couette(n=6, nvel=16, kn=1e7, t_bottom=Tb, t_top=Tt, u_top=0.0, nx=2)
    o = oracle.Oracle(case)
    o.init_uniform(1.0, 0.0, 0.0, 1.2)
    res = o.step(120)
    assert np.all(res < 1e-11), res
    u, v, C1 = _maxwell(case, 1.0, 0.0, 0.0, Tb)
    _, _, C2 = _maxwell(case, 1.0, 0.0, 0.0, Tt)
    w = _weights(case)
    f = o.get_f()
    up, dn = v > 0, v < 0
    rho1, rho2 = f[0, 0, up][0] / C1[up][0], f[0, 0, dn][0] / C2[dn][0]
    # zero net mass flux (discrete half-range balance)
    assert abs(rho1 * np.dot(w[up], v[up] * C1[up]) + rho2 * np.dot(w[dn], v[dn] * C2[dn])) < 1e-6 * rho1
    for c in range(f.shape[1]):
        assert np.allclose(f[0, c, up], rho1 * C1[up], rtol=1e-6)
        assert np.allclose(f[0, c, dn], rho2 * C2[dn], rtol=1e-6)
        assert np.allclose(f[1, c, up], f[0, c, up] * Tb / 4, rtol=1e-6)  # H = G K/(4 lambda_w)
        assert np.allclose(f[1, c, dn], f[0, c, dn] * Tt / 4, rtol=1e-6)
    # heat flux into the top wall = energy flux of the two half-range streams
    p, tau, q = o.wall(1)
    e = lambda C, T: 0.5 * (u * u + v * v) * C + C * T / 4
    q_exact = np.dot(w[up], v[up] * rho1 * e(C1, Tb)[up]) + np.dot(w[dn], v[dn] * rho2 * e(C2, Tt)[dn])
    assert np.allclose(q, q_exact, rtol=1e-6)
    assert np.allclose(tau, 0.0, atol=1e-10)


# ------------------------------------------------------------ multigrid consistency
def test_multigrid_and_single_grid_reach_the_same_steady_state():
    """The converged state solves the discrete steady equations and does not
    depend on the cycle.  A closed cavity fixes its state only up to the total
    mass (which the implicit iterations do not conserve), so the top is a
    farfield stream here, which pins the density level."""
    # 24 nodes on [-6, 6]: quadrature moments of a Maxwellian exact to round-off,
    # so the discrete steady state has a zero macroscopic residual
    out = {}
    for levels, iters in ((1, 600), (3, 200)):
        case = wl.cavity(n=8, nvel=24, kn=0.3, lid=0.2, vmax=6.0, levels=levels)
        case["bcs"][2] = wl.bc(wl.FARFIELD, rho=1.0, u=0.2, v=0.0, t=1.0)
        o = oracle.Oracle(case)
        o.init_uniform(1.0, 0.0, 0.0, 1.0)
        for _ in range(iters):
            res = o.step(1)
            if np.all(res < 1e-12):
                break
        assert np.all(res < 1e-11), (levels, res)
        out[levels] = o.macro()
    for k in ("rho", "u", "v", "t"):
        assert np.allclose(out[1][k], out[3][k], rtol=1e-9, atol=1e-10), k


def test_w_and_f_cycles_reach_the_v_cycle_steady_state():
    """W and F cycles (Sec. 3.4 names them) change the path, not the fixed
    point: all three reach the same discrete steady state, and on a 3-level
    hierarchy the first iterates differ (the coarse levels are visited more)."""
    out, first = {}, {}
    for cyc in ("V", "W", "F"):
        case = wl.cavity(n=8, nvel=24, kn=0.3, lid=0.2, vmax=6.0, levels=3)
        case["bcs"][2] = wl.bc(wl.FARFIELD, rho=1.0, u=0.2, v=0.0, t=1.0)
        o = oracle.Oracle(case)
        o.set_cycle(cyc)
        o.init_uniform(1.0, 0.0, 0.0, 1.0)
        o.step(1)
        first[cyc] = o.get_f()
        for _ in range(300):
            res = o.step(1)
            if np.all(res < 1e-12):
                break
        assert np.all(res < 1e-11), (cyc, res)
        out[cyc] = o.macro()
    for a, b in (("V", "W"), ("W", "F"), ("V", "F")):
        assert np.abs(first[a] - first[b]).max() > 1e-9 * np.abs(first["V"]).max(), (a, b)
    for cyc in ("W", "F"):
        for k in ("rho", "u", "v", "t"):
            assert np.allclose(out[cyc][k], out["V"][k], rtol=1e-9, atol=1e-10), (cyc, k)


def _farfield_cavity(levels=3):
    case = wl.cavity(n=8, nvel=24, kn=0.3, lid=0.2, vmax=6.0, levels=levels)
    case["bcs"][2] = wl.bc(wl.FARFIELD, rho=1.0, u=0.2, v=0.0, t=1.0)
    return case


def test_adaptive_cycle_limits_are_the_v_and_w_cycles():
    """The adaptive cycle (Sec. 3.4 names it; reading: a second coarse visit
    when the first left more than a ratio of the coarse residual) is built
    from the same visits as V and W: with ratio 0 every decision is a second
    visit and its iterates are the W cycle's bit for bit, with a ratio no
    visit reaches they are the V cycle's."""
    f = {}
    for cyc, ratio in (("V", None), ("W", None), ("A0", 0.0), ("Ainf", 1e300)):
        o = oracle.Oracle(_farfield_cavity())
        o.set_cycle(cyc[0])
        if ratio is not None:
            o.set_adapt_ratio(ratio)
        o.init_uniform(1.0, 0.0, 0.0, 1.0)
        o.step(3)
        f[cyc] = o.get_f()
        if cyc == "A0":
            log = o.adapt_log()
            assert log.size > 0 and np.all(log == 1)
        if cyc == "Ainf":
            log = o.adapt_log()
            assert log.size > 0 and np.all(log == 0)
    assert np.array_equal(f["A0"], f["W"])
    assert np.array_equal(f["Ainf"], f["V"])
    assert not np.array_equal(f["V"], f["W"])


def test_adaptive_cycle_reaches_the_v_cycle_steady_state():
    """With the default ratio (0.2) the adaptive cycle takes both decisions along the
    way and converges to the V cycle's discrete steady state."""
    out = {}
    for cyc in ("V", "A"):
        o = oracle.Oracle(_farfield_cavity())
        o.set_cycle(cyc)
        o.init_uniform(1.0, 0.0, 0.0, 1.0)
        for _ in range(300):
            res = o.step(1)
            if np.all(res < 1e-12):
                break
        assert np.all(res < 1e-11), (cyc, res)
        out[cyc] = o.macro()
        if cyc == "A":
            log = o.adapt_log()
            assert 0 < log.sum() < log.size, log
    for k in ("rho", "u", "v", "t"):
        assert np.allclose(out["A"][k], out["V"][k], rtol=1e-9, atol=1e-10), k
