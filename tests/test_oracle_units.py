"""Pins of the oracle's building blocks against what mathematics and the paper
fix independently of the oracle's own code: quadrature exactness, definitions
of the time integrals evaluated by numerical integration, continuous moments
evaluated by brute-force 3-D quadrature, finite-difference Jacobians, the
paper's printed prolongation weights, and textbook limits."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1704_03151_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- quadrature
@pytest.mark.parametrize("n,rule,deg", [(20, 0, 1), (33, 0, 1), (89, 1, 5), (21, 1, 5)])
def test_vgrid_exact_polynomials(n, rule, deg):
    x, w = oracle.vgrid(n, -4.0, 4.0, rule)
    for p in range(deg + 1):
        exact = (4.0 ** (p + 1) - (-4.0) ** (p + 1)) / (p + 1)
        assert abs(np.dot(w, x ** p) - exact) <= 1e-11 * max(1.0, abs(exact))
    if rule == 0:  # trapezoid is not exact for degree 2
        assert abs(np.dot(w, x ** 2) - 128.0 / 3) > 1e-6


def test_vgrid_symmetric_nodes_and_gaussian_moments():
    x, w = oracle.vgrid(40, -6.0, 6.0, 0)
    assert np.array_equal(x[::-1], -x)
    lam = 1.3
    g = np.exp(-lam * x * x)
    assert abs(np.dot(w, g) - math.sqrt(math.pi / lam)) < 1e-13
    assert abs(np.dot(w, x * x * g) - 0.5 * math.sqrt(math.pi / lam) / lam) < 1e-13
    with pytest.raises(RuntimeError):
        oracle.vgrid(20, -4.0, 4.0, 1)  # Boole needs (n-1) % 4 == 0


# ---------------------------------------------------------------- gas model
def test_mu_ref_hard_sphere_textbook():
    # Chapman-Enskog hard sphere: mu = (5 sqrt(pi)/16) rho sqrt(2RT) lambda_mfp
    assert abs(oracle.mu_ref(1.0, 0.5) - 5.0 * math.sqrt(math.pi) / 16.0) < 1e-15
    assert abs(oracle.mu_ref(0.075, 0.81) / oracle.mu_ref(1.0, 0.81) - 0.075) < 1e-15


# ---------------------------------------------------------------- time integrals
def _q_by_quadrature(dt, tau):
    from scipy.integrate import quad
    e = lambda t: math.exp(-t / tau)
    kw = dict(epsabs=0.0, epsrel=1e-13, limit=200)
    return np.array([
        quad(lambda t: 1.0 - e(t), 0, dt, **kw)[0],
        quad(lambda t: (t + tau) * e(t) - tau, 0, dt, **kw)[0],
        quad(lambda t: t - tau * (1.0 - e(t)), 0, dt, **kw)[0],
        quad(lambda t: e(t), 0, dt, **kw)[0],
        quad(lambda t: -t * e(t), 0, dt, **kw)[0],
    ])


@pytest.mark.parametrize("x", [1e-6, 1e-3, 0.3, 0.999, 1.0, 1.7, 30.0])
def test_time_coeffs_match_integrals(x):
    dt = 0.013
    tau = dt / x
    q = oracle.time_coeffs(dt, tau)
    ref = _q_by_quadrature(dt, tau)
    scale = np.array([dt, dt * dt, dt * dt, dt, dt * dt])
    assert np.all(np.abs(q - ref) <= 1e-11 * scale), (q, ref)


def test_time_coeffs_limits():
    dt = 0.02
    q = oracle.time_coeffs(dt, 1e-15)  # continuum: g only
    assert np.allclose(q, [dt, 0.0, dt * dt / 2, 0.0, 0.0], atol=1e-11 * dt)
    q = oracle.time_coeffs(dt, 1e12)  # free molecular: f0 only
    assert np.allclose(q, [0.0, 0.0, 0.0, dt, -dt * dt / 2], atol=1e-13 * dt)
    # branch switch at x = 1 is continuous to round-off
    a, b = oracle.time_coeffs(dt, dt / (1 - 1e-12)), oracle.time_coeffs(dt, dt / (1 + 1e-12))
    assert np.all(np.abs(a - b) <= 1e-14 * np.array([dt, dt * dt, dt * dt, dt, dt * dt]) + 1e-10 * np.abs(a))


# ---------------------------------------------------------------- micro slopes
def _continuous_moments_of_slope(a, U, V, lam):
    """Brute-force 3-D quadrature of int psi (a . psi) g du dv dxi (K = 1)."""
    n = 64
    s = 9.0 / math.sqrt(lam)
    u = np.linspace(U - s, U + s, n)
    v = np.linspace(V - s, V + s, n)
    z = np.linspace(-s, s, n)
    h = (u[1] - u[0]) * (v[1] - v[0]) * (z[1] - z[0])
    Uu, Vv, Zz = np.meshgrid(u, v, z, indexing="ij")
    g = (lam / math.pi) ** 1.5 * np.exp(-lam * ((Uu - U) ** 2 + (Vv - V) ** 2 + Zz ** 2))
    e = 0.5 * (Uu ** 2 + Vv ** 2 + Zz ** 2)
    psi = [np.ones_like(Uu), Uu, Vv, e]
    ap = a[0] + a[1] * Uu + a[2] * Vv + a[3] * e
    return np.array([np.sum(p * ap * g) * h for p in psi])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_micro_slope_reproduces_moments(seed):
    rng = np.random.default_rng(seed)
    U, V, lam = rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5), rng.uniform(0.6, 1.8)
    dw = rng.normal(size=4)
    a = oracle.micro_slope(dw, U, V, lam)
    m = _continuous_moments_of_slope(a, U, V, lam)
    assert np.allclose(m, dw, rtol=1e-10, atol=1e-10), (m, dw)


# ---------------------------------------------------------------- limiter
def test_vanleer_properties():
    assert oracle.vanleer(1.0, -2.0) == 0.0
    assert oracle.vanleer(0.0, 3.0) == 0.0
    assert oracle.vanleer(2.0, 2.0) == 2.0
    rng = np.random.default_rng(5)
    for s1, s2 in rng.normal(size=(200, 2)):
        r = oracle.vanleer(s1, s2)
        assert r == oracle.vanleer(s2, s1)
        if s1 * s2 > 0:
            assert abs(r) <= 2 * min(abs(s1), abs(s2)) + 1e-15
            assert abs(r - 2.0 / (1.0 / s1 + 1.0 / s2)) <= 1e-14 * abs(r)


# ---------------------------------------------------------------- wall BC (macro)
def test_wall_jacobian_matches_finite_differences():
    rng = np.random.default_rng(3)
    for _ in range(5):
        rho, U, V, T = rng.uniform(0.6, 1.4), rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), rng.uniform(0.8, 1.3)
        lam = 1.0 / T
        W = np.array([rho, rho * U, rho * V, 0.5 * rho * (U * U + V * V) + 3 * rho / (4 * lam)])
        Uw, Vw, Tw = rng.uniform(-0.2, 0.2), rng.uniform(-0.2, 0.2), rng.uniform(0.9, 1.2)
        M = oracle.wall_jacobian(W, Uw, Vw, Tw)
        J = np.zeros((4, 4))
        for q in range(4):
            h = 1e-6 * max(1.0, abs(W[q]))
            Wp, Wm = W.copy(), W.copy()
            Wp[q] += h
            Wm[q] -= h
            J[:, q] = (oracle.wall_ghost(Wp, Uw, Vw, Tw) - oracle.wall_ghost(Wm, Uw, Vw, Tw)) / (2 * h)
        assert np.allclose(M, J, rtol=1e-6, atol=1e-7), (M, J)


def test_wall_ghost_relation():
    # ghost density equals interior density, the mean velocity of interior and
    # ghost is the wall velocity, the mean lambda is the wall lambda
    W = np.array([1.2, 0.1, -0.05, 2.0])
    G = oracle.wall_ghost(W, 0.15, 0.0, 1.1)
    assert G[0] == W[0]
    assert abs(0.5 * (W[1] + G[1]) / W[0] - 0.15) < 1e-15
    assert abs(0.5 * (W[2] + G[2]) / W[0]) < 1e-15


# ---------------------------------------------------------------- transfer operators
def _golden(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return json.load(fh)


def test_prolongation_weights_printed_in_paper():
    gold = _golden("prolongation_weights.json")
    case = wl.cavity(n=8, nvel=4, levels=2)
    o = oracle.Oracle(case)
    ncx, ncy = o.level_size(1)
    nfx, nfy = o.level_size(0)

    def weights_of_fine_cell(i, j):
        out = {}
        for J in range(ncy):
            for I in range(ncx):
                e = np.zeros((ncx * ncy, 1))
                e[J * ncx + I] = 1.0
                val = o.prolong(0, e)[j * nfx + i, 0]
                if val != 0.0:
                    out[(I, J)] = val
        return out

    # inner cell: fine (3,3) lies in coarse A = (1,1), towards (2,2)
    w = weights_of_fine_cell(3, 3)
    assert sorted(w.values()) == sorted(gold["inner"].values())
    assert w[(1, 1)] == gold["inner"]["A"] and w[(2, 2)] == gold["inner"]["C"]
    # boundary cell: fine (0,3): A = (0,1), extrapolating in x
    w = weights_of_fine_cell(0, 3)
    assert w[(0, 1)] == gold["boundary"]["A"] and w[(1, 2)] == gold["boundary"]["C"]
    assert sorted(w.values()) == sorted(gold["boundary"].values())
    # corner cell: fine (0,0)
    w = weights_of_fine_cell(0, 0)
    assert w[(0, 0)] == gold["corner"]["A"] and w[(1, 1)] == gold["corner"]["C"]
    assert sorted(w.values()) == sorted(gold["corner"].values())


def test_transfer_accuracy_on_stretched_mesh():
    case = wl.flat_plate(nvel=4, levels=3, n_up=8, n_plate=8, n_down=8, ny=16)
    case["vgrid"].update(nu=4, nv=4)
    o = oracle.Oracle(case)
    xc = 0.5 * (case["x_nodes"][1:] + case["x_nodes"][:-1])
    yc = 0.5 * (case["y_nodes"][1:] + case["y_nodes"][:-1])
    X, Y = np.meshgrid(xc, yc)
    lin = (0.3 + 1.7 * X - 0.4 * Y).reshape(-1, 1)
    dx, dy = np.diff(case["x_nodes"]), np.diff(case["y_nodes"])
    V = np.outer(dy, dx).ravel()
    co = o.restrict(0, lin)
    Vc = np.outer(dy.reshape(-1, 2).sum(1), dx.reshape(-1, 2).sum(1)).ravel()
    # restriction conserves the volume integral and is second order (exact on linear fields)
    assert abs(np.dot(Vc, co[:, 0]) - np.dot(V, lin[:, 0])) < 1e-9 * np.dot(V, np.abs(lin[:, 0]))
    xn2, yn2 = case["x_nodes"][::2], case["y_nodes"][::2]
    Xc, Yc = np.meshgrid(0.5 * (xn2[1:] + xn2[:-1]), 0.5 * (yn2[1:] + yn2[:-1]))
    cen = (0.3 + 1.7 * Xc - 0.4 * Yc).ravel()
    # volume-weighted mean of a linear field = value at the cell centroid
    assert np.allclose(co[:, 0], cen, rtol=1e-12, atol=1e-10)
    # bilinear prolongation reproduces linear fields exactly (m_P = 2)
    back = o.prolong(0, cen.reshape(-1, 1))
    assert np.allclose(back[:, 0], lin[:, 0], rtol=1e-12, atol=1e-9)


# ---------------------------------------------------------------- Shakhov equilibrium
@pytest.mark.parametrize("rho,U,V,T,qx,qy,pr", [
    (1.3, 0.3, -0.2, 1.2, 0.05, -0.03, 2.0 / 3.0),
    (0.7, -0.45, 0.1, 0.8, -0.02, 0.04, 0.5),
    (2.0, 0.0, 0.25, 1.6, 0.1, 0.0, 2.0 / 3.0),
])
def test_shakhov_moments_and_heat_flux(rho, U, V, T, qx, qy, pr):
    """Sec. 2.1 names the Shakhov model as the one that gives the right Prandtl
    number.  Whatever its reduced form, two facts of the model are fixed by
    mathematics: the correction to the Maxwellian carries no mass, momentum or
    energy, and the heat flux of the equilibrium is (1 - Pr) q, so that
    relaxation toward it damps q at Pr times the rate of the stress.  On a wide,
    fine trapezoid grid (spectrally accurate for Gaussians) the discrete sums
    are the integrals to round-off.  A wrong polynomial in G+ fails the
    momentum check, a wrong one in H+ or a wrong prefactor fails the heat flux,
    and a peculiar velocity taken about 0 instead of (U, V) fails the mass
    check."""
    x, w1 = oracle.vgrid(101, -10.0, 10.0, 0)
    u = np.repeat(x, x.size)
    v = np.tile(x, x.size)
    w = np.outer(w1, w1).ravel()
    lam = 1.0 / T
    G, H = oracle.shakhov(rho, U, V, lam, qx, qy, pr, u, v)
    cx, cy = u - U, v - V
    c2 = cx * cx + cy * cy
    GM = rho * lam / math.pi * np.exp(-lam * c2)
    HM = GM / (4.0 * lam)                       # one internal degree of freedom
    tol = 1e-12
    # conservative moments: those of the Maxwellian, rho eps = rho |U|^2/2 + 3 rho/(4 lam)
    mom = [np.dot(w, G), np.dot(w, u * G), np.dot(w, v * G), np.dot(w, 0.5 * (u * u + v * v) * G + H)]
    exact = [rho, rho * U, rho * V, 0.5 * rho * (U * U + V * V) + 3.0 * rho / (4.0 * lam)]
    for a, b in zip(mom, exact):
        assert abs(a - b) < tol * max(1.0, abs(b)), (mom, exact)
    # the correction alone: zero mass, momentum, energy and second moments (it is odd in c)
    dG, dH = G - GM, H - HM
    for psi in (np.ones_like(u), u, v, cx * cx, cx * cy):
        assert abs(np.dot(w, psi * dG)) < tol
    assert abs(np.dot(w, 0.5 * (u * u + v * v) * dG + dH)) < tol
    # heat flux of the equilibrium: (1 - Pr) q
    q = [np.dot(w, cx * (0.5 * c2 * G + H)), np.dot(w, cy * (0.5 * c2 * G + H))]
    assert abs(q[0] - (1.0 - pr) * qx) < tol and abs(q[1] - (1.0 - pr) * qy) < tol, (q, qx, qy)


def test_shakhov_reduces_to_maxwellian():
    """With Pr = 1 or q = 0 the Shakhov equilibrium is the reduced Maxwellian
    G_M = rho (lam/pi) exp(-lam |c|^2), H_M = G_M K_int / (4 lam)."""
    x, _ = oracle.vgrid(24, -5.0, 5.0, 0)
    u, v = np.repeat(x, x.size), np.tile(x, x.size)
    rho, U, V, lam = 1.1, 0.2, -0.1, 0.9
    GM = rho * lam / math.pi * np.exp(-lam * ((u - U) ** 2 + (v - V) ** 2))
    for qx, qy, pr in ((0.3, -0.2, 1.0), (0.0, 0.0, 2.0 / 3.0)):
        G, H = oracle.shakhov(rho, U, V, lam, qx, qy, pr, u, v)
        assert np.allclose(G, GM, rtol=1e-14, atol=0)
        assert np.allclose(H, GM / (4.0 * lam), rtol=1e-14, atol=0)


# ---------------------------------------------------------------- shock capturing (off by default)
def test_pressure_jump_collision_time_only_acts_on_pressure_jumps():
    """The pressure-jump term dt |p_L - p_R| / (p_L + p_R) of the interface
    collision time (the paper is silent; the gas-kinetic schemes' shock
    capturing) vanishes where the two cells have the same pressure: with
    density and temperature uniform and the velocity varying, every face flux
    is the same with the option on (to the rounding of the cell pressures);
    with a pressure jump the faces across it change and the others do not."""
    # 40 nodes on [-6, 6]: the discrete moments of each cell's Maxwellian are its (rho, U, V, T) to
    # round-off, so cells of equal density and temperature have equal pressure
    case = wl.cavity(n=8, nvel=40, vmax=6.0, kn=0.01, lid=0.2, levels=1)
    nx = ny = 8
    rng = np.random.default_rng(5)
    rho, t = np.full(nx * ny, 1.2), np.full(nx * ny, 0.9)
    u, v = 0.1 * rng.uniform(-1, 1, nx * ny), 0.1 * rng.uniform(-1, 1, nx * ny)
    out = {}
    for on in (False, True):
        o = oracle.Oracle(case)
        o.set_shock_capturing(on)
        o.init_fields(rho, u, v, t)
        out[on] = o.stage_flux()
    for a, b in zip(out[False], out[True]):           # pressures equal up to the rounding of W
        assert np.allclose(a, b, rtol=1e-12, atol=1e-14 * np.abs(a).max())
    # a pressure jump across the x-faces between columns 3 and 4
    rho2 = rho.reshape(ny, nx).copy()
    rho2[:, 4:] *= 1.5
    for on in (False, True):
        o = oracle.Oracle(case)
        o.set_shock_capturing(on)
        o.init_fields(rho2.ravel(), u, v, t)
        out[on] = o.stage_flux()
    px0, px1 = out[False][1], out[True][1]          # [2][nfx][nv], x-face index j * (nx + 1) + i
    d = (np.abs(px1 - px0).max(axis=(0, 2)) / np.abs(px0).max()).reshape(ny, nx + 1)
    assert np.all(d[:, 4] > 1e-4) and np.all(np.delete(d, 4, axis=1) < 1e-12), d
    with pytest.raises(RuntimeError):
        o.steady_residual()
