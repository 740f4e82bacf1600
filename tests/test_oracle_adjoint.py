"""Pins of the oracle's adjoint of the steady equations (the differentiation
form of the method): the derivative of each building block against a
high-precision or finite-difference derivative, the transposed Jacobian of the
steady residual by dot-product tests against central differences of the
residual itself, and the whole adjoint gradient against central differences of
fully converged forward solves (open domain: plain; closed cavity: at fixed
total mass, each perturbed state polished onto the fixed-mass steady
manifold by Newton steps with the assembled Jacobian)."""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_1704_03151_gb300 import workloads as wl


def test_time_integral_derivatives_against_high_precision():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50

    def qs(dt, tau):
        x = dt / tau
        e = mp.e ** (-x)
        E1 = 1 - e
        return [dt - tau * E1, -tau * dt * (1 + e) + 2 * tau ** 2 * E1, dt ** 2 / 2 - tau * dt + tau ** 2 * E1,
                tau * E1, tau * dt * e - tau ** 2 * E1]

    for x in (1e-4, 1e-2, 0.3, 0.999, 1.001, 3.0, 40.0):
        dt = mp.mpf("0.7")
        tau = dt / x
        exact = [mp.diff(lambda t, m=m: qs(dt, t)[m], tau) for m in range(5)]
        got = oracle.time_coeffs_dtau(float(dt), float(tau))
        for m in range(5):
            assert abs(got[m] - float(exact[m])) <= 1e-13 * abs(float(exact[m])), (x, m)


def test_micro_slope_reverse_dot_product():
    rng = np.random.default_rng(4)
    for _ in range(5):
        dw, U, V, lam = rng.normal(size=4), rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5), rng.uniform(0.5, 2)
        ab, d = rng.normal(size=4), rng.normal(size=7)
        dwb, pb = oracle.micro_slope_adj(dw, U, V, lam, ab)
        z0 = np.r_[dw, U, V, lam]
        F = lambda z: np.dot(ab, oracle.micro_slope(z[:4], z[4], z[5], z[6]))
        h = 1e-6
        fd = (F(z0 + h * d) - F(z0 - h * d)) / (2 * h)
        assert abs(fd - np.dot(np.r_[dwb, pb], d)) < 1e-7 * max(1.0, abs(fd))


def _stretched_cavity():
    case = wl.cavity(nx=6, ny=5, nvel=8, kn=0.7, lid=0.3, levels=1)
    case["x_nodes"] = wl.geometric_nodes(0.0, 1.0, 6, 0.1)
    return case


def _open_box():
    """Wall below, farfield above, symmetry on the left, outflow on the right."""
    nx, ny = 5, 4
    fbx, fby = wl.edge_face_ids(nx, ny, 2, 3, 0, 1)
    case = wl.couette(n=ny, nx=nx, nvel=8, kn=0.4)
    case["face_bc_x"], case["face_bc_y"] = fbx, fby
    case["y_nodes"] = wl.geometric_nodes(0.0, 1.0, ny, 0.15)
    case["bcs"] = [wl.bc(wl.WALL, u=0.2, t=1.1), wl.bc(wl.FARFIELD, rho=1.0, u=0.3, v=-0.1, t=1.0),
                   wl.bc(wl.SYMMETRY), wl.bc(wl.OUTFLOW)]
    case["init"] = {"rho": 1.0, "u": 0.2, "v": 0.0, "t": 1.0}
    return case


@pytest.mark.parametrize("make", [_stretched_cavity, _open_box])
def test_adjoint_residual_dot_product(make):
    """<mu, dN/df v> by central differences of N equals <(dN/df)^T mu, v>.
    Directions whose difference quotient is not converged in the step (it
    crossed a kink of the van Leer limiter) are skipped."""
    case = make()
    o = oracle.Oracle(case)
    o.init_fields(*wl.random_fields(case, 3, amp=0.1))
    rng = np.random.default_rng(7)
    f = o.get_f() * (1 + 0.03 * rng.uniform(-1, 1, size=(2, o.nc, o.nv)))
    o.set_f(f)
    mu = rng.normal(size=f.shape)
    out = o.adjoint_residual(mu)

    def dd(v, h):
        o.set_f(f + h * v)
        Np = o.steady_residual()
        o.set_f(f - h * v)
        Nm = o.steady_residual()
        o.set_f(f)
        return np.sum(mu * (Np - Nm)) / (2 * h)

    checked = 0
    for trial in range(12):
        v = rng.normal(size=f.shape) * f
        if trial % 3 == 1:        # one cell at a time, to catch index mistakes
            c = rng.integers(o.nc)
            mask = np.zeros(o.nc)
            mask[c] = 1.0
            v = v * mask[None, :, None]
        a, b = dd(v, 1e-6), dd(v, 4e-7)
        if abs(a - b) > 1e-8 * max(1.0, abs(a)):
            continue
        assert abs(a - np.sum(out * v)) < 1e-7 * max(1.0, abs(a)), trial
        checked += 1
    assert checked >= 6


def _tiny_velocity(o, f, scale):
    """f with one velocity (the largest u > 0: k = a nv_y + b with a the last
    u node) replaced in every cell by scale x a profile that grows along x, so
    that its van Leer slopes at the x-faces all have one sign and are of the
    order of scale (both components)."""
    nvv = int(round(np.sqrt(o.nv)))
    k0 = (nvv - 1) * nvv + nvv // 2
    g = f.copy()
    ix = np.arange(o.nc) % o.nx
    for cp in range(2):
        g[cp, :, k0] = scale * (1.0 + 0.2 * ix) * (1 + cp)
    return g


def test_adjoint_residual_stays_finite_for_slopes_near_underflow():
    """The derivative of the van Leer slope 2 s1 s2 / (s1 + s2) is
    2 (s2 / (s1 + s2))^2 (and symmetrically): it depends on the slopes' ratio
    only.  So a velocity whose values (and slopes) sit near the underflow
    threshold of FP64, as in the far tails of a wide velocity grid at Ma 5,
    gives the same transposed Jacobian as the same profile scaled to 1e-150
    (where nothing underflows), to the 1e-150 change of the moments, and no
    Inf or NaN."""
    case = _stretched_cavity()
    o = oracle.Oracle(case)
    o.init_fields(*wl.random_fields(case, 5, amp=0.1))
    f = o.get_f()
    mu = np.random.default_rng(2).normal(size=f.shape)
    outs = []
    for scale in (1e-150, 1e-158):
        o.set_f(_tiny_velocity(o, f, scale))
        outs.append(o.adjoint_residual(mu))
    assert np.all(np.isfinite(outs[1]))
    assert np.max(np.abs(outs[1] - outs[0])) <= 1e-12 * np.max(np.abs(outs[0]))


def test_objective_and_parameter_derivatives():
    case = _stretched_cavity()
    o = oracle.Oracle(case)
    o.init_fields(*wl.random_fields(case, 5, amp=0.1))
    o.step(2)
    f = o.get_f()
    rng = np.random.default_rng(1)
    b = case["bcs"][2]
    for obj in (0, 1, 2):
        J, dJdf, dJdth = o.objective(obj, 2)
        p, tau, q = o.wall(2)
        S = np.diff(case["x_nodes"])
        assert J == pytest.approx(np.dot(S, (tau, q, p)[obj]), rel=1e-13, abs=1e-15)
        v = rng.normal(size=f.shape) * f
        h = 1e-6
        o.set_f(f + h * v)
        Jp = o.objective(obj, 2)[0]
        o.set_f(f - h * v)
        Jm = o.objective(obj, 2)[0]
        o.set_f(f)
        assert (Jp - Jm) / (2 * h) == pytest.approx(np.sum(dJdf * v), rel=1e-7, abs=1e-10)
        for param, key in enumerate(("t", "u", "v")):
            vals = dict(b)
            hh = 1e-6
            vals[key] = b[key] + hh
            o.set_bc(2, vals["rho"], vals["u"], vals["v"], vals["t"])
            Jp = o.objective(obj, 2)[0]
            vals[key] = b[key] - hh
            o.set_bc(2, vals["rho"], vals["u"], vals["v"], vals["t"])
            Jm = o.objective(obj, 2)[0]
            o.set_bc(2, b["rho"], b["u"], b["v"], b["t"])
            assert (Jp - Jm) / (2 * hh) == pytest.approx(dJdth[param], rel=1e-7, abs=1e-10), (obj, key)


def test_residual_parameter_derivative():
    case = _stretched_cavity()
    o = oracle.Oracle(case)
    o.init_fields(*wl.random_fields(case, 6, amp=0.1))
    o.step(1)
    b = case["bcs"][2]
    for param, key in enumerate(("t", "u", "v")):
        dN = o.residual_dtheta(2, param)
        vals = dict(b)
        h = 1e-6
        vals[key] = b[key] + h
        o.set_bc(2, vals["rho"], vals["u"], vals["v"], vals["t"])
        Np = o.steady_residual()
        vals[key] = b[key] - h
        o.set_bc(2, vals["rho"], vals["u"], vals["v"], vals["t"])
        Nm = o.steady_residual()
        o.set_bc(2, b["rho"], b["u"], b["v"], b["t"])
        fd = (Np - Nm) / (2 * h)
        assert np.max(np.abs(fd - dN)) < 1e-7 * np.max(np.abs(dN)), key


def _channel(dt=0.0, du=0.0):
    """Open channel: moving, heated wall below, farfield above, symmetry sides."""
    c = wl.couette(n=3, nx=3, nvel=16, kn=1.0, vmax=5.0, t_bottom=1.0 + dt, t_top=1.0, u_top=0.0)
    c["bcs"][0]["u"] = 0.2 + du
    c["bcs"][1] = wl.bc(wl.FARFIELD, rho=1.0, u=0.0, v=0.0, t=1.2)
    return c


def _converged(case, iters=300):
    o = oracle.Oracle(case)
    o.init_uniform(1.0, 0.0, 0.0, 1.0)
    o.step(iters)
    return o


def test_adjoint_gradient_matches_converged_differences_open_channel():
    o = _converged(_channel())
    assert np.abs(o.steady_residual()).max() < 1e-9
    A = oracle.adjoint_matrix(o)
    for obj, param, h in ((0, 1, 1e-4), (0, 0, 1e-5), (1, 0, 1e-5), (2, 0, 1e-5)):
        g, _ = oracle.adjoint_gradient(o, obj, 0, param, A=A)
        kw = (lambda s: {"dt": s * h}) if param == 0 else (lambda s: {"du": s * h})
        fd = (_converged(_channel(**kw(1))).objective(obj, 0)[0] -
              _converged(_channel(**kw(-1))).objective(obj, 0)[0]) / (2 * h)
        assert g == pytest.approx(fd, rel=2e-6), (obj, param)


def test_adjoint_gradient_matches_fixed_mass_differences_closed_cavity():
    def cav(dt=0.0, du=0.0):
        c = wl.cavity(nx=3, ny=3, nvel=16, kn=1.0, lid=0.2 + du, levels=1, vmax=5.0)
        c["bcs"][2]["t"] = 1.0 + dt
        return c

    o = _converged(cav(), 200)
    A = oracle.adjoint_matrix(o)
    m = oracle.mass_weights(o).ravel()
    M0 = float(m @ o.get_f().ravel())
    n = m.size
    lu = sla.lu_factor(np.block([[A.T, m[:, None]], [m[None, :], np.zeros((1, 1))]]))

    def polish(op):
        """Chord-Newton onto N(f) + s m = 0, M(f) = M0 (Jacobian of the base state)."""
        s = 0.0
        for _ in range(20):
            f = op.get_f().ravel()
            r = np.r_[op.steady_residual().ravel() + s * m, m @ f - M0]
            d = sla.lu_solve(lu, -r)
            op.set_f((f + d[:n]).reshape(2, op.nc, op.nv))
            s += d[n]
        return np.abs(r).max()

    assert polish(o) < 1e-13
    for obj, param, h in ((0, 1, 1e-4), (1, 0, 1e-5), (2, 0, 1e-5)):
        g, _ = oracle.adjoint_gradient(o, obj, 2, param, A=A)
        kw = (lambda s: {"dt": s * h}) if param == 0 else (lambda s: {"du": s * h})
        Js = []
        for sg in (1, -1):
            op = _converged(cav(**kw(sg)), 200)
            assert polish(op) < 1e-11
            Js.append(op.objective(obj, 2)[0])
        assert g == pytest.approx((Js[0] - Js[1]) / (2 * h), rel=2e-6), (obj, param)


def _body_box(dt=0.0):
    """A 3x3 box with a one-cell body at its centre (the square cylinder of
    Sec. 4.3 in miniature): isothermal wall on the body (BC 0, T_w = 1 + dt),
    farfield inflow, top and bottom (BC 1), zero-gradient outflow (BC 2).  16
    velocities per axis on [-5, 5] keep the discrete moments of the Maxwellians
    exact to ~1e-10, so the iteration's fixed point solves N = 0 to that level."""
    c = wl.square_cylinder(ma=0.5, kn=1.0, nvel=16, vmax=5.0, levels=1, nx_side=1, nx_sq=1, ny_side=1, ny_sq=1,
                           half=1.5, dtn_growth=0.0)
    c["bcs"][0]["t"] = 1.0 + dt
    c.pop("rear")
    return c


def test_adjoint_residual_dot_product_with_a_body():
    """As test_adjoint_residual_dot_product, around a body: its faces are wall
    faces of the fluid cells beside it, and a cell in the body holds no state
    (N = -f there keeps the Jacobian regular)."""
    test_adjoint_residual_dot_product(_body_box)


def test_objective_and_parameter_derivatives_on_a_body_wall():
    case = _body_box()
    o = oracle.Oracle(case)
    o.init_fields(*wl.random_fields(case, 5, amp=0.1))
    o.step(2)
    f = o.get_f()
    rng = np.random.default_rng(2)
    b = case["bcs"][0]
    for obj in (0, 1, 2):
        J, dJdf, dJdth = o.objective(obj, 0)
        p, tau, q = o.wall(0)
        assert len(q) == 4                       # the four faces of the body
        v = rng.normal(size=f.shape) * f
        h = 1e-6
        o.set_f(f + h * v)
        Jp = o.objective(obj, 0)[0]
        o.set_f(f - h * v)
        Jm = o.objective(obj, 0)[0]
        o.set_f(f)
        assert (Jp - Jm) / (2 * h) == pytest.approx(np.sum(dJdf * v), rel=1e-7, abs=1e-10)
        for param, key in enumerate(("t", "u", "v")):
            vals = dict(b)
            vals[key] = b[key] + h
            o.set_bc(0, vals["rho"], vals["u"], vals["v"], vals["t"])
            Jp = o.objective(obj, 0)[0]
            vals[key] = b[key] - h
            o.set_bc(0, vals["rho"], vals["u"], vals["v"], vals["t"])
            Jm = o.objective(obj, 0)[0]
            o.set_bc(0, b["rho"], b["u"], b["v"], b["t"])
            assert (Jp - Jm) / (2 * h) == pytest.approx(dJdth[param], rel=1e-7, abs=1e-9), (obj, key)
    for param, key in enumerate(("t", "u", "v")):
        dN = o.residual_dtheta(0, param)
        vals = dict(b)
        vals[key] = b[key] + h
        o.set_bc(0, vals["rho"], vals["u"], vals["v"], vals["t"])
        Np = o.steady_residual()
        vals[key] = b[key] - h
        o.set_bc(0, vals["rho"], vals["u"], vals["v"], vals["t"])
        Nm = o.steady_residual()
        o.set_bc(0, b["rho"], b["u"], b["v"], b["t"])
        assert np.max(np.abs((Np - Nm) / (2 * h) - dN)) < 1e-7 * np.max(np.abs(dN)), key


def test_adjoint_gradient_around_a_body_matches_converged_differences():
    """d(heat flux into the body)/d(body wall temperature) and the shear and
    pressure gradients: the adjoint against central differences of fully
    converged forward solves (the open box fixes the state without a mass
    constraint)."""
    def conv(dt):
        o = oracle.Oracle(_body_box(dt))
        c = o.case
        o.init_uniform(1.0, c["init"]["u"], 0.0, 1.0)
        o.step(300)
        return o

    o = conv(0.0)
    fluid = ~np.asarray(o.case["solid"]).astype(bool)
    assert np.abs(o.steady_residual()[:, fluid]).max() < 1e-9
    A = oracle.adjoint_matrix(o)
    h = 1e-5
    op, om = conv(h), conv(-h)
    for obj in (1, 0, 2):
        g, _ = oracle.adjoint_gradient(o, obj, 0, 0, A=A)
        fd = (op.objective(obj, 0)[0] - om.objective(obj, 0)[0]) / (2 * h)
        assert g == pytest.approx(fd, rel=2e-6), obj
