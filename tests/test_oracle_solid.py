"""Pins of the oracle's solid cells (bodies inside the mesh, the square
cylinder of Sec. 4.3): a body is a block of cells with no state whose faces
with the fluid are boundary faces.  Pinned by (a) equivalence: a solid strip
along one edge of a cavity gives the smaller cavity exactly, for every
orientation of the wall and with multigrid; (b) conservation and the rest
Maxwellian fixed point around an interior body (I1, I2); (c) the
serial-vs-wavefront identity of the sweeps with a body (I4); (d) the
prolongation reproducing linear fields next to a body."""
import numpy as np
import pytest

import oracle
from paper_1704_03151_gb300 import workloads as wl


def _strip_case(side, n_fluid=(12, 8), n_strip=4, levels=1, nvel=8):
    """Cavity of n_fluid cells (spacing 1/12 x 1/8) with a solid strip of
    n_strip cells added on `side`; its fluid part is wl.cavity(nx, ny)."""
    nxf, nyf = n_fluid
    base = wl.cavity(nx=nxf, ny=nyf, nvel=nvel, kn=0.5, lid=0.25, levels=levels)
    hx, hy = 1.0 / nxf, 1.0 / nyf
    nx, ny = nxf, nyf
    x = np.asarray(base["x_nodes"]).copy()
    y = np.asarray(base["y_nodes"]).copy()
    off_x = off_y = 0
    if side == "east":
        nx += n_strip
        x = np.concatenate([x, 1.0 + hx * np.arange(1, n_strip + 1)])
    elif side == "west":
        nx += n_strip
        off_x = n_strip
        x = np.concatenate([-hx * np.arange(n_strip, 0, -1), x])
    elif side == "north":
        ny += n_strip
        y = np.concatenate([y, 1.0 + hy * np.arange(1, n_strip + 1)])
    else:
        ny += n_strip
        off_y = n_strip
        y = np.concatenate([-hy * np.arange(n_strip, 0, -1), y])
    solid = np.ones((ny, nx), dtype=np.uint8)
    solid[off_y:off_y + nyf, off_x:off_x + nxf] = 0
    # edges of the big rectangle carry the cavity's ids; the fluid-solid faces
    # take the id of the cavity wall they replace
    wall_id = {"south": 0, "east": 1, "north": 2, "west": 3}[side]
    fbx, fby = wl.edge_face_ids(nx, ny, 3, 1, 0, 2)
    fbx, fby = wl.body_face_ids(solid, fbx, fby, wall_id)
    case = dict(base, nx=nx, ny=ny, x_nodes=x, y_nodes=y, face_bc_x=fbx, face_bc_y=fby, solid=solid.ravel())
    return base, case, (off_x, off_y)


def _fluid(big, small, off, field):
    nx, ny = big["nx"], big["ny"]
    ox, oy = off
    return field.reshape(ny, nx, -1)[oy:oy + small["ny"], ox:ox + small["nx"]].reshape(small["ny"] * small["nx"], -1)


@pytest.mark.parametrize("levels", [1, 2])
@pytest.mark.parametrize("side", ["east", "west", "north", "south"])
def test_solid_strip_equals_smaller_cavity(side, levels):
    small, big, off = _strip_case(side, levels=levels)
    a, b = oracle.Oracle(small), oracle.Oracle(big)
    fs = wl.random_fields(small, 5)
    fb = [np.ones(big["nx"] * big["ny"]) for _ in range(4)]
    for q in range(4):
        fb[q][:] = 1.0 if q in (0, 3) else 0.0
        fb[q].reshape(big["ny"], big["nx"])[off[1]:off[1] + small["ny"], off[0]:off[0] + small["nx"]] = \
            fs[q].reshape(small["ny"], small["nx"])
    a.init_fields(*fs)
    b.init_fields(*fb)
    for _ in range(3):
        ra, rb = a.step(1), b.step(1)
        np.testing.assert_allclose(rb, ra, rtol=1e-12, atol=1e-15)
    ma, mb = a.macro(), b.macro()
    for k in ma:
        qb = _fluid(big, small, off, mb[k].reshape(-1, 1))[:, 0]
        np.testing.assert_allclose(qb, ma[k], rtol=1e-12, atol=1e-14)
    wa = a.wall({"south": 0, "east": 1, "north": 2, "west": 3}[side])
    wb = b.wall({"south": 0, "east": 1, "north": 2, "west": 3}[side])
    for qa, qb in zip(wa, wb):
        np.testing.assert_allclose(qb, qa, rtol=1e-12, atol=1e-14)


def _box_with_body(n=16, body=(6, 10, 6, 10), nvel=12, lid=0.3, levels=2, vmax=4.0):
    case = wl.cavity(n=n, nvel=nvel, kn=0.5, lid=lid, levels=levels, vmax=vmax)
    solid = np.zeros((n, n), dtype=np.uint8)
    i0, i1, j0, j1 = body
    solid[j0:j1, i0:i1] = 1
    case["bcs"] = case["bcs"] + [wl.bc(wl.WALL, t=1.0)]
    fbx, fby = wl.body_face_ids(solid, case["face_bc_x"], case["face_bc_y"], len(case["bcs"]) - 1)
    return dict(case, face_bc_x=fbx, face_bc_y=fby, solid=solid.ravel())


def test_mass_conservation_around_a_body():
    case = _box_with_body()
    o = oracle.Oracle(case)
    o.init_fields(*wl.random_fields(case, 3))
    V = np.full(case["nx"] * case["ny"], 1.0 / (case["nx"] * case["ny"]))
    solid = case["solid"].astype(bool)
    for _ in range(3):
        R = o.residual()
        assert np.all(R[solid] == 0.0)
        assert abs(np.dot(V, R[:, 0])) < 1e-14 * np.abs(R[:, 0]).max() * len(V) + 1e-16
        o.step(1)


def test_rest_maxwellian_with_a_body_is_a_fixed_point():
    case = _box_with_body(n=8, body=(2, 6, 4, 6), nvel=28, lid=0.0, vmax=7.0)
    o = oracle.Oracle(case)
    o.init_uniform(1.0, 0.0, 0.0, 1.0)
    f0 = o.get_f()
    res = o.step(2)
    assert np.all(res < 1e-13), res
    f1 = o.get_f()
    assert np.max(np.abs(f1 - f0)) < 1e-13 * np.max(np.abs(f0))


def test_sweep_wavefront_order_matches_serial_with_a_body():
    case = _box_with_body(n=12, body=(4, 8, 2, 6), nvel=8, levels=1)
    o = oracle.Oracle(case)
    o.init_fields(*wl.random_fields(case, 9))
    rng = np.random.default_rng(4)
    nc, nv = case["nx"] * case["ny"], o.nv
    r = rng.standard_normal((2, nc, nv))
    r[:, case["solid"].astype(bool)] = 0.0
    it = 1.0 + rng.random(nc)
    x0 = o.sgs_micro(0, it, r, order=0)
    x1 = o.sgs_micro(0, it, r, order=1)
    assert np.array_equal(x0, x1)
    assert np.all(x0[:, case["solid"].astype(bool)] == 0.0)
    W = np.tile([1.0, 0.1, -0.05, 0.8], (nc, 1)) + 0.01 * rng.standard_normal((nc, 4))
    R = 0.01 * rng.standard_normal((nc, 4))
    R[case["solid"].astype(bool)] = 0.0
    d0 = o.sgs_macro(0, W, W, R, order=0)
    d1 = o.sgs_macro(0, W, W, R, order=1)
    assert np.array_equal(d0, d1)


def test_prolongation_reproduces_linear_fields_next_to_a_body():
    case = _box_with_body(n=16, body=(4, 8, 8, 12), levels=2)
    x = np.linspace(0, 1, 17)
    case["x_nodes"] = x ** 1.3   # stretched, so the weights are not the uniform ones
    o = oracle.Oracle(case)
    xc = 0.5 * (case["x_nodes"][1:] + case["x_nodes"][:-1])
    yc = 0.5 * (case["y_nodes"][1:] + case["y_nodes"][:-1])
    # coarse centres are the centres of the coarse cells (every second grid line)
    xn = case["x_nodes"]
    Xc = 0.5 * (xn[0:-1:2] + xn[2::2])
    yn = case["y_nodes"]
    Yc = 0.5 * (yn[0:-1:2] + yn[2::2])
    lin = lambda X, Y: 0.3 + 1.7 * X - 0.9 * Y
    XX, YY = np.meshgrid(Xc, Yc)
    coarse = lin(XX, YY).reshape(-1, 1)
    fine = o.prolong(0, coarse)
    FX, FY = np.meshgrid(xc, yc)
    want = lin(FX, FY).reshape(-1)
    solid = case["solid"].astype(bool)
    np.testing.assert_allclose(fine[~solid, 0], want[~solid], rtol=0, atol=1e-13)
    assert np.all(fine[solid] == 0.0)


def test_body_faces_need_boundary_ids():
    case = _box_with_body(n=8, body=(2, 6, 2, 6), levels=1)
    fbx = np.array(case["face_bc_x"]).reshape(8, 9)
    fbx[3, 2] = -1
    with pytest.raises(RuntimeError, match="x-face"):
        oracle.Oracle(dict(case, face_bc_x=fbx.ravel()))
    case2 = _box_with_body(n=8, body=(1, 5, 2, 6), levels=2)
    with pytest.raises(RuntimeError, match="whole coarse cells"):
        oracle.Oracle(case2)


def test_hypersonic_square_start_stays_physical():
    """Ma 5 past the square from the rear-region start (Sec. 4.3) on a small
    two-level mesh: the first FAS correction overshoots at the shock (negative
    internal energy in about a dozen fine cells); dropping the correction
    there keeps every state physical and the iteration going."""
    case = wl.square_cylinder(nx_side=4, nx_sq=4, ny_side=4, ny_sq=4, levels=2, nvel=89, dtn_growth=3.0)
    o = oracle.Oracle(case)
    o.init_fields(*wl.initial_fields(case))
    res = [o.step(1) for _ in range(3)]
    assert all(np.all(np.isfinite(r)) for r in res)
    assert max(res[-1]) < max(res[0])
    m = o.macro()
    fluid = ~case["solid"].astype(bool)
    assert np.all(m["rho"][fluid] > 0) and np.all(m["t"][fluid] > 0)


def test_fmg_start_falls_back_where_prolongation_is_unphysical():
    """After the coarse mesh has formed the Ma 5 bow shock, the bilinear
    extrapolation of f at the domain edge gives negative temperatures; those
    cells take their coarse cell's f and every fine state is physical."""
    case = wl.square_cylinder(nx_side=4, nx_sq=4, ny_side=4, ny_sq=4, levels=2, nvel=89, dtn_growth=3.0)
    coarse = wl.coarsen_case(case)
    oc = oracle.Oracle(coarse)
    oc.init_fields(*wl.initial_fields(coarse))
    oc.step(40)
    o = oracle.Oracle(case)
    o.init_from_coarse(oc)
    m = o.macro()
    fluid = ~case["solid"].astype(bool)
    assert np.all(m["rho"][fluid] > 0) and np.all(m["t"][fluid] > 0)
    r = o.step(2)
    assert np.all(np.isfinite(r))


def test_flow_around_a_centred_body_is_mirror_symmetric():
    """I5 around a body: subsonic flow past a square centred in y between
    farfield edges reaches a state symmetric about the centre line (rho, u,
    T even, v odd) once the residual has stopped falling; the sweep order
    breaks the symmetry only at the level of that floor."""
    case = wl.square_cylinder(ma=0.5, kn=0.5, nvel=12, vmax=4.0, levels=2, nx_side=4, nx_sq=4, ny_side=4,
                              ny_sq=4, half=2.0, dtn_growth=0.0)
    case["rear"] = None
    o = oracle.Oracle(case)
    o.init_fields(*wl.initial_fields(case))
    r = o.step(400)
    assert max(r) < 1e-5
    m = o.macro()
    ny, nx = case["ny"], case["nx"]
    for k, sign in (("rho", 1), ("u", 1), ("v", -1), ("t", 1)):
        a = m[k].reshape(ny, nx)
        assert np.abs(a - sign * a[::-1, :]).max() < 1e-5 * np.abs(a).max(), k
