"""Seeded synthetic problem set-ups shared by the tests, the benchmark and the
smoke check.

This module only builds inputs -- mesh node coordinates, face boundary ids,
boundary-condition tables, velocity-grid / gas / multigrid parameters and
initial fields.  It holds none of the scheme's arithmetic.  The problems follow
the test cases of the paper (Sec. 4): the lid-driven cavity (Sec. 4.1), the
flat plate (Sec. 4.2); units are nondimensional with R = 1/2, reference
density, temperature and length 1 (most probable speed 1).
"""
import math

import numpy as np

WALL, SYMMETRY, FARFIELD, OUTFLOW = 0, 1, 2, 3
TRAPEZOID, BOOLE = 0, 1


def bc(type_, rho=1.0, u=0.0, v=0.0, t=1.0):
    return {"type": int(type_), "rho": float(rho), "u": float(u), "v": float(v), "t": float(t)}


def edge_face_ids(nx, ny, west, east, south, north):
    """Face BC id arrays for a rectangle whose four edges carry the given ids
    (scalars or per-face arrays); interior faces get -1."""
    fbx = -np.ones((ny, nx + 1), dtype=np.int32)
    fby = -np.ones((ny + 1, nx), dtype=np.int32)
    fbx[:, 0] = west
    fbx[:, nx] = east
    fby[0, :] = south
    fby[ny, :] = north
    return fbx.ravel(), fby.ravel()


def cavity(n=24, nvel=20, kn=1.0, lid=0.16, levels=1, vmax=4.0, omega=0.81, pr=2.0 / 3.0,
           nu1=2, nu2=1, nuc=4, cfl=0.8, rule=TRAPEZOID, t_wall=1.0, nx=None, ny=None):
    """Lid-driven cavity on [0,1]^2 (Sec. 4.1): diffuse isothermal walls, the
    top wall moving with speed `lid`; BC ids 0 south, 1 east, 2 north (lid),
    3 west."""
    nx = nx or n
    ny = ny or n
    fbx, fby = edge_face_ids(nx, ny, 3, 1, 0, 2)
    return {
        "name": "cavity%dx%d_v%d_kn%g_L%d" % (nx, ny, nvel, kn, levels),
        "nx": nx, "ny": ny,
        "x_nodes": np.linspace(0.0, 1.0, nx + 1), "y_nodes": np.linspace(0.0, 1.0, ny + 1),
        "face_bc_x": fbx, "face_bc_y": fby,
        "bcs": [bc(WALL, t=t_wall), bc(WALL, t=t_wall), bc(WALL, u=lid, t=t_wall), bc(WALL, t=t_wall)],
        "vgrid": {"nu": nvel, "nv": nvel, "umin": -vmax, "umax": vmax, "vmin": -vmax, "vmax": vmax, "rule": rule},
        "gas": {"kn": kn, "omega": omega, "pr": pr},
        "mg": {"levels": levels, "nu1": nu1, "nu2": nu2, "nuc": nuc, "cfl": cfl, "dtn_growth": 0.0},
        "init": {"rho": 1.0, "u": 0.0, "v": 0.0, "t": 1.0},
    }


def couette(n=8, nvel=16, kn=1e6, t_bottom=1.0, t_top=1.5, u_top=0.2, vmax=4.0, levels=1, nx=None):
    """Plane Couette / Fourier flow between two diffuse walls (bottom y=0,
    top y=1) with symmetry planes on the left and right; BC ids 0 bottom,
    1 top, 2 symmetry."""
    nx = nx or n
    fbx, fby = edge_face_ids(nx, n, 2, 2, 0, 1)
    return {
        "name": "couette%d_kn%g" % (n, kn),
        "nx": nx, "ny": n,
        "x_nodes": np.linspace(0.0, 1.0, nx + 1), "y_nodes": np.linspace(0.0, 1.0, n + 1),
        "face_bc_x": fbx, "face_bc_y": fby,
        "bcs": [bc(WALL, t=t_bottom), bc(WALL, u=u_top, t=t_top), bc(SYMMETRY)],
        "vgrid": {"nu": nvel, "nv": nvel, "umin": -vmax, "umax": vmax, "vmin": -vmax, "vmax": vmax,
                  "rule": TRAPEZOID},
        "gas": {"kn": kn, "omega": 0.81, "pr": 2.0 / 3.0},
        "mg": {"levels": levels, "nu1": 2, "nu2": 1, "nuc": 4, "cfl": 0.8, "dtn_growth": 0.0},
        "init": {"rho": 1.0, "u": 0.0, "v": 0.0, "t": 1.0},
    }


def geometric_nodes(x0, x1, n, h_first, at_start=True):
    """n cells on [x0, x1] whose widths grow geometrically away from one end,
    the first cell of width h_first (ratio found by bisection)."""
    L = x1 - x0
    if abs(n * h_first - L) < 1e-14 * L:
        r = 1.0
    else:
        lo, hi = 1.0 + 1e-12, 2.0
        while h_first * (hi ** n - 1) / (hi - 1) < L:
            hi *= 2
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if h_first * (mid ** n - 1) / (mid - 1) < L:
                lo = mid
            else:
                hi = mid
        r = 0.5 * (lo + hi)
    w = h_first * r ** np.arange(n)
    w *= L / w.sum()
    if not at_start:
        w = w[::-1]
    return x0 + np.concatenate([[0.0], np.cumsum(w)])


def flat_plate(kn=0.1, ma=0.2, nvel=48, vmax=5.0, levels=4, n_up=32, n_plate=64, n_down=32, ny=96,
               growth=1.1, omega=0.77):
    """Half-domain flat plate (Sec. 4.2): plate on y=0, x in [0,1], farfield
    20 plate lengths away; symmetry on y=0 off the plate; cells stretched
    geometrically (ratio `growth` in y) toward the plate.  BC ids: 0 plate
    wall, 1 symmetry, 2 farfield."""
    gamma = 5.0 / 3.0
    u_inf = ma * math.sqrt(gamma / 2.0)
    h_plate = 1.0 / n_plate
    xu = geometric_nodes(-20.0, 0.0, n_up, h_plate, at_start=False)
    xp = np.linspace(0.0, 1.0, n_plate + 1)
    xd = geometric_nodes(1.0, 21.0, n_down, h_plate, at_start=True)
    x = np.concatenate([xu, xp[1:], xd[1:]])
    h1 = 20.0 * (growth - 1.0) / (growth ** ny - 1.0)
    y = geometric_nodes(0.0, 20.0, ny, h1, at_start=True)
    nx = len(x) - 1
    south = np.where((np.arange(nx) >= n_up) & (np.arange(nx) < n_up + n_plate), 0, 1)
    fbx, fby = edge_face_ids(nx, ny, 2, 2, south, 2)
    return {
        "name": "plate%dx%d_v%d_kn%g" % (nx, ny, nvel, kn),
        "nx": nx, "ny": ny, "x_nodes": x, "y_nodes": y,
        "face_bc_x": fbx, "face_bc_y": fby,
        "bcs": [bc(WALL, t=1.0), bc(SYMMETRY), bc(FARFIELD, rho=1.0, u=u_inf, v=0.0, t=1.0)],
        "vgrid": {"nu": nvel, "nv": nvel, "umin": -vmax, "umax": vmax, "vmin": -vmax, "vmax": vmax,
                  "rule": TRAPEZOID},
        "gas": {"kn": kn, "omega": omega, "pr": 2.0 / 3.0},
        "mg": {"levels": levels, "nu1": 2, "nu2": 1, "nuc": 4, "cfl": 0.8, "dtn_growth": 0.0},
        "init": {"rho": 1.0, "u": u_inf, "v": 0.0, "t": 1.0},
    }


def body_face_ids(solid, fbx, fby, bc_id):
    """Give every face between a fluid cell and a solid cell the BC id `bc_id`
    and mark faces with no fluid cell on either side inactive (-1); returns
    new (fbx, fby) arrays.  `solid` is (ny, nx)."""
    solid = np.asarray(solid, dtype=bool)
    ny, nx = solid.shape
    fbx = np.asarray(fbx, dtype=np.int32).reshape(ny, nx + 1).copy()
    fby = np.asarray(fby, dtype=np.int32).reshape(ny + 1, nx).copy()
    fl = np.zeros((ny, nx + 1), dtype=bool)   # fluid cell on the lower side of x-face i
    fr = np.zeros((ny, nx + 1), dtype=bool)
    fl[:, 1:] = ~solid
    fr[:, :-1] = ~solid
    fbx[(fl ^ fr) & ~((np.arange(nx + 1) == 0) | (np.arange(nx + 1) == nx))[None, :]] = bc_id
    fbx[~fl & ~fr] = -1
    gl = np.zeros((ny + 1, nx), dtype=bool)
    gr = np.zeros((ny + 1, nx), dtype=bool)
    gl[1:, :] = ~solid
    gr[:-1, :] = ~solid
    fby[(gl ^ gr) & ~((np.arange(ny + 1) == 0) | (np.arange(ny + 1) == ny))[:, None]] = bc_id
    fby[~gl & ~gr] = -1
    return fbx.ravel(), fby.ravel()


def square_cylinder(ma=5.0, kn=0.1, nvel=89, vmax=15.0, levels=4, nx_side=64, nx_sq=32, ny_side=48, ny_sq=24,
                    half=7.5, omega=0.81, dtn_growth=3.0, rule=TRAPEZOID):
    """Flow past a unit square at the centre of the box [-half, half]^2
    (Sec. 4.3, on the full domain): nx_side | nx_sq | nx_side cells in x and
    ny_side | ny_sq | ny_side in y, uniform across the square and stretched
    geometrically away from its faces (the first outer cell as wide as a square
    cell).  The square's cells are solid.  BC ids: 0 square wall (T_w = T_inf),
    1 farfield (inflow, top, bottom), 2 outflow (zero gradient, downstream).
    The initial state is the freestream with a rear region x > 0.5 at 0.1 of
    its density and at rest (`rear` key, see initial_fields).  Velocity
    weights: the trapezoid rule, the closed Newton-Cotes rule of degree 1
    (Sec. 4.3 names Newton-Cotes rules without their degree); composite Boole
    (rule=BOOLE) is available for (nvel - 1) % 4 == 0."""
    gamma = 5.0 / 3.0
    u_inf = ma * math.sqrt(gamma / 2.0)
    hx, hy = 1.0 / nx_sq, 1.0 / ny_sq
    x = np.concatenate([geometric_nodes(-half, -0.5, nx_side, hx, at_start=False),
                        np.linspace(-0.5, 0.5, nx_sq + 1)[1:], geometric_nodes(0.5, half, nx_side, hx)[1:]])
    y = np.concatenate([geometric_nodes(-half, -0.5, ny_side, hy, at_start=False),
                        np.linspace(-0.5, 0.5, ny_sq + 1)[1:], geometric_nodes(0.5, half, ny_side, hy)[1:]])
    nx, ny = len(x) - 1, len(y) - 1
    solid = np.zeros((ny, nx), dtype=np.uint8)
    solid[ny_side:ny_side + ny_sq, nx_side:nx_side + nx_sq] = 1
    fbx, fby = edge_face_ids(nx, ny, 1, 2, 1, 1)
    fbx, fby = body_face_ids(solid, fbx, fby, 0)
    return {
        "name": "square%dx%d_v%d_ma%g_kn%g" % (nx, ny, nvel, ma, kn),
        "nx": nx, "ny": ny, "x_nodes": x, "y_nodes": y,
        "face_bc_x": fbx, "face_bc_y": fby, "solid": solid.ravel(),
        "bcs": [bc(WALL, t=1.0), bc(FARFIELD, rho=1.0, u=u_inf, v=0.0, t=1.0), bc(OUTFLOW)],
        "vgrid": {"nu": nvel, "nv": nvel, "umin": -vmax, "umax": vmax, "vmin": -vmax, "vmax": vmax, "rule": rule},
        "gas": {"kn": kn, "omega": omega, "pr": 2.0 / 3.0},
        "mg": {"levels": levels, "nu1": 2, "nu2": 1, "nuc": 4, "cfl": 0.8, "dtn_growth": dtn_growth},
        "init": {"rho": 1.0, "u": u_inf, "v": 0.0, "t": 1.0},
        "rear": {"x": 0.5, "rho": 0.1, "u": 0.0, "v": 0.0, "t": 1.0},
    }


def initial_fields(case):
    """Per-cell initial (rho, u, v, T): the uniform `init` state, with the
    `rear` region (cell centres downstream of rear["x"]), if the case has one,
    at its own state (Sec. 4.3)."""
    nx, ny = case["nx"], case["ny"]
    out = [np.full(nx * ny, float(case["init"][k])) for k in ("rho", "u", "v", "t")]
    rear = case.get("rear")
    if rear is not None:
        xc = 0.5 * (np.asarray(case["x_nodes"])[1:] + np.asarray(case["x_nodes"])[:-1])
        sel = np.broadcast_to(xc[None, :] > rear["x"], (ny, nx)).ravel()
        for q, k in enumerate(("rho", "u", "v", "t")):
            out[q][sel] = rear[k]
    return out


def coarsen_case(case):
    """The same problem on the next coarser mesh (every second grid line, as
    the multigrid levels of Sec. 3.1), with one multigrid level fewer: the
    coarse problems of a full-multigrid start-up."""
    nx, ny = case["nx"], case["ny"]
    if nx % 2 or ny % 2 or case["mg"]["levels"] < 2:
        raise ValueError("cannot coarsen %dx%d with %d levels" % (nx, ny, case["mg"]["levels"]))
    fbx = np.asarray(case["face_bc_x"]).reshape(ny, nx + 1)
    fby = np.asarray(case["face_bc_y"]).reshape(ny + 1, nx)
    if not (np.array_equal(fbx[0::2, 0::2], fbx[1::2, 0::2]) and np.array_equal(fby[0::2, 0::2], fby[0::2, 1::2])):
        raise ValueError("a coarse face would span two boundary ids")
    c = dict(case)
    c["name"] = case["name"] + "_coarse"
    c["nx"], c["ny"] = nx // 2, ny // 2
    c["x_nodes"] = np.asarray(case["x_nodes"])[0::2].copy()
    c["y_nodes"] = np.asarray(case["y_nodes"])[0::2].copy()
    c["face_bc_x"] = fbx[0::2, 0::2].ravel().copy()
    c["face_bc_y"] = fby[0::2, 0::2].ravel().copy()
    if case.get("solid") is not None:
        sol = np.asarray(case["solid"]).reshape(ny, nx)
        blocks = sol.reshape(ny // 2, 2, nx // 2, 2).sum(axis=(1, 3))
        if np.any((blocks != 0) & (blocks != 4)):
            raise ValueError("solid cells do not fill whole coarse cells")
        c["solid"] = (blocks == 4).astype(np.uint8).ravel()
    c["mg"] = dict(case["mg"], levels=case["mg"]["levels"] - 1)
    c["bcs"] = [dict(b) for b in case["bcs"]]
    return c


def splitmix64(seed):
    """SplitMix64 stream of uniform doubles in [0, 1) (53-bit)."""
    state = seed & 0xFFFFFFFFFFFFFFFF
    while True:
        state = (state + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
        z ^= z >> 31
        yield (z >> 11) * 2.0 ** -53


def kn_sweep(count=32, seed=1704, n=96, nvel=40, levels=4):
    """Independent cavities with Kn log-uniform on [0.01, 10] and lid speed
    uniform on [0.1, 0.3] (Kn drawn first, then the lid speed, per case)."""
    g = splitmix64(seed)
    out = []
    for _ in range(count):
        kn = 10.0 ** (-2.0 + 3.0 * next(g))
        lid = 0.1 + 0.2 * next(g)
        out.append(cavity(n=n, nvel=nvel, kn=kn, lid=lid, levels=levels))
    return out


def random_fields(case, seed, amp=0.05):
    """Smooth seeded perturbation of the initial state (rho, u, v, T)."""
    rng = np.random.default_rng(seed)
    nx, ny = case["nx"], case["ny"]
    xc = 0.5 * (case["x_nodes"][1:] + case["x_nodes"][:-1])
    yc = 0.5 * (case["y_nodes"][1:] + case["y_nodes"][:-1])
    X, Y = np.meshgrid((xc - xc.min()) / max(np.ptp(xc), 1e-30), (yc - yc.min()) / max(np.ptp(yc), 1e-30))
    out = []
    for base, scale in ((case["init"]["rho"], 1.0), (case["init"]["u"], 0.0), (case["init"]["v"], 0.0),
                        (case["init"]["t"], 1.0)):
        a = rng.uniform(-1, 1, 4)
        field = a[0] * np.sin(math.pi * X) * np.sin(math.pi * Y) + a[1] * X * Y + a[2] * np.cos(2 * X) * Y \
            + a[3] * (X - 0.5) ** 2
        out.append((base + amp * (scale if scale else 1.0) * field).ravel())
    return out


CONFIGS = {
    "c1": lambda: cavity(n=24, nvel=20, kn=1.0, lid=0.16, levels=1),
    "c2": lambda kn=1.0: cavity(n=64, nvel=32, kn=kn, lid=0.16, levels=3),
    "c3": lambda: flat_plate(),
    "c4": lambda: square_cylinder(),
}
