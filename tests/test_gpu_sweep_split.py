"""The two launch layouts of the evolution smoother (Eq. microFinalDefect).

In a sweep pass a velocity whose u (or v) points away from the upwind x (or y)
neighbour has an exact-zero coefficient there, so only the velocities coupled
in both directions need the anti-diagonal wavefront; the others are swept
along rows, along columns or per cell by a line-parallel kernel.  That layout
must give the wavefront-only layout's results bit for bit (same arithmetic,
only the visiting order of independent velocities changes), and both must
match the oracle's serial sweep at 1e-10: on the domain edge's walls,
symmetry planes, farfield and outflow faces, on stretched meshes, with odd
velocity counts (a zero velocity component), and around bodies (whose lines
split the sweep into segments)."""
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


def body_case(levels, ma=0.3, nvel=11):
    return wl.square_cylinder(ma=ma, kn=0.5, nvel=nvel, vmax=6.0, levels=levels, nx_side=8, nx_sq=4, ny_side=8,
                              ny_sq=4, half=3.0, dtn_growth=0.0)


def cases():
    c_sym = wl.couette(n=10, nvel=12, kn=0.3, t_bottom=1.0, t_top=1.3, u_top=0.2, nx=6)
    c_open = wl.cavity(n=12, nvel=14, kn=0.2, lid=0.2, levels=2)
    c_open["bcs"][2] = wl.bc(wl.FARFIELD, rho=1.0, u=0.2, v=0.0, t=1.0)
    c_out = wl.cavity(n=8, nvel=10, kn=0.5, lid=0.0, levels=1, nx=12)
    c_out["bcs"][1] = wl.bc(wl.OUTFLOW)
    c_out["bcs"][3] = wl.bc(wl.FARFIELD, rho=1.0, u=0.3, v=0.0, t=1.0)
    return {
        "cavity": wl.cavity(n=16, nvel=12, kn=0.5, lid=0.2, levels=3),
        "cavity_odd": wl.cavity(n=8, nvel=9, kn=0.4, lid=0.15, levels=2, rule=wl.BOOLE, vmax=4.0),
        "couette_sym": c_sym, "open_top": c_open, "outflow": c_out,
        "plate": wl.flat_plate(kn=0.2, nvel=12, levels=2, n_up=4, n_plate=8, n_down=4, ny=12),
        "square_L1": body_case(1), "square_L2_odd": body_case(2, ma=2.0, nvel=13),
    }


CASES = cases()


def solver(lib, case, mode, precision="fp64", seed=2):
    g = lib.Solver(case, precision=precision)
    g.set_sweep_split(mode)
    fields = wl.initial_fields(case) if case.get("rear") is not None else wl.random_fields(case, seed, amp=0.08)
    g.init_fields(*fields)
    return g, fields


@pytest.mark.parametrize("name", sorted(CASES))
def test_split_sweep_matches_oracle_and_wavefront_bitwise(lib, name):
    case = CASES[name]
    o = oracle.Oracle(case)
    gs, fields = solver(lib, case, "split")
    gw, _ = solver(lib, case, "wave")
    o.init_fields(*fields)
    rng = np.random.default_rng(3)
    for lev in range(case["mg"]["levels"]):
        nx, ny = o.level_size(lev)
        nc = nx * ny
        it = rng.uniform(0.2, 3.0, nc)
        r = rng.normal(size=(2, nc, o.nv))
        xs, xw, xo = gs.sgs_micro(lev, it, r), gw.sgs_micro(lev, it, r), o.sgs_micro(lev, it, r)
        assert np.array_equal(xs, xw), (name, lev)
        assert rel(xs, xo) < TOL, (name, lev)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["cavity", "plate", "square_L2_odd", "open_top"])
def test_split_layout_whole_iterations_bitwise(lib, name, precision):
    case = CASES[name]
    gs, _ = solver(lib, case, "split", precision, seed=7)
    gw, _ = solver(lib, case, "wave", precision, seed=7)
    for n in (1, 3):
        rs, rw = gs.step(n), gw.step(n)
        assert np.array_equal(rs, rw), (name, precision, n)
        assert np.array_equal(gs.get_f(), gw.get_f()), (name, precision, n)
