"""Full-multigrid start-up (Sec. 3.5) through the C ABI: the prolonged initial
state and the iterations after it against the oracle, refusal of mismatched
solvers, and the FMG driver reaching the steady state of a plain solve."""
import numpy as np
import pytest

import oracle
from paper_1704_03151_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03151_gb300 import fmg, miugks
    miugks.load()
    return miugks, fmg


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _box_with_body():
    case = wl.cavity(n=16, nvel=10, kn=0.5, lid=0.2, levels=3)
    solid = np.zeros((16, 16), dtype=np.uint8)
    solid[8:12, 4:8] = 1
    case["bcs"] = case["bcs"] + [wl.bc(wl.WALL, t=1.2)]
    fbx, fby = wl.body_face_ids(solid, case["face_bc_x"], case["face_bc_y"], len(case["bcs"]) - 1)
    return dict(case, face_bc_x=fbx, face_bc_y=fby, solid=solid.ravel())


@pytest.mark.parametrize("make", [
    _box_with_body,
    lambda: wl.cavity(n=16, nvel=12, kn=0.5, lid=0.2, levels=3),
    lambda: wl.flat_plate(kn=0.2, nvel=12, levels=2, n_up=4, n_plate=8, n_down=4, ny=12),
])
def test_init_from_coarse_matches_oracle(env, make):
    miugks, _ = env
    case = make()
    coarse = wl.coarsen_case(case)
    oc = oracle.Oracle(coarse)
    oc.init_fields(*wl.random_fields(coarse, 2, amp=0.1))
    oc.step(2)
    gc = miugks.Solver(coarse)
    gc.init_uniform(1.0, 0.0, 0.0, 1.0)
    gc.set_f(oc.get_f())
    o, g = oracle.Oracle(case), miugks.Solver(case)
    o.init_from_coarse(oc)
    g.init_from_coarse(gc)
    assert rel(g.get_f(), o.get_f()) < 1e-12
    for k in ("rho", "u", "v", "t"):
        assert rel(g.macro()[k], o.macro()[k]) < 1e-12, k
    o.step(2), g.step(2)
    assert rel(g.get_f(), o.get_f()) < 1e-10


def test_init_from_coarse_refuses_mismatch(env):
    miugks, _ = env
    case = wl.cavity(n=16, nvel=12, kn=0.5, lid=0.2, levels=3)
    same = miugks.Solver(case)
    same.init_uniform(1.0, 0.0, 0.0, 1.0)
    fine = miugks.Solver(case)
    with pytest.raises(miugks.MiugksError):
        fine.init_from_coarse(same)                       # not the next coarser mesh
    other = miugks.Solver(wl.coarsen_case(wl.cavity(n=16, nvel=10, kn=0.5, lid=0.2, levels=3)))
    other.init_uniform(1.0, 0.0, 0.0, 1.0)
    with pytest.raises(miugks.MiugksError):
        fine.init_from_coarse(other)                      # another velocity grid
    fresh = miugks.Solver(wl.coarsen_case(case))
    with pytest.raises(miugks.MiugksError):
        fine.init_from_coarse(fresh)                      # coarse solver without a state


def test_fmg_reaches_the_plain_steady_state(env):
    miugks, fmg = env
    # farfield top and a wide velocity grid: a unique steady state with a residual that falls to round-off
    case = wl.cavity(n=16, nvel=24, kn=0.3, lid=0.2, vmax=6.0, levels=3)
    case["bcs"][2] = wl.bc(wl.FARFIELD, rho=1.0, u=0.2, v=0.0, t=1.0)
    s, info = fmg.run(case, tol=1e-11, max_iter=600)
    assert [m["nx"] for m in info["meshes"]] == [4, 8, 16]
    assert info["meshes"][-1]["stopped_at"] == "tolerance", info
    p = miugks.Solver(case)
    p.init_uniform(1.0, 0.0, 0.0, 1.0)
    it, res, ok = p.run(1e-11, 600)
    assert ok, res
    a, b = s.macro(), p.macro()
    for k in ("rho", "u", "v", "t"):
        assert np.allclose(a[k], b[k], rtol=1e-8, atol=1e-9), k


def test_init_from_coarse_falls_back_where_the_prolonged_state_is_unphysical(env):
    """Ma 5 past the square: after the coarse mesh has formed the bow shock,
    extrapolating f at the domain edge gives cells negative temperatures; those
    cells take their coarse cell's f, in both implementations alike."""
    miugks, _ = env
    case = wl.square_cylinder(nx_side=4, nx_sq=4, ny_side=4, ny_sq=4, levels=2, nvel=89, dtn_growth=3.0)
    coarse = wl.coarsen_case(case)
    oc = oracle.Oracle(coarse)
    oc.init_fields(*wl.initial_fields(coarse))
    oc.step(40)
    gc = miugks.Solver(coarse)
    gc.init_uniform(1.0, 0.0, 0.0, 1.0)
    gc.set_f(oc.get_f())
    o, g = oracle.Oracle(case), miugks.Solver(case)
    o.init_from_coarse(oc)
    g.init_from_coarse(gc)
    fo, fg = o.get_f(), g.get_f()
    assert rel(fg, fo) < 1e-12
    fc = oc.get_f()
    nx, cx = case["nx"], coarse["nx"]
    fell_back = [c for c in range(case["nx"] * case["ny"])
                 if np.array_equal(fo[:, c], fc[:, (c // nx // 2) * cx + (c % nx) // 2])
                 and not case["solid"][c]]
    assert len(fell_back) > 0
    m = g.macro()
    fluid = ~case["solid"].astype(bool)
    assert np.all(m["rho"][fluid] > 0) and np.all(m["t"][fluid] > 0)
    o.step(3), g.step(3)
    assert rel(g.get_f(), o.get_f()) < 1e-10
