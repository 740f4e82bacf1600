"""Parity of the CUDA library (through its C ABI) with the FP64 CPU oracle.

Stage by stage (fluxes, LU-SGS smoothers, operators, transfers) on small
seeded problems that span several tiles and ragged diagonals, then whole
iterations, then the full-size 64x64 cavity with 32x32 velocities.  The bar
for the FP64 path is 1e-10 relative (max abs difference over the max
magnitude of the compared array)."""
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


def cases():
    c_sym = wl.couette(n=10, nvel=12, kn=0.3, t_bottom=1.0, t_top=1.3, u_top=0.2, nx=6)
    c_open = wl.cavity(n=12, nvel=14, kn=0.2, lid=0.2, levels=2)
    c_open["bcs"][2] = wl.bc(wl.FARFIELD, rho=1.0, u=0.2, v=0.0, t=1.0)
    c_out = wl.cavity(n=8, nvel=10, kn=0.5, lid=0.0, levels=1, nx=12)
    c_out["bcs"][1] = wl.bc(wl.OUTFLOW)
    c_out["bcs"][3] = wl.bc(wl.FARFIELD, rho=1.0, u=0.3, v=0.0, t=1.0)
    c_str = wl.flat_plate(kn=0.2, nvel=12, levels=2, n_up=4, n_plate=8, n_down=4, ny=12)
    c_boole = wl.cavity(n=8, nvel=9, kn=0.4, lid=0.15, levels=2, rule=wl.BOOLE, vmax=4.0)
    return {
        "cavity": wl.cavity(n=16, nvel=12, kn=0.5, lid=0.2, levels=3),
        "cavity_rect": wl.cavity(n=8, nvel=10, kn=2.0, lid=0.3, levels=2, nx=12),
        "couette_sym": c_sym, "open_top": c_open, "outflow": c_out, "plate": c_str, "boole_odd": c_boole,
    }


CASES = cases()


def make_pair(lib, case, seed=0):
    o = oracle.Oracle(case)
    g = lib.Solver(case)
    fields = wl.random_fields(case, seed, amp=0.08)
    o.init_fields(*fields)
    g.init_fields(*fields)
    return o, g


@pytest.mark.parametrize("name", sorted(CASES))
def test_init_moments(lib, name):
    o, g = make_pair(lib, CASES[name])
    assert rel(g.get_f(), o.get_f()) < 1e-13
    mo, mg = o.macro(), g.macro()
    for k in ("rho", "u", "v", "t", "qx", "qy"):
        assert rel(mg[k], mo[k]) < 1e-11 or np.max(np.abs(mg[k] - mo[k])) < 1e-14, k


@pytest.mark.parametrize("name", sorted(CASES))
def test_flux_stage(lib, name):
    o, g = make_pair(lib, CASES[name], seed=1)
    Ro, pxo, pyo = o.stage_flux()
    Rg, pxg, pyg = g.stage_flux()
    assert rel(pxg, pxo) < TOL
    assert rel(pyg, pyo) < TOL
    assert rel(Rg, Ro) < 1e-9


@pytest.mark.parametrize("name", sorted(CASES))
def test_micro_sgs_and_operator(lib, name):
    case = CASES[name]
    o, g = make_pair(lib, case, seed=2)
    rng = np.random.default_rng(3)
    for lev in range(case["mg"]["levels"]):
        nx, ny = o.level_size(lev)
        nc = nx * ny
        it = rng.uniform(0.2, 3.0, nc)
        r = rng.normal(size=(2, nc, o.nv))
        assert rel(g.sgs_micro(lev, it, r), o.sgs_micro(lev, it, r)) < TOL, lev
        x = rng.normal(size=(2, nc, o.nv))
        assert rel(g.apply_micro(lev, it, x), o.apply_micro(lev, it, x)) < TOL, lev


@pytest.mark.parametrize("name", sorted(CASES))
def test_macro_smoother_and_residual(lib, name):
    case = CASES[name]
    o, g = make_pair(lib, case, seed=4)
    rng = np.random.default_rng(5)
    for lev in range(case["mg"]["levels"]):
        nx, ny = o.level_size(lev)
        nc = nx * ny
        rho = 1 + 0.1 * rng.uniform(-1, 1, nc)
        U, V, T = 0.1 * rng.uniform(-1, 1, nc), 0.1 * rng.uniform(-1, 1, nc), 1 + 0.1 * rng.uniform(-1, 1, nc)
        W = np.stack([rho, rho * U, rho * V, 0.5 * rho * (U * U + V * V) + 0.75 * rho * T], axis=1)
        Wg = W * (1 + 0.01 * rng.uniform(-1, 1, W.shape))
        R = 1e-2 * rng.normal(size=W.shape)
        assert rel(g.resid_macro(lev, W, Wg), o.resid_macro(lev, W, Wg)) < TOL
        assert rel(g.sgs_macro(lev, W, Wg, R), o.sgs_macro(lev, W, Wg, R)) < TOL


@pytest.mark.parametrize("name", ["cavity", "plate", "boole_odd"])
def test_transfers(lib, name):
    case = CASES[name]
    o, g = make_pair(lib, case)
    rng = np.random.default_rng(6)
    for lev in range(case["mg"]["levels"] - 1):
        nx, ny = o.level_size(lev)
        cx, cy = o.level_size(lev + 1)
        for m in (4, o.nv):
            fine = rng.normal(size=(nx * ny, m))
            assert rel(g.restrict(lev, fine), o.restrict(lev, fine)) < 1e-14
            coarse = rng.normal(size=(cx * cy, m))
            assert rel(g.prolong(lev, coarse), o.prolong(lev, coarse)) < 1e-14


@pytest.mark.parametrize("name", sorted(CASES))
def test_whole_iterations(lib, name):
    o, g = make_pair(lib, CASES[name], seed=7)
    for n in (1, 4):
        ro, rg = o.step(n), g.step(n)
        assert rel(rg, ro) < 1e-8, (n, rg, ro)
        assert rel(g.get_f(), o.get_f()) < TOL, n
        mo, mg = o.macro(), g.macro()
        for k in ("rho", "u", "v", "t"):
            assert rel(mg[k], mo[k]) < TOL, (n, k)


def test_config1_cavity_30_iterations(lib):
    """The 24x24 single-grid cavity (Kn 1, 20x20 velocities) over 30 iterations."""
    case = wl.CONFIGS["c1"]()
    o, g = oracle.Oracle(case), lib.Solver(case)
    for s in (o, g):
        s.init_uniform(1.0, 0.0, 0.0, 1.0)
    for _ in range(3):
        ro, rg = o.step(10), g.step(10)
        assert rel(rg, ro) < 1e-8
    mo, mg = o.macro(), g.macro()
    for k in ("rho", "u", "v", "t", "qx", "qy"):
        assert rel(mg[k], mo[k]) < TOL, k
    for b in range(4):
        for qo, qg in zip(o.wall(b), g.wall(b)):
            assert rel(qg, qo) < TOL


def test_config2_full_size_iteration(lib):
    """64x64 cells, 32x32 velocities, 3-level V-cycle: the configuration the
    benchmark times, compared on every output after two iterations."""
    case = wl.CONFIGS["c2"](kn=0.075)
    o, g = make_pair(lib, case, seed=9)
    ro, rg = o.step(2), g.step(2)
    assert rel(rg, ro) < 1e-8
    assert rel(g.get_f(), o.get_f()) < TOL
    mo, mg = o.macro(), g.macro()
    for k in ("rho", "u", "v", "t", "qx", "qy"):
        assert rel(mg[k], mo[k]) < TOL, k


def test_degenerate_limits(lib):
    """Near-continuum (dt/tau >> 1) and near-collisionless (dt/tau << 1) faces
    take the two branches of the time integrals; both must match."""
    for kn in (1e-4, 1e4):
        case = wl.cavity(n=8, nvel=10, kn=kn, lid=0.2, levels=2)
        o, g = make_pair(lib, case, seed=10)
        o.step(2)
        g.step(2)
        assert rel(g.get_f(), o.get_f()) < TOL, kn


def test_errors_are_reported(lib):
    bad = wl.cavity(n=6, nvel=8, levels=3)      # 6 is not divisible by 4
    with pytest.raises(lib.MiugksError):
        lib.Solver(bad)
    case = wl.cavity(n=8, nvel=8, levels=1)
    g = lib.Solver(case)
    with pytest.raises(lib.MiugksError):
        g.step(1)                                # before init
    g.init_uniform(1.0, 0.0, 0.0, 1.0)
    g.step(1)
