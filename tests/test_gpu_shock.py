"""Shock capturing (the pressure-jump term of the interface collision time;
off by default, the paper describes none) through the C ABI against the
oracle: whole iterations of a supersonic flow past a square body, where the
term acts at the bow shock, at the 1e-10 FP64 bar, and in the mixed form at
the mixed form's bound against the oracle (2e-5, as in test_gpu_mixed).  The
adjoint refuses the term."""
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


def square(levels):
    """Ma 3 past a square body from the uniform freestream (no rear region: a
    start violent enough to trip the positivity rules takes different discrete
    decisions in FP32 and FP64)."""
    c = wl.square_cylinder(ma=3.0, kn=0.05, nvel=17, vmax=8.0, levels=levels, nx_side=8, nx_sq=4, ny_side=8,
                           ny_sq=4, half=3.0, dtn_growth=0.0)
    c.pop("rear")
    return c


@pytest.mark.parametrize("precision,tol", [("fp64", TOL), ("mixed", 2e-5)])
@pytest.mark.parametrize("levels", [1, 2])
def test_shock_capturing_matches_oracle(lib, levels, precision, tol):
    case = square(levels)
    o, g, plain = oracle.Oracle(case), lib.Solver(case, precision=precision), lib.Solver(case, precision=precision)
    o.set_shock_capturing(True)
    g.set_shock_capturing(True)
    for s in (o, g, plain):
        s.init_fields(*wl.initial_fields(case))
    for n in (1, 3):
        ro, rg = o.step(n), g.step(n)
        plain.step(n)
        assert rel(g.get_f(), o.get_f()) < tol, (levels, precision, n)
        assert np.allclose(rg, ro, rtol=100 * tol, atol=1e-14), (n, rg, ro)
    # the term acts: the iterates differ from the solver without it
    assert rel(plain.get_f(), g.get_f()) > 1e-6


def test_adjoint_refuses_shock_capturing(lib):
    case = wl.cavity(n=8, nvel=8, kn=0.5, lid=0.2, levels=1)
    s = lib.Solver(case)
    s.init_uniform(1.0, 0.0, 0.0, 1.0)
    s.step(2)
    s.set_shock_capturing(True)
    with pytest.raises(lib.MiugksError) as e:
        s.adjoint(0, 2, 1, tol=1e-6, max_iter=5)
    assert e.value.status == lib.MIUGKS_EINVAL
