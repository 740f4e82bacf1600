"""Failure detection through the C ABI without faulting or hanging the GPU.

A state that is no longer physical (a NaN in f, or a cell with negative
density) is planted on the host through miugks_set_f.  The next outer
iteration must report MIUGKS_EDIVERGED with the iteration in its message and
return normally; the CUDA context stays usable, so the solver can be given a
physical state again and iterate, and another solver on the same device runs
and matches a fresh solver bit for bit."""
import numpy as np
import pytest

from paper_1704_03151_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03151_gb300 import miugks
    miugks.load()
    return miugks


def plant(f, kind, cell):
    f = f.copy()
    if kind == "nan":
        f[0, cell, f.shape[2] // 3] = np.nan
    else:
        f[:, cell, :] *= -1.0               # negative density and internal energy
    return f


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("kind", ["nan", "negative"])
@pytest.mark.parametrize("levels", [1, 2])
def test_unphysical_state_reports_ediverged(lib, precision, kind, levels):
    case = wl.cavity(n=16, nvel=12, kn=0.5, lid=0.2, levels=levels)
    s = lib.Solver(case, precision=precision)
    s.init_uniform(1.0, 0.0, 0.0, 1.0)
    s.step(2)
    good = s.get_f()
    s.set_f(plant(good, kind, cell=5 * 16 + 7))
    with pytest.raises(lib.MiugksError) as e:
        s.step(1)
    assert e.value.status == lib.MIUGKS_EDIVERGED, str(e.value)
    assert "diverged at iteration" in str(e.value)
    # the context survives: a physical state iterates again, and a second solver agrees with a fresh one
    s.set_f(good)
    r = s.step(1)
    assert np.all(np.isfinite(r))
    a, b = lib.Solver(case, precision=precision), lib.Solver(case, precision=precision)
    for t in (a, b):
        t.init_uniform(1.0, 0.0, 0.0, 1.0)
        t.step(3)
    assert np.array_equal(a.get_f(), b.get_f())
    s.close()


def test_bounded_wait_gives_up_and_reports_etimeout(lib):
    """The prediction smoother's cluster sweep waits (bounded) for each
    diagonal's inputs and its neighbours' values.  With the bound at zero
    every such wait gives up (the inputs are normally complete at the first
    test, so only that setting reaches the path): the kernel drains its copies
    in flight with bounded waits, returns, and the host reads MIUGKS_ETIMEOUT.
    No fault, no hang: the solver is destroyed cleanly and a new one on the
    same device iterates as a fresh one does."""
    case = wl.cavity(n=64, nvel=8, kn=0.5, lid=0.2, levels=2)
    s = lib.Solver(case)
    s.init_uniform(1.0, 0.0, 0.0, 1.0)
    s.step(1)
    s.set_wait_limit(0.0)
    with pytest.raises(lib.MiugksError) as e:
        s.step(1)
    assert e.value.status == lib.MIUGKS_ETIMEOUT, str(e.value)
    s.close()
    a, b = lib.Solver(case), lib.Solver(case)
    for t in (a, b):
        t.init_uniform(1.0, 0.0, 0.0, 1.0)
        t.step(3)
    assert np.array_equal(a.get_f(), b.get_f())
    with pytest.raises(lib.MiugksError):
        a.set_wait_limit(-1.0)
