"""Checkpoint and resume through the C ABI: a run resumed from a saved state
repeats the uninterrupted run bit for bit, in a fresh solver too; a file of
another problem is refused."""
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


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_resume_repeats_the_run(lib, tmp_path, precision):
    case = wl.cavity(n=16, nvel=12, kn=0.5, lid=0.2, levels=2)
    s = lib.Solver(case, precision=precision)
    s.init_uniform(1.0, 0.0, 0.0, 1.0)
    s.step(3)
    path = str(tmp_path / "state.miugks")
    s.save(path)
    r_a = s.step(2)
    f_a = s.get_f()
    s.load(path)
    assert s.iterations() == 3
    r_b = s.step(2)
    assert np.array_equal(s.get_f(), f_a) and np.array_equal(r_a, r_b)
    t = lib.Solver(case, precision=precision)
    t.load(path)
    t.step(2)
    assert np.array_equal(t.get_f(), f_a)


def test_mismatching_checkpoint_is_refused(lib, tmp_path):
    a = lib.Solver(wl.cavity(n=8, nvel=10, kn=0.5, lid=0.2))
    a.init_uniform(1.0, 0.0, 0.0, 1.0)
    path = str(tmp_path / "a.miugks")
    a.save(path)
    b = lib.Solver(wl.cavity(n=8, nvel=12, kn=0.5, lid=0.2))
    with pytest.raises(lib.MiugksError):
        b.load(path)
    with pytest.raises(lib.MiugksError):
        b.load(str(tmp_path / "missing.miugks"))
