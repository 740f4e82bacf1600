"""Graph replay and concurrent solvers give exactly the results of eager,
one-at-a-time runs (same kernels in the same order, so bitwise)."""
import numpy as np
import pytest

from paper_1704_03151_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03151_gb300 import miugks, sweep
    miugks.load()
    return torch, miugks, sweep


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_replay_equals_eager(env, precision):
    torch, miugks, _ = env
    case = wl.cavity(n=16, nvel=12, kn=0.3, lid=0.2, levels=3)
    a = miugks.Solver(case, stream=torch.cuda.Stream(), precision=precision)
    b = miugks.Solver(case, stream=torch.cuda.Stream(), precision=precision)
    fields = wl.random_fields(case, 5, amp=0.05)
    a.init_fields(*fields)
    b.init_fields(*fields)
    a.set_timing(True)                    # stage timing keeps every iteration eager
    ra, rb = a.step(6), b.step(6)          # b replays a captured graph after its first iteration
    assert np.array_equal(ra, rb)
    assert np.array_equal(a.get_f(), b.get_f())


def test_concurrent_solvers_match_sequential(env):
    torch, miugks, sweep = env
    cases = [wl.cavity(n=16, nvel=12, kn=kn, lid=lid, levels=3) for kn, lid in ((0.05, 0.1), (0.5, 0.2), (5.0, 0.3))]
    out = sweep.run_concurrent(cases, tol=1e-5, max_iter=400, chunk=4, precision="mixed", floor_rtol=0.0)
    for q, case in enumerate(cases):
        s = miugks.Solver(case, stream=torch.cuda.Stream(), precision="mixed")
        s.init_uniform(1.0, 0.0, 0.0, 1.0)
        s.step(out["iterations"][q])
        assert np.array_equal(s.get_f(), out["solvers"][q].get_f()), q
        assert max(out["residuals"][q]) < 1e-5, (q, out["residuals"][q])
