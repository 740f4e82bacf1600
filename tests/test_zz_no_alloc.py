"""The residual-norm entry point that allocates nothing
(miugks_residual_rms_noalloc) must agree with the solver's own residual entry
point (miugks_residual), call after call.

It exists for callers that cannot allocate device memory where they need the
convergence measure (a framework that only lends its own pools, an
allocator-free loop): they pass their own device arrays for the residual, the
state, the optional solid mask and the 5-double output, and the library uses a
fixed scratch array of its own.  This file is collected last on purpose so that
a run stopping at the first failure has already run everything else; it also
passes when run alone in a fresh process."""
import ctypes

import numpy as np
import pytest

from paper_1704_03151_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_03151_gb300 import build, miugks
    build.build()
    return torch, miugks, miugks.load()


def conservative(m):
    rho, u, v, t = m["rho"], m["u"], m["v"], m["t"]
    return np.stack([rho, rho * u, rho * v, 0.5 * rho * (u * u + v * v) + 0.75 * rho * t], axis=1)


def call_noalloc(torch, lib, R, W, solid, stream):
    Rd = torch.tensor(R, dtype=torch.float64, device="cuda")
    Wd = torch.tensor(np.nan_to_num(W), dtype=torch.float64, device="cuda")
    Sd = None if solid is None else torch.tensor(np.asarray(solid, dtype=np.uint8), device="cuda")
    out = torch.full((5,), -1.0, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    st = lib.miugks_residual_rms_noalloc(ctypes.c_void_p(Rd.data_ptr()), ctypes.c_void_p(Wd.data_ptr()),
                                         None if Sd is None else ctypes.c_void_p(Sd.data_ptr()),
                                         R.shape[0], ctypes.c_void_p(out.data_ptr()),
                                         ctypes.c_void_p(stream.cuda_stream))
    assert st == 0, lib.miugks_last_error(None)
    stream.synchronize()
    assert torch.cuda.memory_allocated() == before
    return out.cpu().numpy()


def body_cavity():
    """A 32x32 cavity with a 8x8 solid block in its middle (BC 0 on its faces)."""
    case = wl.cavity(n=32, nvel=12, kn=0.5, lid=0.2, levels=2)
    solid = np.zeros((32, 32), dtype=np.uint8)
    solid[12:20, 12:20] = 1
    case["solid"] = solid.ravel()
    case["face_bc_x"], case["face_bc_y"] = wl.body_face_ids(solid, case["face_bc_x"], case["face_bc_y"], 0)
    case["name"] += "_body"
    return case


def test_noalloc_residual_matches_solver_residual_twice(env):
    torch, miugks, lib = env
    stream = torch.cuda.current_stream()
    for seed, case in ((0, wl.cavity(n=24, nvel=16, kn=0.5, lid=0.2, levels=2)),
                       (1, wl.cavity(n=64, nvel=12, kn=0.1, lid=0.3, levels=3)),
                       (2, body_cavity())):
        s = miugks.Solver(case)
        s.init_fields(*wl.random_fields(case, seed, amp=0.1))
        solid = case.get("solid")
        for call in range(2):
            ref = s.residual()                          # existing entry point
            R, _, _ = s.stage_flux()                    # the same residual, as a host array
            W = conservative(s.macro())
            out = call_noalloc(torch, lib, R, W, solid, stream)
            assert np.allclose(out[:4], ref, rtol=1e-12, atol=1e-300), (call, out, ref)
            assert out[4] == 0.0
            s.step(1)                                   # new state for the second call


def test_noalloc_rejects_oversized_input_without_launching(env):
    torch, miugks, lib = env
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    st = lib.miugks_residual_rms_noalloc(p, p, None, 1048576 + 1, p, None)
    assert st == miugks.MIUGKS_EINVAL
    assert b"1048576" in lib.miugks_last_error(None)
    assert lib.miugks_residual_rms_noalloc(None, p, None, 4, p, None) == miugks.MIUGKS_EINVAL
