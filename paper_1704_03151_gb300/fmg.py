"""Full-multigrid start-up (Sec. 3.5): solve the problem on the coarsest mesh
of its hierarchy first, then carry each converged state to the next finer mesh
by bilinear prolongation of f (miugks_init_from_coarse; a cell whose prolonged
state is unphysical takes its coarse cell's f) and iterate there,
until the finest mesh converges.  Each mesh runs the MIUGKS outer iteration
with the multigrid levels below it.

Orchestration only: every step runs in the library's kernels through its C ABI.
A mesh is done when each component of its RMS residual is below its tolerance,
or when the residual stops falling (relative change below `floor_rtol` over
one chunk: the floor that a truncated velocity grid sets at small Kn).
"""
import time

from . import miugks, workloads


def hierarchy(case, meshes):
    """[finest, ..., coarsest]: `meshes` problems, each on every second grid
    line of the previous one with one multigrid level fewer."""
    out = [case]
    for _ in range(meshes - 1):
        out.append(workloads.coarsen_case(out[-1]))
    return out


def _iterate(s, tol, max_iter, chunk, floor_rtol):
    iters, prev, stop, res = 0, None, "max_iter", None
    while iters < max_iter:
        res = s.step(chunk)
        iters += chunk
        if max(res) < tol:
            stop = "tolerance"
            break
        if prev is not None and abs(max(res) - prev) < floor_rtol * prev:
            stop = "floor"
            break
        prev = max(res)
    return iters, res, stop


def run(case, tol=1e-6, meshes=None, coarse_tol=None, max_iter=3000, chunk=5, precision="fp64", floor_rtol=1e-3):
    """Solve `case` with a full-multigrid start-up over `meshes` meshes
    (default: its multigrid levels).  Coarse meshes stop at `coarse_tol`
    (default `tol`).  Returns the finest solver and, per mesh from the
    coarsest, its size, iterations, seconds and stopping reason."""
    import torch
    meshes = meshes or case["mg"]["levels"]
    cases = hierarchy(case, meshes)[::-1]
    prev, levels = None, []
    t_all = time.perf_counter()
    for q, c in enumerate(cases):
        s = miugks.Solver(c, precision=precision)
        if prev is None:
            s.init_fields(*workloads.initial_fields(c))
        else:
            s.init_from_coarse(prev)
            prev.close()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        last = q == len(cases) - 1
        iters, res, stop = _iterate(s, tol if last else (coarse_tol or tol), max_iter, chunk, floor_rtol)
        levels.append({"nx": c["nx"], "ny": c["ny"], "iterations": iters, "seconds": time.perf_counter() - t0,
                       "stopped_at": stop, "residual": None if res is None else [float(x) for x in res]})
        prev = s
    return prev, {"seconds": time.perf_counter() - t_all, "meshes": levels}
