"""Mixed-precision solve finished in FP64: iterate in the mixed form (FP32
per-velocity state, fluxes and smoothers; FP64 moments, prediction and
residual) until the residual is below the tolerance or stops falling, then
carry the state to an FP64 solver of the same problem (miugks_copy_state)
and iterate there to the tolerance.

On meshes with cells of very different sizes (the flat plate's first cell is
2e-4 of the plate length) the FP32 rounding of the per-velocity fluxes,
divided by the smallest cell widths, sets the mixed form's residual floor
near 1e-5; the FP64 iterations that remove it start from the mixed form's
state.  Orchestration only: every step runs in the library's kernels.
"""
import time

from . import miugks, workloads


def _iterate(s, tol, max_iter, chunk, floor_rtol, hist):
    iters, prev, stop, res = 0, None, "max_iter", None
    while iters < max_iter:
        try:
            res = s.step(chunk)
        except miugks.MiugksError as e:
            return iters, res, "unphysical state (%s)" % str(e).split(": ", 1)[-1]
        iters += chunk
        hist.append(float(max(res)))
        if max(res) < tol:
            stop = "tolerance"
            break
        if prev is not None and abs(max(res) - prev) < floor_rtol * prev:
            stop = "floor"
            break
        prev = max(res)
    return iters, res, stop


def run(case, tol=1e-6, max_iter=3000, chunk=5, floor_rtol=1e-3, switch_rtol=1e-3, stream=None):
    """Solve `case` from its initial state to RMS residual `tol`: the mixed
    form first, then FP64 from the mixed form's state if the mixed form
    stopped at its floor.  The mixed form counts as at its floor once its
    largest residual component changes by less than `switch_rtol` (relative)
    over `chunk` iterations.  Near the floor the FP32 rounding makes the
    residual wander by about a per cent: on a strongly stretched mesh the
    mixed iterations still remove slow error modes there that the residual
    does not show (switch late: 1e-3), on a mesh of similar cells they add
    nothing that the FP64 phase has to repeat (switch early: 2e-2).  The FP64
    phase stops at `tol` or when it changes by less than `floor_rtol`.
    Returns the final solver and the iterations, seconds, stopping reason and
    residual history (the largest component after every `chunk` iterations)
    of each phase."""
    import torch
    s = miugks.Solver(case, precision="mixed", stream=stream)
    s.init_fields(*workloads.initial_fields(case))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h1 = []
    it1, res1, stop1 = _iterate(s, tol, max_iter, chunk, switch_rtol, h1)
    t1 = time.perf_counter()
    phases = [{"precision": "mixed", "iterations": it1, "seconds": t1 - t0, "stopped_at": stop1,
               "residual": None if res1 is None else [float(x) for x in res1], "history": h1}]
    if stop1 == "floor":
        d = miugks.Solver(case, precision="fp64", stream=stream)
        d.copy_state(s)
        s.close()
        s = d
        h2 = []
        it2, res2, stop2 = _iterate(s, tol, max_iter - it1, chunk, floor_rtol, h2)
        torch.cuda.synchronize()
        phases.append({"precision": "fp64", "iterations": it2, "seconds": time.perf_counter() - t1,
                       "stopped_at": stop2, "residual": None if res2 is None else [float(x) for x in res2],
                       "history": h2})
    torch.cuda.synchronize()
    last = phases[-1]
    return s, {"seconds": time.perf_counter() - t0, "iterations": sum(p["iterations"] for p in phases),
               "converged": last["stopped_at"] == "tolerance", "phases": phases}


def polish(s, case, tol=1e-9, max_iter=200, chunk=5, floor_rtol=1e-3, stream=None):
    """An FP64 solver of `case` that starts from the state of solver `s` (of
    either precision) and iterates to RMS residual `tol` or its floor.  The
    state to linearise the adjoint at: at a state converged in the mixed form
    (its FP32 rounding left in f) flexible GMRES needed 203 and over 400
    iterations for 96x96 cavities at Kn 1 and 5.8, against 61 and 75 after
    this polish.  Returns the FP64 solver (the caller closes both) and the
    polish's iterations and stopping reason."""
    d = miugks.Solver(case, precision="fp64", stream=stream)
    d.copy_state(s)
    h = []
    it, res, stop = _iterate(d, tol, max_iter, chunk, floor_rtol, h)
    return d, {"iterations": it, "stopped_at": stop, "residual": None if res is None else [float(x) for x in res]}

