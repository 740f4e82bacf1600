"""Concurrent solution of independent problems (e.g. the Kn sweep of
lid-driven cavities): one solver per problem, each on its own CUDA stream,
driven by a single host thread through miugks_step_async / miugks_wait.

Every problem is iterated until each component of its RMS residual is below
`tol` (Sec. 4.1), until the residual stops falling (relative change below
`floor_rtol` over one chunk: the floor that a truncated velocity grid sets at
small Kn, where the discrete moments of the Maxwellian miss W by about the
truncation error and the collision term divides that by tau), or `max_iter`;
the wavefront kernels of one problem leave most of the GPU idle, so running the
problems side by side fills it.
"""
import time

from . import miugks


def run_concurrent(cases, tol=1e-6, max_iter=2000, chunk=5, precision="mixed", floor_rtol=1e-3):
    import torch
    streams = [torch.cuda.Stream() for _ in cases]
    solvers = []
    for case, st in zip(cases, streams):
        s = miugks.Solver(case, stream=st, precision=precision)
        init = case["init"]
        s.init_uniform(init["rho"], init["u"], init["v"], init["t"])
        solvers.append(s)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    active = list(range(len(cases)))
    iters = [0] * len(cases)
    res = [None] * len(cases)
    stop = ["max_iter"] * len(cases)
    while active:
        for q in active:
            solvers[q].step_async(chunk)
        still = []
        for q in active:
            r = solvers[q].wait()
            iters[q] += chunk
            prev, res[q] = res[q], r
            if max(r) < tol:
                stop[q] = "tolerance"
            elif prev is not None and abs(max(r) - max(prev)) < floor_rtol * max(prev):
                stop[q] = "floor"
            elif iters[q] < max_iter:
                still.append(q)
        active = still
    torch.cuda.synchronize()
    seconds = time.perf_counter() - t0
    return {"seconds": seconds, "iterations": iters, "residuals": [list(map(float, r)) for r in res],
            "stopped_at": stop, "solvers": solvers}
