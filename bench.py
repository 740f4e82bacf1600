"""Benchmark: MIUGKS outer iterations on one GB300.

A step is one outer iteration (Steps 1-8 of arXiv 1704.03151, Sec. 2.4) of the
64x64-cell lid-driven cavity with 32x32 discrete velocities on [-4,4]^2,
Kn = 1, lid speed 0.16, 3-level V-cycle (nu1 = 2, nu2 = 1, 4 coarsest
smoothings).  The headline is the mixed form (FP32 per-velocity arithmetic,
FP64 moments, prediction and residual); the same run also measures the FP64
form (key "fp64").  value = cell-velocity updates per second
(64*64*32*32 per step) with the state resident in HBM; e2e = the same through
the C ABI with host arrays each step (initial fields in, macroscopic fields and
residual out); time_to_residual = wall time to RMS residual 1e-6 from rest.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle (its OpenMP build, on every host
core) on the same workload.  Under torchrun with N > 1 every rank runs an independent
replica (the method has no data-parallel exchange step) and value sums the
ranks' updates over the slowest rank's time.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

NX = NY = 64
NVEL = 32
KN = 1.0
LEVELS = 3
METRIC = "cell-velocity updates/s (MIUGKS outer iterations)"
UNIT = "cell*velocity/s"
WORKLOAD = "cavity64x64_v32x32_kn1_lid0.16_3level_Vcycle"
# algorithmic work of the interface-flux kernel: flops per (face, velocity)
FLUX_FLOPS_PER_FACE_VELOCITY = 175.0
# ALU peaks of a GB300 from its unit counts and clock: 152 SMs x 128 FP32
# lanes x 2 flops (FMA) x 2.07 GHz; FP64 at its nominal 1.25 TFLOP/s
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP64_PEAK_TFLOPS = 1.25


def hbm_peak():
    """Measured copy bandwidth of the GB300s (MEASURED_PEAKS.json),
    else the fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return 6800.0, "fallback 6.8 TB/s"


def case():
    from paper_1704_03151_gb300 import workloads
    return workloads.cavity(n=NX, nvel=NVEL, kn=KN, lid=0.16, levels=LEVELS)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.rows, self.proc = index, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in self.rows for q in range(4) if r[3 + q].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_setup(n):
    rank, world = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        import torch.distributed as dist
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_iterations_per_s(n_iter, omp=False):
    import oracle
    o = oracle.Oracle(case(), omp=omp)
    o.init_uniform(1.0, 0.0, 0.0, 1.0)
    t0 = time.perf_counter()
    o.step(n_iter)
    dt = time.perf_counter() - t0
    return n_iter / dt, dt


def run_reference(args):
    rank, world = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return 0
    cv = NX * NY * NVEL * NVEL
    import oracle
    o = oracle.Oracle(case(), omp=True)                 # the OpenMP build: every host core, serial bits
    o.init_uniform(1.0, 0.0, 0.0, 1.0)
    for _ in range(args.warmup):
        o.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(1)
    dt = time.perf_counter() - t0
    value = cv * args.steps / dt
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nx": NX, "ny": NY, "nvel": NVEL, "levels": LEVELS, "kn": KN},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
                             "sample": "%d full outer iterations of the workload, OpenMP build of the C oracle "
                                       "on all host cores" % args.steps},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def measure(precision, steps, warmup, world, rank, dev, with_e2e=True, with_ttr=True, clocks=True,
            with_adjoint=False):
    import torch
    from paper_1704_03151_gb300 import miugks, workloads
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = miugks.Solver(case(), stream=stream, precision=precision)
    s.init_uniform(1.0, 0.0, 0.0, 1.0)
    cv = NX * NY * NVEL * NVEL
    s.step(warmup)
    barrier(world)
    torch.cuda.synchronize()
    sampler = ClockSampler(dev) if clocks else None
    if sampler:
        sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = s.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = sampler.stop() if sampler else None
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    # stage breakdown in a separate pass (per-stage events synchronise the host every iteration)
    s.set_timing(True)
    s.kernel_times()
    s.macro_sweep_times()
    nst = max(3, steps // 5)
    s.step(nst)
    flux_ms, sweep_ms, total_ms = s.kernel_times()
    macro_ms, macro_n = s.macro_sweep_times()
    s.set_timing(False)
    out = {"value": cv * steps * world / (ms * 1e-3), "ms_per_step": ms / steps, "clocks": clk,
           "flux_ms_per_launch": flux_ms / nst / 2.0,
           "macro_ms_per_launch": macro_ms / max(macro_n, 1), "macro_launches_per_step": macro_n / nst,
           "stage_ms_per_step": {"flux": flux_ms / nst, "evolution_cs": sweep_ms / nst, "total": total_ms / nst},
           "residual_last": [float(x) for x in res]}
    if with_e2e:
        c = case()
        fields = workloads.random_fields(c, 0, amp=0.0)
        n = max(3, steps // 5)
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n):
            s.init_fields(*fields)
            s.step(1)
            s.macro()
        torch.cuda.synchronize()
        sec = max_over_ranks(time.perf_counter() - t0, world)
        out["e2e"] = {"value": cv * n * world / sec, "unit": UNIT, "h2d_bytes_per_step": 4 * NX * NY * 8,
                      "d2h_bytes_per_step": 6 * NX * NY * 8 + 4 * 8}
    if with_ttr and rank == 0:
        s.init_uniform(1.0, 0.0, 0.0, 1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        iters, rr, ok = s.run(1e-6, 3000)
        out["time_to_residual"] = {"seconds": time.perf_counter() - t0, "iterations": iters, "converged": bool(ok),
                                   "residual": [float(x) for x in rr]}
        if with_adjoint:
            # differentiation form at the converged state: d(lid shear)/d(lid speed), FP64 adjoint
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g, info = s.adjoint(0, 2, 1, tol=1e-8, max_iter=600)
            out["adjoint"] = {"objective": "lid-wall shear force", "parameter": "lid speed", "gradient": g,
                              "seconds": time.perf_counter() - t0, "gmres_iterations": info["iterations"],
                              "relative_residual": info["residual"], "converged": info["converged"]}
    s.close()
    return out


# Dominant kernel of the step (largest share of the ncu launch list): the
# prediction smoother's LU-SGS sweep, k_macro_sgs, on the finest level.
# Algorithmic bytes per cell and launch: reads W, R (4 doubles each), the
# inverse diagonal (1), the Gamma of the faces (2 per cell), writes dW and W
# (4 each): 19 doubles = 152 B.
MACRO_BYTES_PER_CELL = 152.0
# DRAM bytes (read + write) of one finest-level k_macro_sgs<float> launch from
# the ncu capture summarised in profiles/k_macro_sgs_cavity64_v32_mixed.md
MACRO_TRAFFIC_MIXED = 1.796352e6


def macro_roofline(m, precision):
    t = m["macro_ms_per_launch"] * 1e-3
    hpeak, hsrc = hbm_peak()
    gbs = MACRO_BYTES_PER_CELL * NX * NY / t / 1e9
    return {"bound": "hbm", "kernel": "k_macro_sgs (finest level)", "achieved": gbs, "peak": hpeak, "unit": "GB/s",
            "frac": gbs / hpeak, "traffic": MACRO_TRAFFIC_MIXED if precision == "mixed" else None,
            "peak_source": hsrc, "launch_ms": m["macro_ms_per_launch"],
            "limiter": "dependency chain: %d anti-diagonals per sweep, one halo exchange each" % (NX + NY - 1)}


def flux_roofline(m, precision, nx=None, ny=None, nv=None, traffic=None):
    """Roofline of the face-flux kernel: algorithmic flops per (face, velocity)
    in the arithmetic type against that type's measured peak, and algorithmic
    bytes (f read once, fluxes written once) against the measured copy rate."""
    nx, ny, nv = nx or NX, ny or NY, nv or NVEL * NVEL
    nfx, nfy = (nx + 1) * ny, nx * (ny + 1)
    fv = (nfx + nfy) * nv / 2.0                               # (face, velocity) pairs per launch
    t = m["flux_ms_per_launch"] * 1e-3
    size = 4 if precision == "mixed" else 8
    flops = FLUX_FLOPS_PER_FACE_VELOCITY * fv / t / 1e12
    bytes_ = (2 * nx * ny * nv + 2 * fv) * size / t / 1e9
    fpeak = FP32_PEAK_TFLOPS if precision == "mixed" else FP64_PEAK_TFLOPS
    hpeak, hsrc = hbm_peak()
    if flops / fpeak >= bytes_ / hpeak:
        return {"bound": "alu", "kernel": "k_face_flux", "achieved": flops, "peak": fpeak, "unit": "TFLOP/s",
                "frac": flops / fpeak, "traffic": None,
                "peak_source": "%s peak from unit counts and clock (152 SMs, 2.07 GHz)" %
                               ("FP32" if precision == "mixed" else "FP64 nominal"),
                "hbm_frac": bytes_ / hpeak, "hbm_peak_source": hsrc}
    return {"bound": "hbm", "kernel": "k_face_flux", "achieved": bytes_, "peak": hpeak, "unit": "GB/s",
            "frac": bytes_ / hpeak, "traffic": traffic, "peak_source": hsrc, "alu_frac": flops / fpeak}


# algorithmic passes over one per-velocity array (Nc Nv 2 values) per outer
# iteration of the 3-level V(2,1) cycle with 4 coarsest smoothings: flux and
# residual 2, every fine smoothing 4-5, transfers 3.5, update 3, coarse levels
# about 6 (see the design notes): 29 passes
PASSES_PER_ITERATION = 29.0


def step_hbm(m, precision):
    """Whole-step bandwidth: the method's compulsory bytes per iteration over
    the measured time per iteration."""
    size = 4 if precision == "mixed" else 8
    b = PASSES_PER_ITERATION * 2 * NX * NY * NVEL * NVEL * size
    hpeak, hsrc = hbm_peak()
    gbs = b / (m["ms_per_step"] * 1e-3) / 1e9
    return {"bytes_per_step": b, "achieved": gbs, "peak": hpeak, "unit": "GB/s", "frac": gbs / hpeak,
            "peak_source": hsrc}


def kn_series(max_iter=600):
    """The 64x64 cavity at the three Kn of its configuration (0.075, 1, 10):
    time to RMS residual 1e-6 from rest in the FP64 and the mixed form (or to
    the floor that the truncated [-4,4]^2 velocity grid sets at small Kn: the
    discrete moments of the Maxwellian miss W by about 1e-7, which the
    collision term divides by tau), and the
    mixed form's converged error against the FP64 solver (relative L-infinity of
    density, velocity, temperature and lid-wall shear)."""
    import torch
    from paper_1704_03151_gb300 import miugks, workloads
    out = []
    for kn in (0.075, 1.0, 10.0):
        row = {"kn": kn}
        sol = {}
        for prec in ("fp64", "mixed"):
            c = workloads.cavity(n=NX, nvel=NVEL, kn=kn, lid=0.16, levels=LEVELS)
            s = miugks.Solver(c, precision=prec)
            s.init_uniform(1.0, 0.0, 0.0, 1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            # to RMS 1e-6, or to the discretisation floor: the residual of the truncated
            # velocity grid stops falling (change below 0.1 % over 5 iterations)
            iters, prev, stop = 0, None, "max_iter"
            while iters < max_iter:
                rr = s.step(5)
                iters += 5
                if max(rr) < 1e-6:
                    stop = "tolerance"
                    break
                if prev is not None and abs(max(rr) - prev) < 1e-3 * prev:
                    stop = "floor"
                    break
                prev = max(rr)
            row[prec] = {"seconds": time.perf_counter() - t0, "iterations": iters, "stopped_at": stop,
                         "residual": [float(x) for x in rr]}
            m = s.macro()
            sol[prec] = (m, s.wall(2)[1])
            s.close()
        (m64, tw64), (m32, tw32) = sol["fp64"], sol["mixed"]
        speed = np.hypot(m64["u"], m64["v"]).max()
        row["mixed_error"] = {
            "rho": float(np.abs(m32["rho"] - m64["rho"]).max() / np.abs(m64["rho"]).max()),
            "velocity": float(max(np.abs(m32["u"] - m64["u"]).max(), np.abs(m32["v"] - m64["v"]).max()) / speed),
            "t": float(np.abs(m32["t"] - m64["t"]).max() / np.abs(m64["t"]).max()),
            "lid_shear": float(np.abs(tw32 - tw64).max() / np.abs(tw64).max())}
        out.append(row)
    return out


def measure_plate(steps, warmup):
    """The flat-plate configuration at full size (128x96 stretched cells, 48x48
    velocities on [-5,5]^2, Kn = 0.1, 4-level V-cycle, mixed form): 28.3 M cell-
    velocity pairs, one FP32 per-velocity array 226 MB, larger than L2.  Same
    timing as the headline (events on the solver's stream, state resident)."""
    import torch
    from paper_1704_03151_gb300 import miugks, workloads
    c = workloads.flat_plate()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = miugks.Solver(c, stream=stream, precision="mixed")
    s.init_uniform(c["init"]["rho"], c["init"]["u"], c["init"]["v"], c["init"]["t"])
    s.step(warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = s.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    # per-launch event timing of the flux and evolution-sweep kernels (timing mode, a separate pass)
    s.set_timing(True)
    s.kernel_times()
    s.sweep_kernel_times()
    nst = 3
    s.step(nst)
    flux_ms, sweep_ms, total_ms = s.kernel_times()
    sk = s.sweep_kernel_times()
    s.set_timing(False)
    cv = c["nx"] * c["ny"] * c["vgrid"]["nu"] * c["vgrid"]["nv"]
    b = PASSES_PER_ITERATION * 2 * cv * 4
    hpeak, hsrc = hbm_peak()
    s.close()
    return {"workload": "flat_plate_%dx%d_v48x48_kn0.1_4level_mixed" % (c["nx"], c["ny"]), "steps": steps,
            "value": cv / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "residual_last": [float(x) for x in res],
            "stage_ms_per_step": {"flux": flux_ms / nst, "evolution_cs": sweep_ms / nst, "total": total_ms / nst},
            "roofline_flux": flux_roofline({"flux_ms_per_launch": flux_ms / nst / 2.0}, "mixed", c["nx"], c["ny"],
                                           c["vgrid"]["nu"] * c["vgrid"]["nv"], traffic=FLUX_TRAFFIC_PLATE_MIXED),
            "roofline_sweep": sweep_roofline(sk, "mixed"),
            "step_hbm": {"bytes_per_step": b, "achieved": b / (ms * 1e-3) / 1e9, "peak": hpeak, "unit": "GB/s",
                         "frac": b / (ms * 1e-3) / 1e9 / hpeak, "peak_source": hsrc}}


# Evolution-sweep kernels: per (cell, velocity) and sweep direction the
# algorithmic traffic is three values read (the residual of G and H and the
# inverse diagonal forward; the forward result and the inverse diagonal
# backward) and two written (the new G and H): 20 B in FP32, 40 B in FP64.
SWEEP_VALUES_PER_CV = 5
# DRAM bytes per cell-velocity pair of the flat plate's finest-level sweep
# kernels (mixed), from the ncu captures summarised in
# profiles/k_sgs_plate128x96_v48_mixed.md (forward and backward launches)
SWEEP_TRAFFIC_PER_CV = {"lines": 30.2, "wave": 29.8}
# DRAM bytes (read + written) of one launch of the flat plate's face-flux kernel
# (mixed, x-faces), from the ncu capture in profiles/k_face_flux_plate128x96_v48_mixed.md
FLUX_TRAFFIC_PLATE_MIXED = 417.3e6
# the same for one launch of the square cylinder's face flux (mixed, x-faces): the ncu capture of the half-size
# case (80x60 cells, 4,860 x-faces, 580.9 MB; profiles/k_face_flux_square80x60_v89_mixed.md) scaled by the
# faces of the full case (19,320), since each face reads its cells' rows and writes its own fluxes
FLUX_TRAFFIC_SQUARE_MIXED = 580.9e6 * 19320 / 4860


def sweep_roofline(sk, precision):
    """Per kernel: algorithmic bytes of its finest-level launches over their
    event-timed duration, against the measured copy rate."""
    size = 4 if precision == "mixed" else 8
    hpeak, hsrc = hbm_peak()
    out = {}
    for name in ("lines", "wave"):
        ms, n, units = sk[name]
        if n <= 0 or ms <= 0:
            continue
        gbs = SWEEP_VALUES_PER_CV * size * units / (ms * 1e-3) / 1e9
        tr = SWEEP_TRAFFIC_PER_CV[name]
        out[name] = {"bound": "hbm", "kernel": "k_sgs_lines" if name == "lines" else "k_sgs_wave",
                     "achieved": gbs, "peak": hpeak, "unit": "GB/s", "frac": gbs / hpeak,
                     "traffic": None if tr is None else tr * units / n, "peak_source": hsrc,
                     "launch_ms": ms / n, "cv_per_launch": units / n}
    return out


def measure_square(steps, warmup, precision="mixed"):
    """The square-cylinder configuration at full size (160x120 cells with the
    32x24-cell square solid, 18,432 fluid cells, 89x89 velocities on
    [-15,15]^2 with the trapezoid rule, Ma 5, Kn 0.1, 4-level V-cycle,
    dt_n growth 3, rear region at 0.1 of the freestream density): 152 M
    cell-velocity pairs (the body's cells counted, as they are swept), one
    FP32 per-velocity array 1.2 GB.  Same timing as the headline."""
    import torch
    from paper_1704_03151_gb300 import miugks, workloads
    c = workloads.square_cylinder()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = miugks.Solver(c, stream=stream, precision=precision)
    s.init_fields(*workloads.initial_fields(c))
    s.step(warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = s.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    # stage breakdown in a separate pass (events per stage)
    s.set_timing(True)
    s.kernel_times()
    s.step(2)
    flux_ms, sweep_ms, total_ms = s.kernel_times()
    s.set_timing(False)
    cv = c["nx"] * c["ny"] * c["vgrid"]["nu"] * c["vgrid"]["nv"]
    b = PASSES_PER_ITERATION * 2 * cv * (4 if precision == "mixed" else 8)
    hpeak, hsrc = hbm_peak()
    s.close()
    stage = {"flux_ms_per_launch": flux_ms / 2 / 2.0}
    return {"workload": "square_cylinder_%dx%d_v89x89_ma5_kn0.1_4level_%s" % (c["nx"], c["ny"], precision),
            "steps": steps, "value": cv / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
            "stage_ms_per_step": {"flux": flux_ms / 2, "evolution_cs": sweep_ms / 2, "total": total_ms / 2},
            "roofline_flux": flux_roofline(stage, precision, c["nx"], c["ny"], c["vgrid"]["nu"] * c["vgrid"]["nv"],
                                           traffic=FLUX_TRAFFIC_SQUARE_MIXED if precision == "mixed" else None),
            "residual_last": [float(x) for x in res],
            "step_hbm": {"bytes_per_step": b, "achieved": b / (ms * 1e-3) / 1e9, "peak": hpeak, "unit": "GB/s",
                         "frac": b / (ms * 1e-3) / 1e9 / hpeak, "peak_source": hsrc}}


def converge_big(name, max_iter=1500):
    """The flat plate or the square cylinder at full size from its initial
    state to RMS residual 1e-6 (Sec. 4.1): the mixed form until the residual
    stops falling (the FP32 floor of these stretched meshes), then FP64 from
    that state (refine.run); and the FP64 form alone, for comparison.  Wall
    times include every host read of the residual (one per 5 iterations)."""
    import torch
    from paper_1704_03151_gb300 import miugks, refine, workloads
    c = workloads.flat_plate() if name == "plate" else workloads.square_cylinder()
    warm = miugks.Solver(c, precision="mixed")               # one-time kernel set-up of both forms
    warm.init_fields(*workloads.initial_fields(c))
    warm.step(2)
    w64 = miugks.Solver(c, precision="fp64")
    w64.copy_state(warm)
    w64.step(2)
    warm.close()
    w64.close()
    # the mixed form's switch to FP64: late on the stretched plate mesh, early on the square's (refine.run)
    s, info = refine.run(c, tol=1e-6, max_iter=max_iter, switch_rtol=1e-3 if name == "plate" else 2e-2)
    info["switch_rtol"] = 1e-3 if name == "plate" else 2e-2
    s.close()
    d = miugks.Solver(c, precision="fp64")
    d.init_fields(*workloads.initial_fields(c))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    iters, prev, stop = 0, None, "max_iter"
    while iters < max_iter:
        rr = d.step(5)
        iters += 5
        if max(rr) < 1e-6:
            stop = "tolerance"
            break
        if prev is not None and abs(max(rr) - prev) < 1e-3 * prev:
            stop = "floor"
            break
        prev = max(rr)
    torch.cuda.synchronize()
    fp64 = {"seconds": time.perf_counter() - t0, "iterations": iters, "stopped_at": stop,
            "residual": [float(x) for x in rr]}
    d.close()
    return {"mixed_then_fp64": info, "fp64": fp64,
            "speedup": fp64["seconds"] / info["seconds"] if info["converged"] and stop == "tolerance" else None}


def square_convergence(precision, max_iter, chunk=5, dtn_growth=None):
    """Iterate the full-size square cylinder from its initial state to RMS 1e-6,
    to its floor (change below 0.1 % over a chunk), to max_iter, or until the
    solver reports an unphysical state; the residual history and the end state."""
    import torch
    from paper_1704_03151_gb300 import miugks, workloads
    c = workloads.square_cylinder() if dtn_growth is None else workloads.square_cylinder(dtn_growth=dtn_growth)
    s = miugks.Solver(c, precision=precision)
    s.init_fields(*workloads.initial_fields(c))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    iters, prev, stop, rr = 0, None, "max_iter", [float("nan")] * 4
    hist = []
    while iters < max_iter:
        try:
            rr = s.step(chunk)
        except miugks.MiugksError as e:
            stop = "unphysical state (%s)" % str(e).split(": ", 1)[-1]
            break
        iters += chunk
        hist.append([iters, float(max(rr))])
        if max(rr) < 1e-6:
            stop = "tolerance"
            break
        if prev is not None and abs(max(rr) - prev) < 1e-3 * prev:
            stop = "floor"
            break
        prev = max(rr)
    secs = time.perf_counter() - t0
    out = {"precision": precision, "dtn_growth": c["mg"]["dtn_growth"], "iterations": iters, "seconds": secs,
           "stopped_at": stop,
           "residual": [float(x) for x in rr], "history": hist[::max(1, len(hist) // 25)]}
    if not stop.startswith("unphysical"):
        p, tau, q = s.wall(0)
        m = s.macro()
        fl = ~np.asarray(c["solid"]).astype(bool)
        out.update({"wall_heat_flux_total": float(np.sum(q)), "wall_faces": int(len(q)),
                    "rho_range": [float(np.min(m["rho"][fl])), float(np.max(m["rho"][fl]))],
                    "t_range": [float(np.min(m["t"][fl])), float(np.max(m["t"][fl]))]})
        out["_state"] = ({k: m[k][fl] for k in ("rho", "u", "v", "t")}, q)
    s.close()
    return out


def square_mixed_error(conv):
    """Mixed form against FP64 at the same iteration count: relative L-infinity
    difference of density, velocity, temperature and the wall heat flux."""
    a, b = conv[0].pop("_state", None), conv[1].pop("_state", None)
    if a is None or b is None or conv[0]["iterations"] != conv[1]["iterations"]:
        return None
    (m32, q32), (m64, q64) = a, b
    speed = np.hypot(m64["u"], m64["v"]).max()
    return {"iterations": conv[0]["iterations"],
            "rho": float(np.abs(m32["rho"] - m64["rho"]).max() / np.abs(m64["rho"]).max()),
            "velocity": float(max(np.abs(m32["u"] - m64["u"]).max(), np.abs(m32["v"] - m64["v"]).max()) / speed),
            "t": float(np.abs(m32["t"] - m64["t"]).max() / np.abs(m64["t"]).max()),
            "wall_heat_flux": float(np.abs(q32 - q64).max() / np.abs(q64).max())}


def run_square_adjoint(args):
    """--workload square_adjoint: the square cylinder at full size solved to RMS
    1e-8 (mixed form to its floor, then FP64: refine.run), then the FP64
    adjoint gradient of the heat flux into the square (the sum over its wall
    faces of face length x heat flux, BC 0) with respect to its wall
    temperature: flexible GMRES(--restart) to --adj-tol, preconditioned by the
    transposed multigrid cycle, body faces included.  With --fd,
    also central differences of two more converged solves (T_w = 1 +- 5e-3)."""
    import torch
    from paper_1704_03151_gb300 import build, miugks, refine, workloads
    build.build()
    c = workloads.square_cylinder()
    s, fwd = refine.run(c, tol=1e-8, max_iter=args.max_iter, switch_rtol=2e-2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g, info = s.adjoint(1, 0, 0, tol=args.adj_tol, max_iter=600, restart=args.restart)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    J = info["J"]
    s.close()
    fd = None
    if args.fd:
        h = 5e-3
        Js = []
        for sg in (1, -1):
            cc = workloads.square_cylinder()
            cc["bcs"][0]["t"] = 1.0 + sg * h
            sp, _ = refine.run(cc, tol=1e-8, max_iter=args.max_iter, switch_rtol=2e-2)
            Js.append(sp.objective(1, 0)[0])
            sp.close()
        fd = (Js[0] - Js[1]) / (2 * h)
    print(json.dumps({"metric": "square-cylinder heat-flux gradient w.r.t. wall temperature (adjoint)", "unit": "s",
                      "value": secs, "higher_is_better": False,
                      "config": {"workload": "square_cylinder_160x120_v89x89_ma5_kn0.1_4level", "restart": args.restart},
                      "forward": fwd, "heat_flux": J, "gradient": g, "gmres_iterations": info["iterations"],
                      "relative_residual": info["residual"], "converged": info["converged"],
                      "central_difference": fd}))
    return 0


def run_plate_iter(args):
    """--workload plate_iter: --steps outer iterations of the full-size flat
    plate (mixed form) from its initial state, eagerly launched after the
    first; a small, fixed target for kernel profiles."""
    import torch
    from paper_1704_03151_gb300 import build, miugks, workloads
    build.build()
    c = workloads.flat_plate()
    s = miugks.Solver(c, precision=args.precision)
    s.init_fields(*workloads.initial_fields(c))
    res = s.step(args.steps)
    torch.cuda.synchronize()
    print(json.dumps({"workload": "flat_plate_%dx%d_v48x48_kn0.1_4level_%s" % (c["nx"], c["ny"], args.precision),
                      "iterations": args.steps, "residual": [float(x) for x in res]}))
    return 0


def run_square_iter(args):
    """--workload square_iter: --steps outer iterations (mixed form unless
    --precision fp64) of the square cylinder at half size per axis (80x60
    cells, 16x12-cell square, 89x89 velocities, 3 levels; a few GB on the
    device) from its initial state, eagerly launched after the first; a
    small profiling target with the full-size case's velocity grid."""
    import torch
    from paper_1704_03151_gb300 import build, miugks, workloads
    build.build()
    c = workloads.square_cylinder(levels=3, nx_side=32, nx_sq=16, ny_side=24, ny_sq=12)
    s = miugks.Solver(c, precision=args.precision)
    s.init_fields(*workloads.initial_fields(c))
    res = s.step(args.steps)
    torch.cuda.synchronize()
    print(json.dumps({"workload": "square_cylinder_%dx%d_v89x89_3level_%s" % (c["nx"], c["ny"], args.precision),
                      "iterations": args.steps, "residual": [float(x) for x in res]}))
    return 0


def run_square(args):
    """--workload square: the full-size square cylinder, throughput in both
    forms over iterations 3-5 from the initial state (the start is violent at
    Ma 5; the state stays physical there in both implementations), then the
    iteration toward the steady state in both forms (--max-iter), reported up
    to where it stops."""
    from paper_1704_03151_gb300 import build
    build.build()
    # the first iterations from the initial state (every iteration runs the same kernels)
    mixed = measure_square(3, 2, "mixed")
    fp64 = measure_square(2, 2, "fp64")
    conv = [square_convergence("mixed", args.max_iter, dtn_growth=args.dtn_growth),
            square_convergence("fp64", min(args.max_iter, 60), dtn_growth=args.dtn_growth)]
    mixed_error = square_mixed_error(conv)
    for cv in conv:
        cv.pop("_state", None)
    # full-multigrid start-up (Sec. 3.5, used by the paper for this case): 20x15 -> 40x30 -> 80x60 -> 160x120
    from paper_1704_03151_gb300 import fmg, miugks, workloads
    c = workloads.square_cylinder() if args.dtn_growth is None else workloads.square_cylinder(dtn_growth=args.dtn_growth)
    info = None
    if args.max_iter > 0:
        try:
            sfin, info = fmg.run(c, tol=1e-6, max_iter=args.max_iter, precision="mixed")
            sfin.close()
        except miugks.MiugksError as e:
            info = {"stopped": "unphysical state (%s)" % str(e).split(": ", 1)[-1]}
    line = {"metric": "square-cylinder cell-velocity updates/s (Ma 5, Kn 0.1)", "value": mixed["value"],
            "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "dtype": "f32/f64", "data": "synthetic",
            "config": {"workload": mixed["workload"]}, "mixed": mixed, "fp64": fp64, "convergence": conv,
            "mixed_error": mixed_error, "fmg": info}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ttr", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison run")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint gradient at the converged state")
    ap.add_argument("--no-plate", action="store_true", help="skip the full-size flat-plate throughput line")
    ap.add_argument("--no-square", action="store_true", help="skip the full-size square-cylinder throughput line")
    ap.add_argument("--workload", default="cavity64",
                    choices=["cavity64", "kn_sweep", "adjoint", "cycles", "plate_adjoint", "square", "plate_iter",
                             "square_adjoint", "square_iter"])
    ap.add_argument("--count", type=int, default=32, help="cavities of the Kn sweep")
    ap.add_argument("--restart", type=int, default=20, help="GMRES restart length of --workload square_adjoint")
    ap.add_argument("--adj-tol", type=float, default=1e-6, help="adjoint GMRES tolerance of --workload square_adjoint")
    ap.add_argument("--fd", action="store_true", help="square_adjoint: also central differences of converged solves")
    ap.add_argument("--max-iter", type=int, default=1500)
    ap.add_argument("--adjoint", action="store_true", help="Kn sweep: adjoint lid-shear gradient of every case")
    ap.add_argument("--dtn-growth", type=float, default=None,
                    help="square cylinder: growth factor of the numerical time step for the convergence runs")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "kn_sweep":
        return run_kn_sweep(args)
    if args.workload == "adjoint":
        return run_adjoint(args)
    if args.workload == "cycles":
        return run_cycles(args)
    if args.workload == "plate_adjoint":
        return run_plate_adjoint(args)
    if args.workload == "plate_iter":
        return run_plate_iter(args)
    if args.workload == "square_adjoint":
        return run_square_adjoint(args)
    if args.workload == "square_iter":
        return run_square_iter(args)
    if args.workload == "square":
        return run_square(args)
    args.warmup = max(args.warmup, 3)
    import torch
    rank, world = dist_setup(args.gpus)
    from paper_1704_03151_gb300 import build
    build.build()
    dev = torch.cuda.current_device()
    head = measure(args.precision, args.steps, args.warmup, world, rank, dev, with_ttr=not args.no_ttr,
                   with_adjoint=not args.no_adjoint)
    other = None
    if not args.no_fp64 and args.precision == "mixed":
        other = measure("fp64", max(3, args.steps // 3), args.warmup, world, rank, dev, with_e2e=False,
                        with_ttr=not args.no_ttr, clocks=False)
    plate = series = square = None
    if not args.no_plate and rank == 0:
        plate = measure_plate(max(5, args.steps // 5), args.warmup)
        if not args.no_ttr:
            plate["time_to_residual"] = converge_big("plate")
    if not args.no_square and rank == 0:
        square = measure_square(3, 2, "mixed")
        if not args.no_ttr:
            square["time_to_residual"] = converge_big("square", max_iter=400)
    if not args.no_ttr and rank == 0:
        series = kn_series()
    if rank != 0:
        return 0
    cv = NX * NY * NVEL * NVEL
    cpu = None
    if not args.no_cpu_baseline:
        # the oracle as it stands on the host: its OpenMP build on every core (the same bits as the
        # serial build), and the serial build on one core
        n_omp, n_ser = 10, 5
        ips, secs = oracle_iterations_per_s(n_omp, omp=True)
        ips1, secs1 = oracle_iterations_per_s(n_ser, omp=False)
        cpu = {"value": ips * cv, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
               "sample": "%d outer iterations of the same workload from rest (%.1f s), OpenMP build of the C "
                         "oracle on all host cores" % (n_omp, secs),
               "serial": {"value": ips1 * cv, "unit": UNIT, "cores": 1,
                          "sample": "%d outer iterations (%.1f s), serial build" % (n_ser, secs1)}}
    line = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32/f64" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": NX, "ny": NY, "nvel": NVEL, "levels": LEVELS, "kn": KN,
                   "precision": args.precision,
                   "l2": "working set (f, face fluxes, level arrays, 0.3-0.6 GB) larger than L2",
                   "parallelism": "replicas" if world > 1 else "single"},
        "gpu_launches": count_launches() * args.steps,
        "clocks": head["clocks"],
        "e2e": head["e2e"],
        "roofline": macro_roofline(head, args.precision),
        "roofline_flux": flux_roofline(head, args.precision),
        "step_hbm": step_hbm(head, args.precision),
        "stage_ms_per_step": head["stage_ms_per_step"],
        "residual_last": head["residual_last"],
        "time_to_residual": head.get("time_to_residual"),
        "adjoint": head.get("adjoint"),
        "flat_plate": plate,
        "square_cylinder": square,
        "kn_series": series,
        "cpu_baseline": cpu,
    }
    if other:
        line["fp64"] = {"value": other["value"], "ms_per_step": other["ms_per_step"],
                        "stage_ms_per_step": other["stage_ms_per_step"],
                        "time_to_residual": other.get("time_to_residual"),
                        "roofline": macro_roofline(other, "fp64"),
                        "roofline_flux": flux_roofline(other, "fp64"),
                        "step_hbm": step_hbm(other, "fp64")}
    print(json.dumps(line))
    return 0


def run_adjoint(args):
    """The differentiation form alone: the 64x64 cavity solved in the mixed form
    to RMS residual 1e-6 from rest, then the FP64 adjoint gradient of the
    lid-wall shear force with respect to the lid speed (GMRES to 1e-8 or
    --max-iter iterations)."""
    import torch
    from paper_1704_03151_gb300 import build, miugks
    build.build()
    s = miugks.Solver(case(), precision=args.precision)
    s.init_uniform(1.0, 0.0, 0.0, 1.0)
    iters, rr, ok = s.run(1e-6, 3000)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g, info = s.adjoint(0, 2, 1, tol=1e-8, max_iter=args.max_iter)
    sec = time.perf_counter() - t0
    print(json.dumps({"metric": "adjoint gradient time (d lid-wall shear / d lid speed)", "value": sec, "unit": "s",
                      "higher_is_better": False, "config": {"workload": WORKLOAD, "forward_precision": args.precision,
                                                             "forward_iterations": iters},
                      "gradient": g, "gmres_iterations": info["iterations"],
                      "relative_residual": info["residual"], "converged": info["converged"]}))
    return 0


def run_plate_adjoint(args):
    """The full-size flat plate (128x96 stretched cells, 48x48 velocities,
    Kn 0.1, Ma 0.2, 4 levels): forward solve from the freestream to RMS 1e-6
    (or its residual floor), then the FP64 adjoint gradient of the plate drag
    (the shear force on the plate wall of the half domain) with respect to the
    plate wall temperature, GMRES to 1e-6 or --max-iter iterations."""
    import torch
    from paper_1704_03151_gb300 import build, miugks, workloads
    build.build()
    c = workloads.flat_plate()
    s = miugks.Solver(c, precision=args.precision)
    ini = c["init"]
    s.init_uniform(ini["rho"], ini["u"], ini["v"], ini["t"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    iters, prev, stop = 0, None, "max_iter"
    while iters < 3000:
        rr = s.step(10)
        iters += 10
        if max(rr) < 1e-6:
            stop = "tolerance"
            break
        if prev is not None and abs(max(rr) - prev) < 1e-3 * prev:
            stop = "floor"
            break
        prev = max(rr)
    fwd = time.perf_counter() - t0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g, info = s.adjoint(0, 0, 0, tol=1e-6, max_iter=args.max_iter)
    print(json.dumps({"metric": "flat-plate drag gradient w.r.t. plate wall temperature", "unit": "s",
                      "higher_is_better": False,
                      "config": {"workload": "flat_plate_128x96_v48x48_kn0.1_4level", "precision": args.precision},
                      "forward": {"seconds": fwd, "iterations": iters, "stopped_at": stop,
                                  "residual": [float(x) for x in rr]},
                      "drag": info["J"], "gradient": g, "seconds": time.perf_counter() - t0,
                      "gmres_iterations": info["iterations"], "relative_residual": info["residual"],
                      "converged": info["converged"]}))
    return 0


def run_cycles(args):
    """Cycle and smoothing-count study (Sec. 3.4 names V, W and F cycles and
    leaves the smoothing counts open): the 64x64 cavity from rest to RMS 1e-6
    (or to the residual floor, as in the Kn series) for each cycle type and
    (nu1, nu2), at Kn 1 and 10, in the precision of --precision."""
    import torch
    from paper_1704_03151_gb300 import build, miugks, workloads
    build.build()
    rows = []
    for kn in (1.0, 10.0):
        for cyc in ("V", "W", "F"):
            for nu1, nu2 in ((1, 1), (2, 1), (2, 2), (3, 1)):
                c = workloads.cavity(n=NX, nvel=NVEL, kn=kn, lid=0.16, levels=LEVELS, nu1=nu1, nu2=nu2)
                s = miugks.Solver(c, precision=args.precision)
                s.set_cycle(cyc)
                s.init_uniform(1.0, 0.0, 0.0, 1.0)
                s.step(1)                                  # one eager iteration (kernel set-up)
                s.init_uniform(1.0, 0.0, 0.0, 1.0)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                iters, rr, ok = s.run(1e-6, args.max_iter)
                rows.append({"kn": kn, "cycle": cyc, "nu1": nu1, "nu2": nu2, "iterations": iters,
                             "seconds": time.perf_counter() - t0, "converged": bool(ok),
                             "residual": [float(x) for x in rr]})
                s.close()
    # full-multigrid start-up (3 meshes: 16x16, 32x32, 64x64) against the plain start from rest, V(2,1)
    from paper_1704_03151_gb300 import fmg
    for kn in (0.075, 1.0, 10.0):
        c = workloads.cavity(n=NX, nvel=NVEL, kn=kn, lid=0.16, levels=LEVELS)
        warm, _ = fmg.run(c, tol=1e-6, max_iter=5, precision=args.precision)   # kernel set-up of every mesh
        warm.close()
        torch.cuda.synchronize()
        s, info = fmg.run(c, tol=1e-6, max_iter=args.max_iter, precision=args.precision)
        rows.append({"kn": kn, "cycle": "FMG start-up + V", "nu1": 2, "nu2": 1, "seconds": info["seconds"],
                     "meshes": info["meshes"]})
        s.close()
    print(json.dumps({"metric": "time to RMS residual 1e-6 by multigrid cycle and smoothing counts", "unit": "s",
                      "higher_is_better": False, "config": {"workload": WORKLOAD, "precision": args.precision},
                      "rows": rows}))
    return 0


def run_kn_sweep(args):
    """Kn sweep: `count` independent 96x96 cavities, 40x40 velocities, 4-level
    V-cycle, mixed form, Kn log-uniform on [0.01, 10] and lid speed uniform on
    [0.1, 0.3] from SplitMix64 seed 1704; all solved concurrently (one stream
    each) to RMS residual 1e-6."""
    import torch
    from paper_1704_03151_gb300 import build, sweep, workloads
    build.build()
    cases = workloads.kn_sweep(count=args.count)
    out = sweep.run_concurrent(cases, tol=1e-6, max_iter=args.max_iter, chunk=5, precision=args.precision)
    adj = None
    if args.adjoint:
        # differentiation form per case at its converged state: d(lid-wall shear)/d(lid speed), FP64
        # adjoint at the state polished in FP64 from the mixed solve (refine.polish); each solver is
        # released after its gradient so the work memory is reused
        from paper_1704_03151_gb300 import refine
        adj = {"objective": "lid-wall shear force", "parameter": "lid speed", "gradients": [], "seconds": [],
               "polish_seconds": [], "polish_iterations": [], "gmres_iterations": [], "converged": []}
        for q, s in enumerate(out["solvers"]):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            d, pinfo = refine.polish(s, cases[q])
            s.close()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            g, info = d.adjoint(0, 2, 1, tol=1e-8, max_iter=800)
            adj["polish_seconds"].append(t1 - t0)
            adj["polish_iterations"].append(pinfo["iterations"])
            adj["seconds"].append(time.perf_counter() - t1)
            adj["gradients"].append(g)
            adj["gmres_iterations"].append(info["iterations"])
            adj["converged"].append(info["converged"])
            d.close()
    cv = 96 * 96 * 40 * 40
    total_updates = cv * sum(out["iterations"])
    line = {"metric": "Kn-sweep cell-velocity updates/s (concurrent cavities to RMS residual 1e-6)",
            "value": total_updates / out["seconds"], "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
            "dtype": "f32/f64" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": "kn_sweep_%dx_cavity96_v40_L4" % args.count, "count": args.count},
            "seconds_to_solve_all": out["seconds"], "iterations": out["iterations"],
            "converged": [max(r) < 1e-6 for r in out["residuals"]], "stopped_at": out["stopped_at"],
            "residuals": out["residuals"],
            "kn": [c["gas"]["kn"] for c in cases], "lid": [c["bcs"][2]["u"] for c in cases], "adjoint": adj}
    print(json.dumps(line))
    return 0


def count_launches():
    """Kernel launches of one outer iteration of the workload, following the
    library's launch sequence (every launch is one of this library's kernels;
    memsets and copies are not counted).  Matches the ncu launch list of the
    same workload (134 per iteration for 3 levels)."""
    L, nu1, nu2, nuc = LEVELS, 2, 1, 4
    macro_sweep = 2            # per-diagonal record kernel + cluster sweep
    micro_sweep = 6            # boundary-line chain, line fold and wavefront, forward and backward
    n = 2 + 1 + 2              # Step 1: two face-flux launches, cell residual, RMS (partial + final)
    for l in range(L):         # Step 2: FAS
        coarsest = l == L - 1
        npre = nuc if coarsest else nu1
        n += 2 + 1             # Gamma and inverse diagonal, forcing
        n += npre * macro_sweep + (npre - 1 if coarsest else npre)
        if not coarsest:
            n += 2 + 1 + 1 + nu2 * (1 + macro_sweep)   # restrictions, difference, prolongation, post-smoothing
    n += 1                     # the predicted state (FAS result, or W^n where it is unphysical)
    n += 1 + 2 * (L - 1)       # Steps 3-4: micro residual; per coarse level restriction + coefficients
    for l in range(L):         # Step 5: CS
        coarsest = l == L - 1
        npre = nuc if coarsest else nu1
        n += npre * (micro_sweep + 1)
        if not coarsest:
            n += 1 + 1 + nu2 * (1 + micro_sweep + 1)
    n += 1                     # Steps 6-7
    return n

if __name__ == "__main__":
    sys.exit(main())
