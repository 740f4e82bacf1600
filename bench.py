"""Benchmark: MIUGKS outer iterations on one GB300.

A step is one outer iteration (Steps 1-8 of arXiv 1704.03151, Sec. 2.4) of the
64x64-cell lid-driven cavity with 32x32 discrete velocities on [-4,4]^2,
Kn = 1, lid speed 0.16, 3-level V-cycle (nu1 = 2, nu2 = 1, 4 coarsest
smoothings), FP64.  value = cell-velocity updates per second
(64*64*32*32 per step) with the state resident in HBM; e2e = the same through
the C ABI with host arrays each step (initial fields in, macroscopic fields and
residual out); time_to_residual = wall time to RMS residual 1e-6 from rest.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle (serial C) on the host on the
same workload.  Under torchrun with N > 1 every rank runs an independent
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
# algorithmic work of the dominant kernel ("Roofline"): FP64
# flops of the interface-flux kernel per (face, velocity), and the measured
# FP64 FMA throughput of a GB300 (FMA-chain kernel, no MEASURED_PEAKS.json entry)
FLUX_FLOPS_PER_FACE_VELOCITY = 175.0
FP64_PEAK_TFLOPS = 1.20


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


def oracle_iterations_per_s(n_iter):
    import oracle
    o = oracle.Oracle(case())
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
    o = oracle.Oracle(case())
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
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "%d full outer iterations of the workload, serial C oracle" % args.steps},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ttr", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    args.warmup = max(args.warmup, 3)
    import torch
    rank, world = dist_setup(args.gpus)
    from paper_1704_03151_gb300 import build, miugks
    build.build()
    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = miugks.Solver(case(), stream=stream)
    s.init_uniform(1.0, 0.0, 0.0, 1.0)
    cv = NX * NY * NVEL * NVEL
    launches_per_step = count_launches()

    # ---- device-resident timed region
    s.step(args.warmup)
    s.set_timing(True)
    s.kernel_times()
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = s.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    flux_ms, sweep_ms, total_ms = s.kernel_times()
    s.set_timing(False)
    ms = max_over_ranks(ms, world)
    value = cv * args.steps * world / (ms * 1e-3)

    # ---- end to end through the C ABI with host arrays every step
    from paper_1704_03151_gb300 import workloads
    c = case()
    fields = workloads.random_fields(c, 0, amp=0.0)
    e2e_steps = max(3, args.steps // 5)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        s.init_fields(*fields)
        s.step(1)
        s.macro()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e_value = cv * e2e_steps * world / e2e_s

    # ---- time to residual 1e-6 from rest
    ttr = None
    if not args.no_ttr and rank == 0:
        s.init_uniform(1.0, 0.0, 0.0, 1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        iters, rr, ok = s.run(1e-6, 3000)
        ttr = {"seconds": time.perf_counter() - t0, "iterations": iters, "converged": bool(ok),
               "residual": [float(x) for x in rr]}

    if rank != 0:
        return 0
    nfx, nfy = (NX + 1) * NY, NX * (NY + 1)
    flux_flops = FLUX_FLOPS_PER_FACE_VELOCITY * (nfx + nfy) * NVEL * NVEL
    flux_launch_ms = flux_ms / args.steps / 2.0          # two launches (x and y faces) per step
    achieved = flux_flops / 2.0 / (flux_launch_ms * 1e-3) / 1e12
    cpu = None
    if not args.no_cpu_baseline:
        n_iter = 4
        ips, secs = oracle_iterations_per_s(n_iter)
        cpu = {"value": ips * cv, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "%d outer iterations of the same workload (%.1f s), serial C oracle on the host" %
                         (n_iter, secs)}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": NX, "ny": NY, "nvel": NVEL, "levels": LEVELS, "kn": KN,
                   "l2": "working set (f, face fluxes, level arrays, ~0.6 GB) larger than L2",
                   "parallelism": "replicas" if world > 1 else "single"},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * NX * NY * 8,
                "d2h_bytes_per_step": 6 * NX * NY * 8 + 4 * 8},
        "roofline": {"bound": "alu", "kernel": "k_face_flux (FP64 pipe)", "achieved": achieved,
                     "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                     "traffic": None, "peak_source": "measured FP64 FMA chain on GB300 (no MEASURED_PEAKS.json)"},
        "stage_ms_per_step": {"flux": flux_ms / args.steps, "evolution_cs": sweep_ms / args.steps,
                              "total": total_ms / args.steps},
        "residual_last": [float(x) for x in res],
        "time_to_residual": ttr,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line))
    return 0


def count_launches():
    """Kernel launches of one outer iteration of the workload (host-side count of
    the launch sequence; every launch is one of this library's kernels)."""
    L = LEVELS
    nu1, nu2, nuc = 2, 1, 4
    per_sgs_micro = 4          # chain + interior, forward and backward
    per_renew = 1
    # Step 1: 2 flux + 1 residual + 2 rms
    n = 5
    # Step 2 FAS: gamma + forcing per level, smoother launches and renewals, transfers
    fas = 0
    for l in range(L):
        coarsest = l == L - 1
        fas += 2
        if coarsest:
            fas += nuc + (nuc - 1)
        else:
            fas += nu1 * 2 + 2 + 1 + 1 + nu2 * 2
    n += fas
    # Steps 3-4: micro residual + coarse coefficients (restrict + coeffs per coarse level)
    n += 1 + 2 * (L - 1)
    # Step 5 CS
    cs = 0
    for l in range(L):
        coarsest = l == L - 1
        cs += 0  # memset is not a kernel launch of this library
        if coarsest:
            cs += nuc * (per_sgs_micro + per_renew)
        else:
            cs += nu1 * (per_sgs_micro + per_renew) + 1 + 1 + nu2 * (per_renew + per_sgs_micro + per_renew)
    n += cs
    # Steps 6-7
    n += 1
    return n


if __name__ == "__main__":
    sys.exit(main())
