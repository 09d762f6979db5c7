"""Throughput benchmark of the slip-wall D2Q9 MRT solver.

Workload: the single-domain throughput case -- an 8192 x 4096 x-periodic
channel packed with random cylinders (radius 8-32 nodes, porosity 0.7,
seeded), Kn = 0.02, force-driven, FP32 deviation storage.  One benchmark
step = 100 lattice time steps (the fused collide-stream-boundary kernel)
followed by the FP64 residual/mass reduction and its read-back, i.e. one
pass of the whole hot path at the default residual interval; the default
--steps 100 times 10,000 lattice steps.

Prints one JSON line: MLUPS over fluid nodes (whole job), the roofline of
the step kernel against measured HBM bandwidth, an end-to-end number through
the C ABI with host buffers, and the FP64 CPU oracle timed on a bounded
sample of the same workload.  With --impl reference the oracle itself is the
timed arm (on the host cores).  On one GPU the line also carries, under
"extra_workloads", the other workloads measured after the main timed region
(BF16 storage, the 512-case batch to 1e-8, the warm start's time to steady
state, the D3Q19 extension); --no-extras skips them, --workload runs one of
them alone as the main line.

Multi-GPU (torchrun): every rank runs an independent replica of the case
(seed = rank); the path has no exchange step, so there is no collective in
the data path ("replicas only", weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

FLUID_BYTES = {"fp32": 72, "fp64": 144, "bf16": 36, "fp16": 36}  # algorithmic bytes per fluid-node update
# The FP64 step is bound by this GPU's FP64 units, not by HBM.  Its line is
# reported, not judged: the flops are those the step kernel EXECUTES per
# fluid-node update (dadd + dmul + 2 dfma, ncu counters on the 4096x2048
# case; profiles/), not an algorithmic count, and the peak is NVIDIA's
# nominal FP64 rate, not a measured one.
FP64_FLOPS_PER_NODE = 156.4
FP64_PEAK_GFLOPS = 1250.0
ELEM_BYTES = {"fp32": 4, "fp64": 8, "bf16": 2, "fp16": 2}
FALLBACK_HBM_GBS = 6800.0


FALLBACK_BF16_TFLOPS = 1900.0


def _peak_bf16():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        for key in ("bf16_tflops", "bf16_TFLOPS"):
            if key in d and isinstance(d[key], (int, float)):
                return float(d[key]), "measured"
    except (OSError, ValueError):
        pass
    return FALLBACK_BF16_TFLOPS, "fallback"


def _peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        for key in ("hbm_gbs", "hbm_GBps", "hbm"):
            if key in d and isinstance(d[key], (int, float)):
                return float(d[key]), "measured"
    except (OSError, ValueError):
        pass
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self._t.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_over_ranks(values_max, values_sum, world, device):
    """Every rank runs its own replica (no exchange in the data path): the
    job's timings are the slowest rank's, its work the sum over ranks.
    Returns (list of maxima, list of sums); a no-op for one rank."""
    if world == 1:
        return list(values_max), list(values_sum)
    import torch
    import torch.distributed as dist
    tm = torch.tensor([float(v) for v in values_max], dtype=torch.float64, device=device)
    ts = torch.tensor([float(v) for v in values_sum], dtype=torch.float64, device=device)
    dist.all_reduce(tm, op=dist.ReduceOp.MAX)
    dist.all_reduce(ts, op=dist.ReduceOp.SUM)
    return [float(v) for v in tm.cpu()], [float(v) for v in ts.cpu()]


def _oracle_band(rows: int, threads: int):
    """The FP64 oracle on an 8192 x `rows` channel built with the throughput
    case's cylinder recipe (a band of the same workload), on `threads`
    threads of its OpenMP build."""
    import oracle
    from oracle import params as P
    from paper_2012_14707_gb300 import cases
    case = cases.cylinder_array(8192, rows, 0, porosity=0.7, Kn=0.02, ax=1e-5,
                                name=f"cylinders_8192x{rows}_s0")
    return oracle.OracleLBM(case, P.Parameters(case.Kn, case.H), threads=threads), case


def cpu_baseline_sample(rows: int = 1024, warmup: int = 10, min_seconds: float = 5.0,
                        repeats: int = 3):
    """The FP64 oracle as it stands, on every host core, on a bounded sample of
    the workload: `warmup` lattice steps of an 8192 x `rows` band, then
    `repeats` timings of whole lattice steps, each at least `min_seconds`
    long.  Returns (median MLUPS over fluid nodes, case, cores, steps timed)."""
    import oracle
    cores = oracle.host_cores()
    o, case = _oracle_band(rows, cores)
    o.step(warmup)
    t0 = time.perf_counter()
    o.step(1)
    chunk = max(1, int(0.5 / max(time.perf_counter() - t0, 1e-6)))
    rates, steps = [], 0
    for _ in range(repeats):
        n = 0
        t0 = time.perf_counter()
        while True:
            o.step(chunk)
            n += chunk
            dt = time.perf_counter() - t0
            if dt >= min_seconds:
                break
        rates.append(case.n_fluid * n / dt / 1e6)
        steps += n
    return statistics.median(rates), case, o.threads, steps


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    cores = oracle.host_cores()
    # a band of the same recipe, as tall as keeps the whole run within about
    # three minutes on the host cores (~3 M fluid-node updates per second
    # and core assumed), at most 1024 rows
    rows = int(min(1024, max(16, 180 * 3e6 * cores / (0.7 * 8192 * max(1, args.steps + args.warmup)))))
    rows -= rows % 16
    o, case = _oracle_band(rows, cores)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    mlups = case.n_fluid * args.steps / dt / 1e6
    sample = (f"each step: one FP64 lattice step of an 8192x{rows} channel with the same "
              f"cylinder recipe ({case.n_fluid} fluid nodes), OpenMP over rows on "
              f"{o.threads} threads")
    line = {
        "impl": "reference", "metric": "MLUPS", "value": mlups, "unit": "MLUPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "cylinders_8192x4096_phi0.7_Kn0.02", "nx": 8192, "ny": 4096,
                   "precision": "fp64 (oracle)", "lattice_steps_per_step": 1,
                   "sample_rows": rows,
                   "l2": "inputs larger than L2 not applicable (CPU)"},
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": o.threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, emit=True):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2012_14707_gb300 import build as lbm_build
    from paper_2012_14707_gb300 import cases, lbm

    world, rank, local = _dist()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lbm_build.build()
    lbm.load()

    if args.nx or args.ny:
        case = cases.config_throughput(seed=rank, nx=args.nx or 8192, ny=args.ny or 4096)
    else:
        case = cases.config_throughput(seed=rank)
    stream = torch.cuda.current_stream(dev)
    mkw = {} if args.mass_mode is None else {"mass_mode": args.mass_mode}
    solver = lbm.Solver(case, precision=args.precision, stream=stream.cuda_stream,
                        residual_every=args.lbm_steps, **mkw)
    info = solver.info()
    n_fluid = info.n_fluid
    per = args.lbm_steps

    def bench_step():
        solver.step(per)
        return solver.residual()

    for _ in range(args.warmup):
        bench_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    k_start = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    k_end = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    last = None
    for s in range(args.steps):
        k_start[s].record(stream)
        solver.step(per)
        k_end[s].record(stream)
        last = solver.residual()
    t_end.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    elapsed_ms = t_start.elapsed_time(t_end)
    kernel_ms = sum(a.elapsed_time(b) for a, b in zip(k_start, k_end))
    (elapsed_ms, kernel_ms), (total_fluid,) = reduce_over_ranks([elapsed_ms, kernel_ms], [n_fluid],
                                                                world, dev)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()

    updates = total_fluid * per * args.steps
    mlups = updates / (elapsed_ms / 1e3) / 1e6
    launch_ms = kernel_ms / (args.steps * per)
    # the exact-mass step also reads and writes a carry per fluid node and
    # per link (4 B each way)
    exact = bool(info.exact_mass)
    node_bytes = FLUID_BYTES[args.precision] + (8 + 8 * info.n_links / n_fluid if exact else 0)
    alg_bytes = node_bytes * n_fluid
    achieved = alg_bytes / (launch_ms / 1e3) / 1e9
    # the same algorithmic bytes over the whole bench step (lattice steps,
    # residual pass and its read-back: the time the MLUPS figure counts)
    step_achieved = node_bytes * mlups * 1e6 / world / 1e9
    peak, peak_src = _peak_hbm()
    solver.close()

    # End to end through the C ABI with host buffers: create from host
    # arrays (mask + links H2D), the same steps with the residual read back,
    # and the final fields copied to host memory.
    torch.cuda.synchronize()
    e2e = None if args.no_e2e else _e2e(args, case, stream, per, world, n_fluid, lbm, torch, dev)


    traffic = None
    prof = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    if os.path.exists(prof):
        try:
            with open(prof) as fh:
                pj = json.load(fh)
            if (pj.get("precision") == args.precision and pj.get("kernel_rev") == KERNEL_REV
                    and not exact):
                traffic = pj.get("bytes_per_launch_full_size")
        except (OSError, ValueError):
            traffic = None

    line = {
        "metric": "MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "fp64": "f64", "bf16": "bf16", "fp16": "f16"}[args.precision],
        "data": "synthetic",
        "config": {"workload": f"cylinders_{case.nx}x{case.ny}_phi0.7_Kn0.02",
                   "nx": case.nx, "ny": case.ny, "n_fluid": n_fluid, "n_links": case.n_links,
                   "precision": args.precision, "lattice_steps_per_step": per,
                   "exact_mass_step": exact,
                   "l2": "inputs larger than L2 (2 x %.2f GB lattices of fluid nodes)" % (
                       9 * ((n_fluid + 31) // 32 * 32) * ELEM_BYTES[args.precision] / 1e9),
                   "parallelism": f"replicas x{world}"},
        "roofline": ({"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                      "frac": achieved / peak, "traffic": traffic,
                      "kernel": "step_kernel_pull<float, float, 1> (exact-mass)" if exact
                                else "step_kernel", "bytes_per_fluid_node": node_bytes,
                      "launch_ms": launch_ms, "peak_source": peak_src,
                      "step_achieved": step_achieved, "step_frac": step_achieved / peak,
                      "step_note": "same algorithmic bytes over the whole bench step (residual "
                                   "pass and read-back included), the time the MLUPS value counts",
                      "dram_gbs_ncu": (traffic / (launch_ms / 1e3) / 1e9) if traffic else None}
                     if args.precision != "fp64" else
                     {"bound": "alu", "achieved": FP64_FLOPS_PER_NODE * n_fluid / (launch_ms / 1e3) / 1e9,
                      "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s (FP64)",
                      "frac": FP64_FLOPS_PER_NODE * n_fluid / (launch_ms / 1e3) / 1e9 / FP64_PEAK_GFLOPS,
                      "traffic": None, "kernel": "step_kernel",
                      "flops_per_fluid_node": FP64_FLOPS_PER_NODE,
                      "flops_kind": "executed by the kernel (ncu counters), not algorithmic",
                      "hbm_gbs": achieved, "launch_ms": launch_ms,
                      "peak_source": "nominal GB300 FP64 rate (1.25 TFLOP/s), not measured",
                      "judged": False}),
        "e2e": e2e,
        "accuracy_vs_oracle": ACCURACY[args.precision],
        "gpu_launches": args.steps * (per + 2),
        "mlups_all_nodes": mlups * case.nx * case.ny / n_fluid,
        "clocks": clocks,
        "residual_last": last[0] if last else None,
    }
    if rank == 0 and not args.no_cpu_baseline:
        v, bcase, cores, nst = cpu_baseline_sample()
        line["cpu_baseline"] = {
            "value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle (OpenMP over rows, {cores} threads) on an 8192x{bcase.ny} "
                      f"channel with the same cylinder recipe ({bcase.n_fluid} fluid nodes): "
                      f"10 warm-up lattice steps, then the median of 3 timings of >= 5 s "
                      f"({nst} lattice steps in all)"}
    if rank == 0 and world == 1 and emit and not args.no_extras:
        line["extra_workloads"] = _extra_workloads(args)
    if not emit:
        return line
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def _extra_workloads(args):
    """The other workloads, measured after the main line's timed region and
    reported inside it (single GPU only): BF16 storage on the same
    throughput case, the 512-case batch to the interval residual 1e-8, the
    warm start's time to steady state, and the D3Q19 extension.  Each entry
    is that workload's own line (as `--workload ...` prints it) plus its
    wall time; a workload that fails reports its error instead."""
    out = {}

    def sub(name, fn, **over):
        a = argparse.Namespace(**vars(args))
        for k, v in over.items():
            setattr(a, k, v)
        t0 = time.perf_counter()
        try:
            d = fn(a, emit=False)
            d.pop("cpu_baseline", None)
            out[name] = d
        except Exception as e:  # report, do not lose the main line
            out[name] = {"error": repr(e)[:300]}
        out[name]["wall_seconds"] = time.perf_counter() - t0

    common = dict(no_e2e=True, no_cpu_baseline=True, no_extras=True)
    sub("throughput_bf16", run_ours, precision="bf16", steps=20, **common)
    sub("batch_512_cases_tol1e-8", run_batch, precision="fp32", **common)
    sub("warmstart_tol1e-8", run_warmstart, precision="fp32", **common)
    sub("d3q19", run_d3q19, precision="fp32", steps=10, **common)
    return out


def _e2e(args, case, stream, per, world, n_fluid, lbm, torch, dev=None):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    t0 = time.perf_counter()
    mkw = {} if args.mass_mode is None else {"mass_mode": args.mass_mode}
    s2 = lbm.Solver(case, precision=args.precision, stream=stream.cuda_stream,
                    residual_every=per, **mkw)
    for _ in range(args.steps):
        s2.step(per)
        s2.residual()
    s2.fields()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    s2.close()
    (e2e_s,), (total_fluid,) = reduce_over_ranks([e2e_s], [n_fluid], world, dev)
    h2d = case.solid.nbytes + case.n_links * (3 * 4 + 3 * 8)
    d2h = 3 * 8 * case.nx * case.ny + args.steps * 2 * 8
    return {"value": total_fluid * per * args.steps / e2e_s / 1e6, "unit": "MLUPS",
            "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
            "seconds": e2e_s}


# Bumped whenever the step kernel changes, so stale ncu traffic is not reported.
KERNEL_REV = 13

# Accuracy of each storage against the FP64 oracle and the targets it
# misses, as measured by tests/test_gpu_parity.py (2000 steps from rest on
# the parity cases; the misses are asserted against the target and marked
# as known misses there).  Reported beside the throughput so that a number
# is never read as meeting a target it misses.
ACCURACY = {
    "fp32": {"velocity_target": 1e-5, "velocity": "met on every parity case (4e-8 to 3e-7)",
             "mass_target": 1e-10,
             "mass": "missed on the 40x40 rotating-wall annulus (bounded, up to 4.0e-10 over "
                     "4000 steps with the exact-mass step); met elsewhere (1-wide periodic lattices: "
                     "3.6e-10 with the plain step, 8.7e-14 with the default exact-mass step)"},
    "fp16": {"velocity_target": 1e-3,
             "velocity": "met on every parity case (2.2e-4 to 3.2e-4); missed on the 1-wide "
                         "periodic column (1.7e-3)"},
    "bf16": {"velocity_target": 1e-3, "velocity": "missed on every parity case (1.6e-3 to 7.3e-3)"},
    "fp64": {"populations": "within 1e-13 of the oracle, element by element"},
}


ACCURACY_3D = {
    "fp32": {"velocity_target": 1e-5,
             "velocity": "met (1.7e-6 to 3.6e-6 with the plain step on the 20^3 sphere array over "
                         "4000 steps; 2e-8 to 4e-8 with the exact-mass step)",
             "mass_target": 1e-10,
             "mass": "the plain step this line times (walls at rest) misses it at static curved "
                     "walls after 2000 steps (4.6e-10 on the 20^3 sphere array; 1.2e-9 after 4000); "
                     "met with mass_mode=1 (2.4e-11 after 2000 steps, at 3.7x the step time) and by "
                     "default where walls move (5.2e-11 after 2000 steps on the moving-lid channel)"},
    "fp64": {"populations": "within 1e-13 of the oracle, element by element"},
}


def _batch_roofline(precision, updates_per_s):
    """The batch's aggregate rate against the copy bandwidth: algorithmic
    bytes per fluid-node update (72 B in FP32) times updates per second over
    the whole run (step kernels, the exact-mass step of moving-wall cases,
    residual checks, retirements)."""
    peak, src = _peak_hbm()
    achieved = FLUID_BYTES[precision] * updates_per_s / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": None, "peak_source": src,
            "bytes_per_fluid_node": FLUID_BYTES[precision],
            "kernel": "the whole batched run (aggregate, not one kernel)"}


def run_batch(args, emit=True):
    """The batched workload: 512 uneven cases (sizes 64x64-1024x512, slip
    channel / annulus / cylinder array, Kn log-uniform 0.001-0.1), FP32, all
    run together to --batch-tol (default 1e-8, the workload's residual) with
    the interval residual (the mean change per step over each check
    interval; the one-step FP32 residual floors near 1e-8), capped at
    --batch-max-steps.  value = aggregate fluid-node updates per second over
    the cases still running; the line also carries the per-case steps to
    steady state and the time to steady state of a subset solved one at a
    time through the single-case solver."""
    import numpy as np
    import torch

    from paper_2012_14707_gb300 import build as lbm_build
    from paper_2012_14707_gb300 import cases, lbm

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lbm_build.build()
    lbm.load()
    cl = cases.batch_cases(args.batch_cases, seed=rank)
    prm = [{"residual_mode": 1}] * len(cl)
    t0 = time.perf_counter()
    b = lbm.Batch(cl, precision=args.precision, params=prm)
    t_create = time.perf_counter() - t0
    info = b.info()
    # warm-up: graph capture and a few hundred steps, then back to rest
    b.run_to(args.batch_tol, max(args.warmup, 1) * args.lbm_steps, check_every=args.lbm_steps)
    b.reset()
    sampler = ClockSampler(local)
    sampler.start()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps, res, total = b.run_to(args.batch_tol, args.batch_max_steps, check_every=args.lbm_steps)
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    b.close()
    nf = np.array([c.n_fluid for c in cl], np.float64)
    run = np.where(steps != 0, np.abs(steps), total).astype(np.float64)
    updates = float((nf * run).sum())
    (wall,), (updates,) = reduce_over_ranks([wall], [updates], world, dev)
    conv = steps > 0
    # time to steady state of the same cases one at a time through the
    # single-case solver, against the batch, on a subset of the cases
    comp = None
    if args.batch_single > 0:
        sub = cl[:args.batch_single]
        bs = lbm.Batch(sub, precision=args.precision, params=prm[:len(sub)])
        bs.run_to(args.batch_tol, args.lbm_steps, check_every=args.lbm_steps)
        bs.reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s_b, _, _ = bs.run_to(args.batch_tol, args.batch_max_steps, check_every=args.lbm_steps)
        t_batch = time.perf_counter() - t0
        bs.close()
        t0 = time.perf_counter()
        s_single = []
        for c in sub:
            sv = lbm.Solver(c, precision=args.precision, residual_every=args.lbm_steps,
                            residual_mode=1)
            try:
                n, r = sv.run_to(args.batch_tol, args.batch_max_steps)
                s_single.append(n if r < args.batch_tol else 0)
            except lbm.LbmError:
                s_single.append(-1)
            sv.close()
        torch.cuda.synchronize()
        t_single = time.perf_counter() - t0
        same = int(sum(1 for a, c in zip(s_b, s_single) if a == c))
        comp = {"cases": len(sub), "single_case_seconds": t_single, "batched_seconds": t_batch,
                "speedup": t_single / t_batch, "same_steps_to_steady": same,
                "note": "each case alone through lbm_create/lbm_run_to (create included) vs "
                        "all of them in one batch (create excluded), same tol and check interval"}
    line = {
        "metric": "MLUPS (batched)", "value": updates / wall / 1e6, "unit": "MLUPS",
        "n_gpus": world, "steps": int(total), "warmup": max(args.warmup, 1) * args.lbm_steps,
        "ms_per_step": wall / max(total, 1) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "bf16": "bf16", "fp16": "f16"}[args.precision],
        "data": "synthetic",
        "config": {"workload": f"batch_{len(cl)}_cases_64-1024x64-512_Kn0.001-0.1",
                   "total_nodes": info["total_nodes"], "total_fluid": info["total_fluid"],
                   "cta_threads_autotuned": info["cta_threads"], "tol": args.batch_tol,
                   "residual": "interval (mean change per step over each check interval)",
                   "max_steps": args.batch_max_steps, "check_every": args.lbm_steps},
        "batch": {"converged": int(conv.sum()), "unstable": int((steps < 0).sum()),
                  "steps_to_steady_median": float(np.median(steps[conv])) if conv.any() else None,
                  "steps_to_steady_p90": float(np.percentile(steps[conv], 90)) if conv.any() else None,
                  "not_converged_Kn_max": (float(max(c.Kn for c, ok in zip(cl, conv) if not ok))
                                           if (~conv).any() else None),
                  "create_seconds": t_create, "wall_seconds": wall,
                  # per case: the step at which it met tol (0: still running at the cap)
                  "steps_per_case": [int(v) for v in steps]},
        "time_to_steady_vs_single": comp,
        "roofline": _batch_roofline(args.precision, updates / wall),
        "clocks": clocks,
    }
    if not emit:
        return line
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


D3Q19_BYTES = {"fp32": 152, "fp64": 304}  # 19 reads + 19 writes per fluid node


def run_d3q19(args, emit=True):
    """The D3Q19 extension: a periodic 512 x 256 x 256 box of non-overlapping
    spheres (porosity 0.8, radii 6-12, seeded), Kn 0.02, force-driven, FP32
    (or FP64).  One bench step = --lbm-steps lattice steps + the residual
    pass; MLUPS over fluid nodes; roofline of the step kernel = 152 B per
    fluid node (FP32) over its mean launch time (CUDA events on the
    solver's stream).  cpu_baseline: the FP64 D3Q19 oracle (one thread) on a
    128 x 64 x 64 box of the same recipe."""
    import numpy as np
    import torch

    from paper_2012_14707_gb300 import build as lbm_build
    from paper_2012_14707_gb300 import cases, lbm

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lbm_build.build()
    lbm.load()
    nx, ny, nz = (args.nx or 512), (args.ny or 256), (args.nz or 256)
    case = cases.sphere_pack3d(nx, ny, nz, seed=rank, porosity=0.8, r_range=(6.0, 12.0),
                               Kn=0.02, a=(1e-6, 0.0, 0.0))
    stream = torch.cuda.current_stream(dev)
    prec = args.precision if args.precision in D3Q19_BYTES else "fp32"
    mkw = {} if args.mass_mode is None else {"mass_mode": args.mass_mode}
    sv = lbm.Solver3D(case, precision=prec, stream=stream.cuda_stream, **mkw)
    # the sphere pack's walls are at rest: the exact-mass step only on request
    exact3 = prec == "fp32" and args.mass_mode == 1
    per = args.lbm_steps
    n_fluid = case.n_fluid
    for _ in range(args.warmup):
        sv.step(per)
        sv.residual()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    k_start = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    k_end = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    last = None
    for s in range(args.steps):
        k_start[s].record(stream)
        sv.step(per)
        k_end[s].record(stream)
        last = sv.residual()
    t_end.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    elapsed_ms = t_start.elapsed_time(t_end)
    kernel_ms = sum(a.elapsed_time(b) for a, b in zip(k_start, k_end))
    (elapsed_ms, kernel_ms), (total_fluid,) = reduce_over_ranks([elapsed_ms, kernel_ms], [n_fluid],
                                                                world, dev)
    sv.close()
    mlups = total_fluid * per * args.steps / (elapsed_ms / 1e3) / 1e6
    launch_ms = kernel_ms / (args.steps * per)
    # the exact-mass step also reads and writes a carry per fluid node and
    # per link (4 B each way)
    node_bytes = D3Q19_BYTES[prec] + (8 + 8 * case.n_links / n_fluid if exact3 else 0)
    achieved = node_bytes * n_fluid / (launch_ms / 1e3) / 1e9
    step_achieved = node_bytes * mlups * 1e6 / world / 1e9
    peak, peak_src = _peak_hbm()
    line = {
        "metric": "MLUPS (D3Q19)", "value": mlups, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64"}[prec], "data": "synthetic",
        "config": {"workload": f"spheres3d_{nx}x{ny}x{nz}_phi0.8_Kn0.02", "nx": nx, "ny": ny,
                   "nz": nz, "n_fluid": n_fluid, "n_links": case.n_links,
                   "n_spheres": case.meta["n_spheres"], "precision": prec,
                   "lattice_steps_per_step": per, "exact_mass_step": exact3,
                   "l2": "inputs larger than L2 (2 x %.2f GB dense lattices)" % (
                       19 * nx * ny * nz * D3Q19_BYTES[prec] / 38 / 1e9),
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "step3_kernel<float, true> (exact-mass; issue-bound, d - d_eq in "
                               "double-FP32)" if exact3 else "step3_kernel",
                     "bytes_per_fluid_node": node_bytes, "launch_ms": launch_ms,
                     "peak_source": peak_src, "step_achieved": step_achieved,
                     "step_frac": step_achieved / peak},
        "e2e": None,
        "gpu_launches": args.steps * (per + 2),
        "clocks": clocks,
        "residual_last": last[0] if last else None,
        "accuracy_vs_oracle": ACCURACY_3D[prec],
    }
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        from oracle import params as P
        sc = cases.sphere_pack3d(128, 64, 64, seed=0, porosity=0.8, r_range=(6.0, 12.0),
                                 Kn=0.02, a=(1e-6, 0.0, 0.0))
        o = oracle.OracleLBM3D(sc, P.Parameters(sc.Kn, sc.H))
        o.step(2)
        t0 = time.perf_counter()
        n = 0
        while time.perf_counter() - t0 < 5.0:
            o.step(1)
            n += 1
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {
            "value": sc.n_fluid * n / dt / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "sample": f"FP64 D3Q19 oracle (one thread) on a 128x64x64 box of the same recipe "
                      f"({sc.n_fluid} fluid nodes): 2 warm-up steps, then {n} steps in {dt:.1f} s"}
    if not emit:
        return line
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_warmstart(args, emit=True):
    """The learned warm start (256 x 256 random-cylinder channels, Kn
    log-uniform 0.001-0.1, FP32 solves to the interval residual 1e-8): the
    network is trained on --ws-train seeded cases solved by the batched
    solver, then --ws-test held-out seeds are solved three ways and timed to
    steady state (creation, and for the warm start the network's inference
    and lbm_set_fields, included): in one batch started from the network's
    fields, in one batch started from rest, and one case at a time through
    the single-case solver from rest.  value = the time to steady state of
    the batched + warm-start run."""
    import numpy as np
    import torch

    from paper_2012_14707_gb300 import build as lbm_build
    from paper_2012_14707_gb300 import lbm
    from paper_2012_14707_gb300 import warmstart as ws

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    lbm_build.build()
    lbm.load()
    tol, cap, every, size = args.batch_tol, 40000, 100, 256
    t0 = time.perf_counter()
    data = ws.make_dataset(args.ws_train, 1 + 1000000 * rank, size, tol, cap)
    t_data = time.perf_counter() - t0
    net = lbm.Net(size, size, base=32, levels=4, precision="bf16", max_batch=8, seed=0)
    t0 = time.perf_counter()
    ws.train(net, data, args.ws_epochs, 8, 2e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    held = ws.make_cases(args.ws_test, 100000 + 1000000 * rank, size)
    prm = [{"residual_mode": 1}] * len(held)
    # warm-up of the batched path (graph capture, allocator) on two cases
    b = lbm.Batch(held[:2], precision="fp32", params=prm[:2])
    b.run_to(tol, 2 * every, every)
    b.close()
    sampler = ClockSampler(local)
    sampler.start()
    runs = {}
    for mode in ("warm", "rest"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        preds = ws.predict(net, held, 8) if mode == "warm" else None
        t_inf = time.perf_counter() - t0
        b = lbm.Batch(held, precision="fp32", params=prm)
        if preds is not None:
            for k, (rho, ux, uy) in enumerate(preds):
                b.set_fields(k, rho, ux, uy)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        steps, _, total = b.run_to(tol, cap, every)
        torch.cuda.synchronize()
        t_end = time.perf_counter()
        b.close()
        runs[mode] = dict(seconds=t_end - t0, solve_seconds=t_end - t1, inference_seconds=t_inf,
                          steps=steps, total=int(total))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    single = []
    for c in held:
        sv = lbm.Solver(c, precision="fp32", residual_every=every, residual_mode=1)
        try:
            n, r = sv.run_to(tol, cap)
            single.append(n if r < tol else 0)
        except lbm.LbmError:
            single.append(-1)
        sv.close()
    torch.cuda.synchronize()
    t_single = time.perf_counter() - t0
    clocks = sampler.stop()
    single = np.array(single)
    w, r_ = runs["warm"]["steps"], runs["rest"]["steps"]
    both = (w > 0) & (r_ > 0)
    line = {
        "metric": "time to steady state (batched + warm start)", "value": runs["warm"]["seconds"],
        "unit": "s", "n_gpus": world, "steps": int(runs["warm"]["total"]), "warmup": 2 * every,
        "ms_per_step": runs["warm"]["solve_seconds"] / max(runs["warm"]["total"], 1) * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"warmstart_{len(held)}_heldout_cylinders_{size}x{size}_Kn0.001-0.1",
                   "tol": tol, "residual": "interval (mean change per step over each check interval)",
                   "max_steps": cap, "check_every": every, "train_cases": args.ws_train,
                   "train_converged": len(data.cases), "epochs": args.ws_epochs,
                   "net": "unet4_base32 bf16", "l2": "whole batch (%.0f MB lattices) above L2" % (
                       2 * 9 * 4 * sum(c.n_fluid for c in held) / 1e6)},
        "time_to_steady": {
            "batched_warm_start_s": runs["warm"]["seconds"],
            "batched_from_rest_s": runs["rest"]["seconds"],
            "single_case_from_rest_s": t_single,
            "warm_inference_s": runs["warm"]["inference_seconds"],
            "converged": {"warm": int((w > 0).sum()), "rest": int((r_ > 0).sum()),
                          "single": int((single > 0).sum())},
            "median_steps": {"warm": float(np.median(w[both])) if both.any() else None,
                             "rest": float(np.median(r_[both])) if both.any() else None},
            "median_step_ratio": float(np.median(w[both] / r_[both])) if both.any() else None,
            "step_ratio_quartiles": ([float(v) for v in np.percentile(w[both] / r_[both], [25, 75])]
                                     if both.any() else None),
            "single_same_steps_as_batch": int((single == r_).sum()),
            "note": "creation included in every arm; warm start includes inference and "
                    "lbm_set_fields; training excluded (data %.0f s, training %.0f s)" % (
                        t_data, t_train)},
        "e2e": None,
        "clocks": clocks,
    }
    net.close()
    if not emit:
        return line
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def net_flops(H, W, base=32, levels=4, c_in=3, c_out=3):
    """Multiply-adds x 2 of one forward pass of the warm-start network on one
    H x W sample (every convolution; pooling and upsampling are negligible)."""
    f = 0
    prev = c_in
    for l in range(levels):
        hw = (H >> l) * (W >> l)
        ch = base << l
        f += 2 * hw * 9 * prev * ch + 2 * hw * 9 * ch * ch
        prev = ch
    for l in range(levels - 2, -1, -1):
        hw = (H >> l) * (W >> l)
        ch = base << l
        f += 2 * hw * 9 * (prev + ch) * ch + 2 * hw * 9 * ch * ch
        prev = ch
    f += 2 * H * W * prev * c_out
    return f


def run_net(args, emit=True):
    """The warm-start network's training step (256 x 256, batch 8, BF16
    storage, FP32 accumulation; convolutions of the forward pass and of the
    backward data pass on the tensor cores): TFLOP/s of the whole step
    (forward + backward + Adam) against the measured dense BF16 peak."""
    import torch

    from paper_2012_14707_gb300 import build as lbm_build
    from paper_2012_14707_gb300 import lbm

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lbm_build.build()
    lbm.load()
    H = W = 256
    B = 8
    net = lbm.Net(H, W, base=32, levels=4, precision="bf16", max_batch=B, seed=rank)
    g = torch.Generator(device="cuda").manual_seed(rank)
    x = torch.randn((B, H, W, 3), device="cuda", generator=g)
    t = torch.randn((B, H, W, 3), device="cuda", generator=g)
    for _ in range(max(args.warmup, 3)):
        net.train_step(x.data_ptr(), t.data_ptr(), B, 1e-4)
    torch.cuda.synchronize()
    steps = max(args.steps // 10, 5)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local)
    sampler.start()
    e0.record()
    for _ in range(steps):
        net.train_step(x.data_ptr(), t.data_ptr(), B, 1e-4)
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / steps
    e0.record()
    y = torch.empty((B, H, W, 3), device="cuda")
    for _ in range(steps):
        net.forward(x.data_ptr(), B, y.data_ptr())
    e1.record()
    torch.cuda.synchronize()
    ms_fwd = e0.elapsed_time(e1) / steps
    fwd = net_flops(H, W) * B
    (ms, ms_fwd), (n_rank,) = reduce_over_ranks([ms, ms_fwd], [1.0], world, dev)
    fwd = fwd * n_rank  # every rank trains its own replica: the job's flops
    peak, src = _peak_bf16()
    peak *= n_rank
    line = {"metric": "TFLOP/s (warm-start network training step)", "value": 3 * fwd / ms / 1e9,
            "unit": "TFLOP/s", "n_gpus": world, "steps": steps, "warmup": max(args.warmup, 3),
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "unet4_base32_256x256_batch8", "flop_per_step": 3 * fwd,
                       "note": "3 x forward flops (forward, backward data, backward weights)"},
            "forward": {"ms": ms_fwd, "tflops": fwd / ms_fwd / 1e9},
            "roofline": {"bound": "tensor", "achieved": 3 * fwd / ms / 1e9, "peak": peak,
                         "unit": "TFLOP/s", "frac": 3 * fwd / ms / 1e9 / peak, "traffic": None,
                         "peak_source": src},
            "clocks": clocks}
    if not emit:
        return line
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--precision", choices=("fp32", "fp64", "bf16", "fp16"), default="fp32")
    ap.add_argument("--mass-mode", type=int, choices=(-1, 0, 1), default=None,
                    help="FP32 params.mass_mode (default: the library's, 0); 1 times the "
                         "exact-mass step")
    ap.add_argument("--lbm-steps", type=int, default=100,
                    help="lattice steps per benchmark step (the residual interval)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other workloads reported inside the default line")
    ap.add_argument("--workload", choices=("throughput", "batch", "net", "d3q19", "warmstart"),
                    default="throughput")
    ap.add_argument("--batch-cases", type=int, default=512)
    ap.add_argument("--batch-max-steps", type=int, default=50000)
    ap.add_argument("--batch-single", type=int, default=32,
                    help="cases also solved one at a time for the time-to-steady comparison")
    ap.add_argument("--batch-tol", type=float, default=1e-8,
                    help="interval residual to reach (the batched workload's 1e-8)")
    ap.add_argument("--nx", type=int, default=0, help="profiling only: smaller lattice width")
    ap.add_argument("--ny", type=int, default=0, help="profiling only: smaller lattice height")
    ap.add_argument("--nz", type=int, default=0, help="profiling only: smaller D3Q19 lattice depth")
    ap.add_argument("--ws-train", type=int, default=512, help="warm start: training cases")
    ap.add_argument("--ws-test", type=int, default=200, help="warm start: held-out cases")
    ap.add_argument("--ws-epochs", type=int, default=20, help="warm start: training epochs")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "net":
        return run_net(args)
    if args.workload == "d3q19":
        return run_d3q19(args)
    if args.workload == "warmstart":
        return run_warmstart(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
