#!/usr/bin/env python3
"""Throughput of the direction-split exponential integrator on a GB300.

One bench "step" is one time step of the integrator over the whole state: the
K u + g prepass, the Tucker operator(s) with phi_l(tau A_mu) and the fused FP64
update (Section 3.2).  Default workload: 3D advection-diffusion-reaction,
n = 128 per direction (N = 2,097,152), ETD2RK with split phi_1 and phi_2,
tau = 1e-3, plain FP64.  Metric: DOF-steps/s = N * steps / device time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME] [--prec fp64|tf32x3]

Under torchrun (N > 1) every rank advances its own replica of the workload on its
own GPU (the single-tensor path has no data-parallel split; replicas only): the
timed region is bracketed by barriers, the time is the max over ranks and the
value is the DOF-steps of all ranks over that time.  ``--impl reference`` times
the FP64 CPU oracle on the host cores (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2304_02327_gb300 import parallel, workloads as wl  # noqa: E402

METRIC = "DOF-steps/s"
L2_FLUSH_BYTES = 512 << 20          # > 126 MB L2, written between timed steps
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12   # 152 SMs x 4 FP64 flop/clk x 2.07 GHz
CUBLAS_DGEMM_TFLOPS_MEASURED = 1.10          # torch.matmul float64 8192^3 on this pool
TF32_NOMINAL_RATIO = 1.1 / 2.25                # nominal dense TF32 / BF16 tensor rate


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="adr3d_n128_etd2rk")
    ap.add_argument("--prec", default="fp64", choices=["fp64", "tf32x3", "bf16x3"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="target CPU time of the oracle cpu_baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nc-cap", type=int, default=0,
                    help="batched workloads: use this tile width instead of autotuning it "
                         "(160, 128, 96 or 64; a profiler run then sees the plain run's tiling)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2304_02327_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def profile_traffic(kernel_tag, workload):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the
    current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", f"{kernel_tag}_{workload}.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("source_hash") != source_hash():
        return None
    try:
        return float(kv["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms in the background."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def run_oracle_sample(problem, seconds):
    """The FP64 oracle as it stands on a bounded number of steps from u0."""
    from oracle.integrators import OracleProblem, step
    op = OracleProblem.from_problem(problem)
    U = np.array(problem.u0, dtype=np.float64)
    t0 = time.perf_counter()
    steps = 0
    while steps < problem.steps:
        U = step(op, U, problem.scheme, steps * problem.tau)
        steps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return U, steps, dt


def reference_arm(args):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    if args.workload in wl.BATCHED:
        probs = wl.batched_workload(args.workload)
        cb = oracle_batch_sample(probs, args.cpu_seconds)
        line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": METRIC,
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": args.workload, "precision": "fp64"},
                "cpu_baseline": cb,
                "e2e": {"value": cb["value"], "unit": METRIC, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0
    p = wl.workload(args.workload)
    from oracle.integrators import OracleProblem, step
    op = OracleProblem.from_problem(p)
    U = np.array(p.u0, dtype=np.float64)
    for k in range(args.warmup):
        U = step(op, U, p.scheme, k * p.tau)
    t0 = time.perf_counter()
    for k in range(args.steps):
        U = step(op, U, p.scheme, (args.warmup + k) * p.tau)
    dt = time.perf_counter() - t0
    value = p.N * args.steps / dt
    cores = host_cores()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n": p.n, "N": p.N,
                   "scheme": wl.SCHEME_NAMES[p.scheme], "tau": p.tau, "precision": "fp64"},
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle",
                         "sample": f"{args.warmup}+{args.steps} steps of {args.workload} "
                                   f"(numpy float64, BLAS threads up to {cores})"},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def tensor_peak(prec):
    """(peak TFLOP/s, note) of the form's tensor-core dtype, from the measured BF16 peak."""
    bf16 = float(measured_peaks().get("bf16_tflops", 1900.0))
    if prec == "tf32x3":
        return bf16 * TF32_NOMINAL_RATIO, (f"TF32 dense peak = measured bf16 {bf16:.1f} TFLOP/s "
                                           "(MEASURED_PEAKS.json) x nominal TF32/BF16 ratio 1.1/2.25")
    return bf16, f"BF16 dense peak measured {bf16:.1f} TFLOP/s (MEASURED_PEAKS.json)"


def ours_batched(args):
    """Config 4: many independent 2D Allen-Cahn problems in one batch (mixed form)."""
    import torch
    import torch.distributed as dist
    from paper_2304_02327_gb300 import api

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    api.lib()
    prec = args.prec if args.prec != "fp64" else "bf16x3"
    probs_all = wl.batched_workload(args.workload)
    costs = [parallel.instance_cost(p.n[0]) for p in probs_all]
    mine = parallel.shard_for_rank(costs, rank, world)       # LPT shard, no collective
    probs = [probs_all[i] for i in mine]
    dof = sum(p.u0.size for p in probs)
    dof_all = sum(p.u0.size for p in probs_all)

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plans, gs, Us = api.setup_batch(probs, prec)
    if args.nc_cap:
        b = api.Batch(plans, gs, Us, autotune=False, nc_cap=args.nc_cap, graph=True)
    else:
        b = api.Batch(plans, gs, Us, autotune=True, graph=True)
    torch.cuda.synchronize()
    plan_ms = 1e3 * (time.perf_counter() - t0)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        b.run(1)
    torch.cuda.synchronize()

    # ---- timed region: K steps, one graph launch each, L2 flushed between ----
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    api.trace_enable(False)
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        starts[k].record(stream)
        b.run(1)
        ends[k].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    launches = {c: api.trace_read(c, timed=False)[0] for c in (api.KC_CONTRACT_TF32, api.KC_PREPASS,
                                                                api.KC_SPLIT)}
    assert b.status() == 0, "non-finite state during the timed steps"
    t_ms = parallel.max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(starts, ends)), device="cuda")
    value = parallel.job_throughput([dof_all * args.steps], t_ms / 1e3)

    # ---- per-kernel device times: the same launches, eager and traced ----
    bp = api.Batch(plans, gs, Us, autotune=False, nc_cap=b.info()["nc_cap"], graph=False)
    bp.run(1)
    torch.cuda.synchronize()
    api.trace_enable(True)
    ksteps = min(args.steps, 5)
    for k in range(ksteps):
        flush.fill_(k & 0xff)
        bp.run(1)
    torch.cuda.synchronize()
    n_launch, k_ms = api.trace_read(api.KC_CONTRACT_TF32)
    _, pre_ms = api.trace_read(api.KC_PREPASS)
    _, upd_ms = api.trace_read(api.KC_SPLIT)
    api.trace_enable(False)
    bp.close()

    # ---- e2e: every state in from pinned host memory, one step, every state out ----
    hosts = [torch.from_numpy(np.ascontiguousarray(p.u0)).pin_memory() for p in probs]
    e2e_steps = min(args.steps, 5)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for k in range(e2e_steps):
        for h, u in zip(hosts, Us):
            u.copy_(h, non_blocking=True)
        b.run(1)
        for h, u in zip(hosts, Us):
            h.copy_(u, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = parallel.max_over_ranks(e0.elapsed_time(e1), device="cuda")
    e2e_value = parallel.job_throughput([dof_all * e2e_steps], e2e_ms / 1e3)

    # ---- the per-instance FP64 GPU loop on the same shard, for comparison ----
    fp_plans, fp_gs, fp_Us = api.setup_batch(probs, "fp64")
    fp_ws = [api.expint_workspace(pl, wl.EXPEULER, g) for pl, g in zip(fp_plans, fp_gs)]
    for pl, g, u, w in zip(fp_plans, fp_gs, fp_Us, fp_ws):
        api.expint_step(pl, wl.EXPEULER, u, 1, g=g, ws=w)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fsteps = 2
    f0.record(stream)
    for k in range(fsteps):
        for pl, g, u, w in zip(fp_plans, fp_gs, fp_Us, fp_ws):
            api.expint_step(pl, wl.EXPEULER, u, 1, g=g, ws=w)
    f1.record(stream)
    torch.cuda.synchronize()
    fp_ms = parallel.max_over_ranks(f0.elapsed_time(f1), device="cuda") / fsteps
    del fp_plans, fp_gs, fp_Us, fp_ws

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    nprod = 4 if prec == "tf32x3" else 6
    # logical flops of one grouped launch (one direction of every instance): 2 N_j n_mu
    flops_launch = sum(2.0 * p.u0.size * p.n[0] for p in probs)
    k_avg = k_ms / n_launch if n_launch else None
    peak, note = tensor_peak(prec)
    achieved = nprod * flops_launch / (k_avg / 1e3) / 1e12 if k_avg else None
    info = b.info()
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": f"{prec}+f64", "data": "synthetic",
        "config": {"workload": args.workload, "instances": len(probs_all), "dof": dof_all,
                   "sizes": "n uniform over {48, 64, ..., 512}, square", "scheme": "expeuler",
                   "tau": probs_all[0].tau, "precision": prec, "size_classes": info["classes"],
                   ("nc_cap_pinned" if args.nc_cap else "nc_cap_autotuned"): info["nc_cap"], "tiles_per_mode": info["tiles_mode1"],
                   "graph": "one CUDA graph launch per step (4 kernels)",
                   "l2": "flushed between timed steps (512 MB write); states 0.8 GB > L2",
                   "parallelism": f"LPT shard of instances x{world}"},
        "plan_ms": plan_ms,
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak if achieved else None,
                     "traffic": None,
                     "kernel": "tc_mode_kernel (grouped tcgen05 mu-mode contraction, all instances)",
                     "launches": n_launch, "avg_launch_ms": k_avg,
                     "share_of_step_time": (k_ms / ksteps) / (t_ms / args.steps) if k_ms else None,
                     "flops_per_launch": nprod * flops_launch,
                     "timing": "eager traced run of the same launches (a graph replay has no "
                               "per-kernel events)",
                     "peak_note": note},
        "elementwise_ms_per_step": {"prepass": pre_ms / ksteps, "update": upd_ms / ksteps},
        "fp64_per_instance_loop": {"ms_per_step": fp_ms, "value": dof_all / (fp_ms / 1e3),
                                   "unit": METRIC, "speedup_of_batch": fp_ms / (t_ms / args.steps)},
        "e2e": {"value": e2e_value, "unit": METRIC, "steps": e2e_steps,
                "h2d_bytes_per_step": dof * 8, "d2h_bytes_per_step": dof * 8},
        "gpu_launches": sum(launches.values()),
        "launches_by_kernel": {"contract_tf32": launches[api.KC_CONTRACT_TF32],
                               "prepass": launches[api.KC_PREPASS], "update": launches[api.KC_SPLIT]},
        "clocks": clk,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_batch_sample(probs_all, args.cpu_seconds)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def oracle_batch_sample(probs, seconds):
    """The FP64 oracle on a bounded sample of the batch: whole instances (in the
    batch's order, one step each) until the time is spent."""
    from oracle.integrators import OracleProblem, step
    t0 = time.perf_counter()
    dof = 0
    k = 0
    while k < len(probs) and time.perf_counter() - t0 < seconds:
        p = probs[k]
        op = OracleProblem.from_problem(p, lmax=1)
        step(op, np.array(p.u0, dtype=np.float64), p.scheme, 0.0)
        dof += p.u0.size
        k += 1
    dt = time.perf_counter() - t0
    return {"value": dof / dt, "unit": METRIC, "cores": host_cores(), "kind": "oracle",
            "sample": f"one step of each of the first {k} instances (phi set-up included, "
                      f"numpy float64, {dt:.1f} s)"}


def ours(args):
    import torch
    import torch.distributed as dist
    from paper_2304_02327_gb300 import api

    if args.workload in wl.BATCHED:
        return ours_batched(args)
    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    api.lib()
    p = wl.workload(args.workload)
    N = p.N

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan, g, U = api.setup(p, args.prec)
    torch.cuda.synchronize()
    plan_ms = 1e3 * (time.perf_counter() - t0)
    ws = api.expint_workspace(plan, p.scheme, g)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    for k in range(args.warmup):
        api.expint_step(plan, p.scheme, U, 1, t0=k * p.tau, g=g, ws=ws)
    torch.cuda.synchronize()

    # ---- timed region: K steps (each one replay of the step's captured graph),
    # events per step, L2 flushed between steps; launches counted ----
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    api.trace_enable(False)
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        starts[k].record(stream)
        api.expint_step(plan, p.scheme, U, 1, t0=(args.warmup + k) * p.tau, g=g, ws=ws)
        ends[k].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    counts = {c: api.trace_read(c, timed=False)[0] for c in (api.KC_CONTRACT_FP64, api.KC_CONTRACT_TF32,
                                                             api.KC_PREPASS, api.KC_SPLIT)}
    assert plan.status() == 0, "non-finite state during the timed steps"
    t_ms = parallel.max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(starts, ends)), device="cuda")
    value = parallel.job_throughput([N * args.steps] * world, t_ms / 1e3)

    # ---- per-kernel device times: the same steps launched directly, each launch
    # bracketed by events on its stream (a graph replay has no per-kernel events) ----
    ksteps = min(args.steps, 10)
    api.trace_enable(True)
    for k in range(ksteps):
        flush.fill_(k & 0xff)
        api.expint_step(plan, p.scheme, U, 1, t0=(args.warmup + args.steps + k) * p.tau, g=g, ws=ws)
    torch.cuda.synchronize()
    launches = {c: api.trace_read(c) for c in (api.KC_CONTRACT_FP64, api.KC_CONTRACT_TF32,
                                              api.KC_PREPASS, api.KC_SPLIT)}
    api.trace_enable(False)

    # ---- e2e: pinned host state in, one step, state out, every step ----
    U_host = torch.from_numpy(np.ascontiguousarray(p.u0)).pin_memory()
    U_dev = torch.empty_like(U)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = min(args.steps, 20)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for k in range(e2e_steps):
        U_dev.copy_(U_host, non_blocking=True)
        api.expint_step(plan, p.scheme, U_dev, 1, t0=k * p.tau, g=g, ws=ws)
        U_host.copy_(U_dev, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = parallel.max_over_ranks(e0.elapsed_time(e1), device="cuda")
    e2e_value = parallel.job_throughput([N * e2e_steps] * world, e2e_ms / 1e3)

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    # ---- roofline of the dominant kernel (the mu-mode contraction) ----
    tf32 = args.prec in ("tf32x3", "bf16x3")
    kc = api.KC_CONTRACT_TF32 if tf32 else api.KC_CONTRACT_FP64
    n_launch, k_ms = launches[kc]
    flops_per_launch = 2.0 * N * (sum(p.n) / len(p.n))   # 2 N n_mu per mode product
    achieved = flops_per_launch / (k_ms / n_launch / 1e3) / 1e12 if n_launch else None
    total_launches = sum(counts.values())
    if tf32:
        peaks = {}
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except Exception:
            pass
        bf16 = float(peaks.get("bf16_tflops", 1900.0))
        peak = bf16 * TF32_NOMINAL_RATIO if args.prec == "tf32x3" else bf16
        # MMA products per mode: TF32x3 4 (a0b0 a1b0 a0b1 a0b2), BF16x3 6 (+ a2b0 a1b1)
        nprod = 4 if args.prec == "tf32x3" else 6
        tflops = nprod * flops_per_launch
        achieved = tflops / (k_ms / n_launch / 1e3) / 1e12 if n_launch else None
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if achieved else None,
                "traffic": profile_traffic(f"contract_{args.prec}", args.workload),
                "kernel": "tf32x3_mode_kernel (tcgen05 mu-mode contraction)",
                "launches": n_launch, "avg_launch_ms": k_ms / n_launch if n_launch else None,
                "share_of_step_time": (k_ms / ksteps) / (t_ms / args.steps) if t_ms else None,
                "timing": f"eager traced run of {ksteps} steps (the timed steps replay a CUDA graph)",
                "flops_per_launch": tflops,
                "peak_note": (f"TF32 dense peak = measured bf16 {bf16:.1f} TFLOP/s (MEASURED_PEAKS.json) "
                              "x nominal TF32/BF16 ratio 1.1/2.25") if args.prec == "tf32x3" else
                             f"BF16 dense peak measured {bf16:.1f} TFLOP/s (MEASURED_PEAKS.json)"}
    else:
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS if achieved else None,
                "traffic": profile_traffic("contract_fp64", args.workload),
                "kernel": "dgemm_kernel (FP64 mu-mode contraction)",
                "launches": n_launch, "avg_launch_ms": k_ms / n_launch if n_launch else None,
                "share_of_step_time": (k_ms / ksteps) / (t_ms / args.steps) if t_ms else None,
                "timing": f"eager traced run of {ksteps} steps (the timed steps replay a CUDA graph)",
                "flops_per_launch": flops_per_launch,
                "peak_note": "FP64 peak derived: 152 SMs x 4 flop/clk x 2.07 GHz (nominal 1.25 "
                             f"TFLOP/s); cuBLAS DGEMM measured {CUBLAS_DGEMM_TFLOPS_MEASURED} TFLOP/s"}

    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.prec == "fp64" else f"{args.prec}+f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "n": p.n, "N": N,
                   "scheme": wl.SCHEME_NAMES[p.scheme], "tau": p.tau, "precision": args.prec,
                   "l2": "flushed between timed steps (512 MB write)",
                   "parallelism": f"replicas x{world}"},
        "plan_ms": plan_ms,
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": METRIC, "steps": e2e_steps,
                "h2d_bytes_per_step": N * 8, "d2h_bytes_per_step": N * 8},
        "gpu_launches": total_launches,
        "kernel_ms_per_step": {"contract": k_ms / ksteps,
                               "prepass": launches[api.KC_PREPASS][1] / ksteps,
                               "split_update": launches[api.KC_SPLIT][1] / ksteps},
        "launches_by_kernel": {"contract_fp64": counts[api.KC_CONTRACT_FP64],
                               "contract_tf32": counts[api.KC_CONTRACT_TF32],
                               "prepass": counts[api.KC_PREPASS],
                               "split": counts[api.KC_SPLIT]},
        "graph": "each timed step is one replay of the step's captured CUDA graph",
        "clocks": clk,
    }

    if not args.no_cpu_baseline:
        # GPU run of the same bounded sample from u0, for the relative error.
        Uo, osteps, odt = run_oracle_sample(p, args.cpu_seconds)
        plan2, g2, Ug = api.setup(p, args.prec)
        api.expint_step(plan2, p.scheme, Ug, osteps, g=g2)
        torch.cuda.synchronize()
        from oracle.integrators import rel_err_inf, rel_err_fro
        got = Ug.cpu().numpy()
        line["rel_err_vs_oracle"] = {"steps": osteps, "inf": rel_err_inf(got, Uo),
                                     "fro": rel_err_fro(got, Uo)}
        line["cpu_baseline"] = {"value": N * osteps / odt, "unit": METRIC, "cores": host_cores(),
                                "kind": "oracle",
                                "sample": f"first {osteps} of {p.steps} steps of {args.workload} "
                                          f"from u0 (numpy float64 oracle, {odt:.1f} s)"}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    return ours(args)


if __name__ == "__main__":
    sys.exit(main())
