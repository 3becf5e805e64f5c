#!/usr/bin/env python3
"""Throughput of the direction-split exponential integrator on a GB300.

One bench "step" is one time step of the integrator over the whole state: the
K u + g prepass, the Tucker operator(s) with phi_l(tau A_mu) and the FP64 update
(Section 3.2).  Metric: DOF-steps/s = N * steps / device time, at the relative
error against the FP64 oracle stated in the same line.

Default workload: 3D advection-diffusion-reaction at n = 320 per direction
(N = 32,768,000; 262 MB per FP64 state), ETD2RK with split phi_1 and phi_2,
tau = 1e-3, 100 steps, the largest single-tensor configuration.  The line's
`value` is the plain FP64 form (the paper's arithmetic); beside it

  mixed    the split-precision tensor-core forms (BF16x3, TF32x3) on the same
           workload: DOF-steps/s, speed-up over the FP64 form, the contraction's
           roofline (tensor pipe over the split products, the logical flops, HBM),
           and their error: the full 100-step run against the FP64 GPU run, and
           the last step taken from the FP64 state against the oracle's step on a
           seeded sample of output entries;
  batched  1024 independent 2D Allen-Cahn problems of uneven size (n in {48, 64,
           ..., 512}) in one graph-captured batch (BF16x3), against the
           per-instance FP64 GPU loop, with sampled instances checked against the
           oracle.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME] [--prec fp64|tf32x3|bf16x3] [--mixed LIST]
                    [--batch NAME|none] [--no-accuracy] [--no-cpu-baseline]

Under torchrun (N > 1) every rank advances its own replica of the single-tensor
workload (it has no data-parallel split; replicas only) and its LPT share of the
batch's instances; the timed regions are bracketed by barriers, times are the max
over ranks and values count the DOF-steps of all ranks.  ``--impl reference``
times the FP64 CPU oracle on the host cores (rank 0 only), one full oracle step per
bench step.
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
L2_BYTES = 129 * 10**6        # GB300 L2 (a state above it is not L2-resident between steps)
E2E_BUFS = 3                  # e2e pipeline depth: a buffer's copy in, step, copy out in flight
DEFAULT_WORKLOAD = "adr3d_n320_etd2rk"
DEFAULT_BATCH = "batch_ac2d_1024_expeuler"
# The other measured configurations, recorded beside the headline in every form:
# 2D Allen-Cahn n = 64 (exp. Euler), 3D ADR n = 128 (ETD2RK), matrix Riccati
# n = 2048 (exp. Euler and ETD2RK).
OTHER_CONFIGS = ("ac2d_n64_expeuler", "adr3d_n128_etd2rk", "riccati_n2048_expeuler", "riccati_n2048_etd2rk")
# whose whole run the oracle finishes in seconds on the host cores
ORACLE_WHOLE_RUN = ("ac2d_n64_expeuler", "adr3d_n128_etd2rk")
L2_FLUSH_BYTES = 512 << 20          # > 126 MB L2, written between timed steps
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12   # 152 SMs x 4 FP64 flop/clk x 2.07 GHz
TF32_NOMINAL_RATIO = 1.1 / 2.25                # nominal dense TF32 / BF16 tensor rate
NPROD = {"tf32x3": 4, "bf16x3": 6}             # MMA products per split contraction
ELEM = {"tf32x3": 4, "bf16x3": 2}              # bytes of one operand part element
PARTS = {"tf32x3": 2, "bf16x3": 3}             # parts of a tensor operand

# The sources each profiled kernel is built from: a committed traffic summary is
# used only while their hash matches the one recorded in it.
CSRC = os.path.join(ROOT, "paper_2304_02327_gb300", "csrc")
KERNEL_SOURCES = {
    "contract_fp64": ["dgemm.cu", "common.cuh"],
    "contract_tf32x3": ["tf32.cu", "tf32.cuh", "tcgen05.cuh", "forms.cuh", "mixed.cuh", "common.cuh"],
    "contract_bf16x3": ["tf32.cu", "tf32.cuh", "tcgen05.cuh", "forms.cuh", "mixed.cuh", "common.cuh"],
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--prec", default="fp64", choices=["fp64", "tf32x3", "bf16x3"],
                    help="form of the headline value")
    ap.add_argument("--mixed", default="bf16x3,tf32x3",
                    help="further forms recorded beside the headline ('none' for none)")
    ap.add_argument("--batch", default=DEFAULT_BATCH,
                    help="batched workload recorded beside the headline ('none' to skip)")
    ap.add_argument("--batch-prec", default="bf16x3", choices=["tf32x3", "bf16x3"])
    ap.add_argument("--configs", default="all",
                    help="record the other configurations too ('all' or 'none')")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the error records (full run vs FP64, sampled step vs oracle)")
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


def source_hash(files):
    h = hashlib.sha256()
    for f in sorted(files):
        path = os.path.join(CSRC, f)
        if os.path.exists(path):
            with open(path, "rb") as fh:
                h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def profile_traffic(kernel_tag, workload):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the
    current sources of that kernel (else None)."""
    path = os.path.join(ROOT, "profiles", f"{kernel_tag}_{workload}.txt")
    if not os.path.exists(path) or kernel_tag not in KERNEL_SOURCES:
        return None
    kv = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("source_hash") != source_hash(KERNEL_SOURCES[kernel_tag]):
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


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def library_gemm_tflops():
    """Context for the roofline denominators, measured live: cuBLAS GEMM throughput
    through torch.matmul in FP64 (4096^3), TF32 and BF16 (8192^3), median of 5 each.
    (The FP64 peak used as denominator stays the unit-count derivation and the TF32 one
    the measured BF16 peak x the nominal ratio.)"""
    import torch
    out = {}
    for name, n, dt, tf32 in (("fp64", 4096, torch.float64, False), ("tf32", 8192, torch.float32, True),
                              ("bf16", 8192, torch.bfloat16, False)):
        old = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn(n, n, device="cuda", dtype=torch.float32).to(dt)
        b = torch.randn(n, n, device="cuda", dtype=torch.float32).to(dt)
        torch.matmul(a, b)
        ts = []
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        torch.backends.cuda.matmul.allow_tf32 = old
        out[name] = 2.0 * n ** 3 / (float(np.median(ts)) / 1e3) / 1e12
        del a, b
    torch.cuda.empty_cache()
    out["note"] = "torch.matmul (cuBLAS), FP64 4096^3, TF32 and BF16 8192^3, median of 5, TFLOP/s"
    return out


def hbm_peak():
    pk = measured_peaks()
    if "hbm_gbs" in pk:
        return float(pk["hbm_gbs"]), "HBM copy bandwidth measured (MEASURED_PEAKS.json)"
    return 6800.0, "HBM fallback 6.8 TB/s (no MEASURED_PEAKS.json)"


def tensor_peak(prec):
    """(peak TFLOP/s, note) of the form's tensor-core dtype, from the measured BF16 peak."""
    pk = measured_peaks()
    bf16 = float(pk.get("bf16_tflops", 1900.0))
    src = "measured (MEASURED_PEAKS.json)" if "bf16_tflops" in pk else "fallback"
    if prec == "tf32x3":
        return bf16 * TF32_NOMINAL_RATIO, (f"TF32 dense peak = bf16 {bf16:.1f} TFLOP/s {src} "
                                           "x nominal TF32/BF16 ratio 1.1/2.25")
    return bf16, f"BF16 dense peak {bf16:.1f} TFLOP/s {src}"


# ---------------------------------------------------------------------------
# algorithmic work of the contraction launches
# ---------------------------------------------------------------------------

def last_mode_io_bytes(scheme, N, E, P):
    """Bytes the last mode writes, per Tucker of a step: its FP32 result (the FP64
    integrator update is the separate elementwise pass that follows)."""
    nt = 2 if scheme in (wl.ETD2RK, wl.LAWSON2B) else 1
    return [4 * N] * nt


def mixed_bytes_per_launch(p, prec):
    """Average algorithmic DRAM bytes of one tc_mode_kernel launch in a step: each
    mode reads its operand's parts and the phi parts once and writes the next mode's
    parts; the last mode's epilogue moves the FP64 states instead."""
    E, P, N, d = ELEM[prec], PARTS[prec], p.N, p.d
    stages = last_mode_io_bytes(p.scheme, N, E, P)
    total, launches = 0.0, 0
    for st in stages:
        for mu in range(1, d + 1):
            n = p.n[mu - 1]
            b = P * E * N + 3 * E * n * n           # operand parts + phi parts
            b += P * E * N if mu < d else st
            total += b
            launches += 1
    return total / launches


# ---------------------------------------------------------------------------
# one form of a single-tensor workload
# ---------------------------------------------------------------------------

def time_single(api, p, prec, args, flush, stream, world, local, do_e2e=True):
    import torch
    import torch.distributed as dist
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan, g, U = api.setup(p, prec)
    torch.cuda.synchronize()
    plan_ms = 1e3 * (time.perf_counter() - t0)
    ws = api.expint_workspace(plan, p.scheme, g)
    N = p.N

    # A state larger than L2 is timed as one run of K steps (one expint_step call, as
    # an integration is run; inside it each ETD2RK step's stage-2 update is fused into
    # the next step's prepass); a smaller one step by step with L2 flushed between.
    run_mode = N * 8 > L2_BYTES
    if run_mode:
        for _ in range(max(1, -(-args.warmup // args.steps))):      # >= W steps, graph captured
            api.expint_step(plan, p.scheme, U, args.steps, t0=0.0, g=g, ws=ws)
    else:
        for k in range(args.warmup):
            api.expint_step(plan, p.scheme, U, 1, t0=k * p.tau, g=g, ws=ws)
    torch.cuda.synchronize()

    # ---- timed region: K steps, events around them (run mode) or around each step
    # with L2 flushed between steps outside the events ----
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if run_mode:
        flush.fill_(1)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    api.trace_enable(False)
    if run_mode:
        starts, ends = starts[:1], ends[:1]
        starts[0].record(stream)
        api.expint_step(plan, p.scheme, U, args.steps, t0=0.0, g=g, ws=ws)
        ends[0].record(stream)
    else:
        for k in range(args.steps):
            flush.fill_(k & 0xff)
            starts[k].record(stream)
            api.expint_step(plan, p.scheme, U, 1, t0=(args.warmup + k) * p.tau, g=g, ws=ws)
            ends[k].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    kcs = (api.KC_CONTRACT_FP64, api.KC_CONTRACT_TF32, api.KC_PREPASS, api.KC_SPLIT)
    counts = {c: api.trace_read(c, timed=False)[0] for c in kcs}
    assert plan.status() == 0, "non-finite state during the timed steps"
    t_ms = parallel.max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(starts, ends)), device="cuda")
    value = parallel.job_throughput([N * args.steps] * world, t_ms / 1e3)
    ms_step = t_ms / args.steps

    # ---- per-kernel device times: the same steps launched directly, each launch
    # bracketed by events on its stream (a graph replay has no per-kernel events) ----
    ksteps = min(args.steps, 10)
    api.trace_enable(True)
    if run_mode:
        flush.fill_(2)
        api.expint_step(plan, p.scheme, U, ksteps, t0=0.0, g=g, ws=ws)
    else:
        for k in range(ksteps):
            flush.fill_(k & 0xff)
            api.expint_step(plan, p.scheme, U, 1, t0=(args.warmup + args.steps + k) * p.tau, g=g, ws=ws)
    torch.cuda.synchronize()
    launches = {c: api.trace_read(c) for c in kcs}
    api.trace_enable(False)

    rec = {"value": value, "unit": METRIC, "ms_per_step": ms_step, "plan_ms": plan_ms,
           "roofline": roofline_single(p, prec, launches, ksteps, ms_step),
           "kernel_ms_per_step": {"contract": launches[api.KC_CONTRACT_FP64 if prec == "fp64"
                                                      else api.KC_CONTRACT_TF32][1] / ksteps,
                                  "prepass": launches[api.KC_PREPASS][1] / ksteps,
                                  "split_update": launches[api.KC_SPLIT][1] / ksteps},
           "launches_by_kernel": {"contract_fp64": counts[api.KC_CONTRACT_FP64],
                                  "contract_tf32": counts[api.KC_CONTRACT_TF32],
                                  "prepass": counts[api.KC_PREPASS], "split": counts[api.KC_SPLIT]},
           "gpu_launches": sum(counts.values()),
           "graph": ("the K timed steps are one expint_step call: one replay of its captured CUDA "
                     "graph" if run_mode else "each timed step is one replay of the step's captured CUDA graph"),
           "l2": (f"not flushed between steps inside the run: state {N * 8 / 1e6:.0f} MB > L2 (flushed once "
                  "before)" if run_mode else
                  f"flushed between timed steps (512 MB write); state {N * 8 / 1e6:.0f} MB"),
           "clocks": clk}

    if do_e2e:
        # ---- e2e: per step, a state in from pinned host memory, one step through the C
        # ABI, the result out to pinned host memory.  Successive steps take independent
        # states (a stream of problems), E2E_BUFS buffers deep: step k's copy in and step
        # k - 1's copy out run on their own streams beside step k's kernels, which stay
        # in order on one stream (they share the plan's workspace) ----
        U_host = torch.from_numpy(np.ascontiguousarray(p.u0)).pin_memory()
        outs = [torch.empty_like(U_host).pin_memory() for _ in range(E2E_BUFS)]
        bufs = [torch.empty_like(U) for _ in range(E2E_BUFS)]
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
        ev_in = [torch.cuda.Event() for _ in range(E2E_BUFS)]
        ev_done = [torch.cuda.Event() for _ in range(E2E_BUFS)]
        ev_out = [torch.cuda.Event() for _ in range(E2E_BUFS)]
        for bq in bufs:                      # each buffer's step graph, captured untimed
            bq.copy_(U_host)
            api.expint_step(plan, p.scheme, bq, 1, g=g, ws=ws)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2e_steps = min(args.steps, 10)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        s_in.wait_stream(stream)
        s_out.wait_stream(stream)
        for k in range(e2e_steps):
            b = k % E2E_BUFS
            with torch.cuda.stream(s_in):
                if k >= E2E_BUFS:
                    s_in.wait_event(ev_out[b])       # buffer b's previous result is out
                bufs[b].copy_(U_host, non_blocking=True)
                ev_in[b].record(s_in)
            stream.wait_event(ev_in[b])
            api.expint_step(plan, p.scheme, bufs[b], 1, g=g, ws=ws, stream=stream)
            ev_done[b].record(stream)
            with torch.cuda.stream(s_out):
                s_out.wait_event(ev_done[b])
                outs[b].copy_(bufs[b], non_blocking=True)
                ev_out[b].record(s_out)
        stream.wait_stream(s_out)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = parallel.max_over_ranks(e0.elapsed_time(e1), device="cuda")
        rec["e2e"] = {"value": parallel.job_throughput([N * e2e_steps] * world, e2e_ms / 1e3),
                      "unit": METRIC, "steps": e2e_steps,
                      "h2d_bytes_per_step": N * 8, "d2h_bytes_per_step": N * 8,
                      "pipeline": f"independent states, {E2E_BUFS} device buffers: copies in and out "
                                  "overlap the kernels of neighbouring steps"}
    del plan, g, U, ws
    torch.cuda.empty_cache()
    return rec


def roofline_single(p, prec, launches, ksteps, ms_step):
    from paper_2304_02327_gb300 import api
    N = p.N
    flops_per_launch = 2.0 * N * (sum(p.n) / len(p.n))   # 2 N n_mu per mode product
    if prec == "fp64":
        n_launch, k_ms = launches[api.KC_CONTRACT_FP64]
        avg = k_ms / n_launch if n_launch else None
        achieved = flops_per_launch / (avg / 1e3) / 1e12 if avg else None
        return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS if achieved else None,
                "traffic": profile_traffic("contract_fp64", p.name_tag),
                "kernel": "dgemm_kernel (FP64 mu-mode contraction, fused integrator epilogue)",
                "launches": n_launch, "avg_launch_ms": avg,
                "share_of_step_time": (k_ms / ksteps) / ms_step if ms_step else None,
                "flops_per_launch": flops_per_launch,
                "timing": f"eager traced run of {ksteps} steps (the timed steps replay a CUDA graph)",
                "peak_note": "FP64 peak derived: 152 SMs x 4 flop/clk x 2.07 GHz (nominal 1.25 "
                             "TFLOP/s); cuBLAS DGEMM measured live: library_gemm_tflops"}
    n_launch, k_ms = launches[api.KC_CONTRACT_TF32]
    avg = k_ms / n_launch if n_launch else None
    peak, note = tensor_peak(prec)
    tflops = NPROD[prec] * flops_per_launch
    achieved = tflops / (avg / 1e3) / 1e12 if avg else None
    logical = flops_per_launch / (avg / 1e3) / 1e12 if avg else None
    hb, hnote = hbm_peak()
    bpl = mixed_bytes_per_launch(p, prec)
    gbs = bpl / (avg / 1e3) / 1e9 if avg else None
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak if achieved else None,
            "traffic": profile_traffic(f"contract_{prec}", p.name_tag),
            "kernel": "tc_mode_kernel (tcgen05 mu-mode contraction, TMA-fed)",
            "launches": n_launch, "avg_launch_ms": avg,
            "share_of_step_time": (k_ms / ksteps) / ms_step if ms_step else None,
            "flops_per_launch": tflops,
            "logical": {"flops_per_launch": flops_per_launch, "achieved": logical,
                        "frac": logical / peak if logical else None},
            "hbm": {"algorithmic_bytes_per_launch": bpl, "achieved_gbs": gbs, "peak_gbs": hb,
                    "frac": gbs / hb if gbs else None, "peak_note": hnote},
            "timing": f"eager traced run of {ksteps} steps (the timed steps replay a CUDA graph)",
            "peak_note": note}


def accuracy_single(api, p, forms, nsample=24):
    """Errors of every form at the workload's full step count.

    FP64 GPU run to step S-1 and S; each mixed form's full run from u0 against the
    FP64 GPU state at step S (the FP64 form is pinned to the oracle at <= 1e-12 by
    the tests); and step S taken by each form from the same FP64 state at step S-1
    against the oracle's step on a seeded sample of output entries (the oracle forms
    every intermediate in full and the last Tucker only on the sampled rows)."""
    import torch
    from oracle.integrators import OracleProblem, rel_err_fro, rel_err_inf, step_at
    planf, gf, Uf = api.setup(p, "fp64")
    api.expint_step(planf, p.scheme, Uf, p.steps - 1, g=gf)
    Uprev = Uf.clone()
    t_last = (p.steps - 1) * p.tau
    api.expint_step(planf, p.scheme, Uf, 1, t0=t_last, g=gf)
    torch.cuda.synchronize()
    assert planf.status() == 0
    fp_final = Uf.cpu().numpy()
    del planf, gf, Uf
    rng = np.random.default_rng(2026)
    sets = [np.sort(rng.choice(n, min(n, nsample), replace=False)) for n in p.n]
    ix = np.ix_(*reversed(sets))
    t0 = time.perf_counter()
    op = OracleProblem.from_problem(p)
    ref = step_at(op, Uprev.cpu().numpy(), p.scheme, t_last, sets)
    oracle_s = time.perf_counter() - t0
    den = float(np.max(np.abs(ref)))

    def rel(x):
        return float(np.max(np.abs(x - ref)) / den)

    out = {"fp64": {"last_step_sampled_vs_oracle": rel(fp_final[ix])}}
    for prec in forms:
        if prec == "fp64":
            continue
        plan, g, U = api.setup(p, prec)
        api.expint_step(plan, p.scheme, U, p.steps, g=g)
        torch.cuda.synchronize()
        full = U.cpu().numpy()
        U.copy_(Uprev)
        api.expint_step(plan, p.scheme, U, 1, t0=t_last, g=g)
        torch.cuda.synchronize()
        assert plan.status() == 0
        one = U.cpu().numpy()[ix]
        out[prec] = {"full_run_vs_fp64_gpu": {"steps": p.steps, "inf": rel_err_inf(full, fp_final),
                                              "fro": rel_err_fro(full, fp_final)},
                     "last_step_sampled_vs_oracle": rel(one)}
        del plan, g, U
        torch.cuda.empty_cache()
    sample = (f"step {p.steps} of {p.steps} from the FP64 GPU state at step {p.steps - 1}, "
              f"{'x'.join(str(len(s)) for s in sets)} seeded output entries (oracle {oracle_s:.1f} s)")
    return out, sample


def other_config(api, name, forms, args, flush, stream, world, local, rank):
    """One further configuration in every form: throughput (the same timing as the
    headline, fewer steps, no e2e), the contraction's roofline fraction, and the
    errors: each split-precision run against the FP64 GPU run, the FP64 last step
    against the oracle on sampled entries, and for the small configurations the
    whole FP64 run against the oracle's."""
    import copy
    p = wl.workload(name)
    p.name_tag = name
    a = copy.copy(args)
    a.steps, a.warmup = min(args.steps, 10), min(args.warmup, 3)
    rec = {"N": p.N, "n": p.n, "scheme": wl.SCHEME_NAMES[p.scheme], "steps_of_workload": p.steps, "forms": {}}
    for prec in ["fp64"] + [f for f in forms if f != "fp64"]:
        r = time_single(api, p, prec, a, flush, stream, world, local, do_e2e=False)
        rf = r["roofline"]
        rec["forms"][prec] = {"value": r["value"], "unit": METRIC, "ms_per_step": r["ms_per_step"],
                              "roofline": {k: rf[k] for k in ("bound", "achieved", "peak", "unit", "frac",
                                                              "avg_launch_ms", "share_of_step_time")},
                              "kernel_ms_per_step": r["kernel_ms_per_step"], "gpu_launches": r["gpu_launches"],
                              "clocks": r["clocks"]}
    fp = rec["forms"]["fp64"]["ms_per_step"]
    for prec, r in rec["forms"].items():
        r["speedup_vs_fp64"] = fp / r["ms_per_step"]
    if rank == 0 and not args.no_accuracy:
        errs, sample = accuracy_single(api, p, ["fp64"] + forms, nsample=24 if p.d == 3 else 64)
        for prec, e in errs.items():
            rec["forms"][prec]["rel_err"] = e
        rec["rel_err_sample"] = sample
        if name in ORACLE_WHOLE_RUN:
            import torch
            from oracle.integrators import OracleProblem, integrate, rel_err_fro, rel_err_inf
            ref = integrate(OracleProblem.from_problem(p), p.u0, p.scheme, p.steps)
            plan, g, U = api.setup(p, "fp64")
            api.expint_step(plan, p.scheme, U, p.steps, g=g)
            torch.cuda.synchronize()
            got = U.cpu().numpy()
            rec["forms"]["fp64"]["rel_err"]["whole_run_vs_oracle"] = {
                "steps": p.steps, "inf": rel_err_inf(got, ref), "fro": rel_err_fro(got, ref)}
            del plan, g, U
    return rec


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


# ---------------------------------------------------------------------------
# the batched workload
# ---------------------------------------------------------------------------

def time_batched(api, name, prec, args, flush, stream, world, local, rank, do_check=True):
    """Many independent 2D Allen-Cahn problems advanced in one graph-captured batch,
    against the per-instance FP64 GPU loop on the same instances."""
    import torch
    import torch.distributed as dist
    probs_all = wl.batched_workload(name)
    costs = [parallel.instance_cost(p.n[0]) for p in probs_all]
    mine = parallel.shard_for_rank(costs, rank, world)       # LPT shard, no collective
    probs = [probs_all[i] for i in mine]
    dof = sum(p.u0.size for p in probs)
    dof_all = sum(p.u0.size for p in probs_all)

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plans, gs, Us = api.setup_batch(probs, prec)
    torch.cuda.synchronize()
    plan_ms = 1e3 * (time.perf_counter() - t0)
    t0 = time.perf_counter()
    if args.nc_cap:
        b = api.Batch(plans, gs, Us, autotune=False, nc_cap=args.nc_cap, graph=True)
    else:
        b = api.Batch(plans, gs, Us, autotune=True, graph=True)
    torch.cuda.synchronize()
    create_ms = 1e3 * (time.perf_counter() - t0)
    # warm-up: at least W steps, in runs of K steps (instantiates the K-step graph)
    for _ in range(max(1, -(-args.warmup // args.steps))):
        b.run(args.steps)
    torch.cuda.synchronize()

    # ---- timed region: the K steps as one run (one graph launch; the update of each
    # step fused into the next step's prepass), inputs larger than L2 ----
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    flush.fill_(1)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    api.trace_enable(False)
    e_start.record(stream)
    b.run(args.steps)
    e_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    kcs = (api.KC_CONTRACT_TF32, api.KC_PREPASS, api.KC_SPLIT)
    counts = {c: api.trace_read(c, timed=False)[0] for c in kcs}
    assert b.status() == 0, "non-finite state during the timed steps"
    t_ms = parallel.max_over_ranks(e_start.elapsed_time(e_end), device="cuda")
    value = parallel.job_throughput([dof_all * args.steps], t_ms / 1e3)
    ms_step = t_ms / args.steps

    # ---- per-kernel device times: the same batch's launches, eager and traced, as one
    # run of ksteps steps like the timed region ----
    b.set_graph(False)
    b.run(1)
    torch.cuda.synchronize()
    api.trace_enable(True)
    ksteps = min(args.steps, 5)
    flush.fill_(2)
    b.run(ksteps)
    torch.cuda.synchronize()
    n_launch, k_ms = api.trace_read(api.KC_CONTRACT_TF32)
    _, pre_ms = api.trace_read(api.KC_PREPASS)
    _, upd_ms = api.trace_read(api.KC_SPLIT)
    api.trace_enable(False)
    b.set_graph(True)

    # ---- e2e: every state in from pinned host memory, one step, every state out.  The
    # states sit packed in one device buffer (one copy each way per step); E2E_BUFS batches
    # over as many such buffers take the steps in turn, so that one batch's copies overlap
    # the other's kernels (successive steps take independent states; the kernels stay in
    # order on one stream) ----
    offs, total = api.flat_offsets(probs)
    host_in = torch.zeros(total, dtype=torch.float64).pin_memory()
    for p, o in zip(probs, offs):
        host_in[o:o + p.u0.size].copy_(torch.from_numpy(np.ascontiguousarray(p.u0)).reshape(-1))
    host_out = [torch.empty_like(host_in).pin_memory() for _ in range(E2E_BUFS)]
    pipes = []
    for _ in range(E2E_BUFS):
        Ue, fbuf = api.flat_states(probs)
        be = api.Batch(plans, gs, Ue, autotune=False, nc_cap=b.info()["nc_cap"], graph=True)
        be.run(1)                            # its one-step graph, captured untimed
        pipes.append((be, fbuf))
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(E2E_BUFS)]
    ev_done = [torch.cuda.Event() for _ in range(E2E_BUFS)]
    ev_out = [torch.cuda.Event() for _ in range(E2E_BUFS)]
    e2e_steps = min(args.steps, 9)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    s_in.wait_stream(stream)
    s_out.wait_stream(stream)
    for k in range(e2e_steps):
        j = k % E2E_BUFS
        be, fbuf = pipes[j]
        with torch.cuda.stream(s_in):
            if k >= E2E_BUFS:
                s_in.wait_event(ev_out[j])           # this buffer's previous result is out
            fbuf.copy_(host_in, non_blocking=True)
            ev_in[j].record(s_in)
        stream.wait_event(ev_in[j])
        be.run(1)
        ev_done[j].record(stream)
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev_done[j])
            host_out[j].copy_(fbuf, non_blocking=True)
            ev_out[j].record(s_out)
    stream.wait_stream(s_out)
    e1.record(stream)
    torch.cuda.synchronize()
    assert all(be.status() == 0 for be, _ in pipes)
    e2e_ms = parallel.max_over_ranks(e0.elapsed_time(e1), device="cuda")
    e2e_value = parallel.job_throughput([dof_all * e2e_steps], e2e_ms / 1e3)
    for be, _ in pipes:
        be.close()
    del pipes
    torch.cuda.empty_cache()

    # ---- error: the whole run from u0 of sampled instances against the oracle ----
    check = None
    if do_check and rank == 0:
        for p, u in zip(probs, Us):
            u.copy_(torch.from_numpy(np.ascontiguousarray(p.u0)))
        steps = probs[0].steps
        b.run(steps)
        torch.cuda.synchronize()
        assert b.status() == 0
        check = batch_check(probs, Us, steps)

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

    info = b.info()
    sched = b.schedule()
    b.close()
    del plans, gs, Us
    torch.cuda.empty_cache()

    flops_launch = sum(2.0 * p.u0.size * p.n[0] for p in probs)   # one direction of every instance
    k_avg = k_ms / n_launch if n_launch else None
    peak, note = tensor_peak(prec)
    achieved = NPROD[prec] * flops_launch / (k_avg / 1e3) / 1e12 if k_avg else None
    E, P = ELEM[prec], PARTS[prec]
    # per launch: the operand's parts in and every instance's phi_1 in three parts
    # (3 E n^2 = 3 E DOF for square instances); mode 1 writes the next mode's parts,
    # mode 2 the FP32 result
    bpl = (P * E * dof + 3 * E * dof + P * E * dof + P * E * dof + 3 * E * dof + 4 * dof) / 2
    hb, hnote = hbm_peak()
    gbs = bpl / (k_avg / 1e3) / 1e9 if k_avg else None
    rec = {"workload": name, "value": value, "unit": METRIC, "ms_per_step": ms_step,
           "dtype": f"{prec}+f64", "instances": len(probs_all), "dof": dof_all,
           "sizes": "n uniform over {48, 64, ..., 512}, square", "scheme": "expeuler",
           "tau": probs_all[0].tau, "size_classes": info["classes"],
           ("nc_cap_pinned" if args.nc_cap else "nc_cap_autotuned"): info["nc_cap"],
           "autotuned_schedule": None if args.nc_cap else {
               "widths_by_class": sched["widths"], "per_class_widths_kept": sched["per_class"],
               "tucker_ms_uniform_width": sched["tucker_ms_uniform"],
               "tucker_ms_chosen": sched["tucker_ms_chosen"],
               "tile_order": "decreasing cost, one CTA per SM taking tiles "
                             + ("round-robin" if sched["tile_order"] == "round-robin"
                                else "round-robin with every other round reversed")},
           "tiles_per_mode": info["tiles_mode1"],
           "plan_ms": plan_ms, "batch_create_ms": create_ms,
           "graph": "the K timed steps are one run: one CUDA graph launch, each step's update "
                    "fused into the next step's prepass",
           "l2": f"not flushed between steps inside the run: states {dof_all * 8 / 1e9:.2f} GB > L2 "
                 "(flushed once before)",
           "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                        "frac": achieved / peak if achieved else None, "traffic": None,
                        "kernel": "tc_mode_kernel (grouped tcgen05 mu-mode contraction, all instances)",
                        "launches": n_launch, "avg_launch_ms": k_avg,
                        "share_of_step_time": (k_ms / ksteps) / ms_step if k_ms else None,
                        "flops_per_launch": NPROD[prec] * flops_launch,
                        "logical": {"flops_per_launch": flops_launch,
                                    "frac": (achieved / NPROD[prec]) / peak if achieved else None},
                        "hbm": {"algorithmic_bytes_per_launch": bpl, "achieved_gbs": gbs, "peak_gbs": hb,
                                "frac": gbs / hb if gbs else None, "peak_note": hnote},
                        "timing": "eager traced run of the same launches (a graph replay has no "
                                  "per-kernel events)",
                        "peak_note": note},
           "kernel_ms_per_step": {"contract": k_ms / ksteps, "prepass": pre_ms / ksteps,
                                  "update": upd_ms / ksteps},
           "fp64_per_instance_loop": {"ms_per_step": fp_ms, "value": dof_all / (fp_ms / 1e3),
                                      "unit": METRIC},
           "speedup_vs_fp64_loop": fp_ms / ms_step,
           "e2e": {"value": e2e_value, "unit": METRIC, "steps": e2e_steps,
                   "h2d_bytes_per_step": dof * 8, "d2h_bytes_per_step": dof * 8,
                   "pipeline": f"all states packed in one buffer, one copy each way per step; {E2E_BUFS} "
                               "batches take the steps in turn so that copies overlap the others' kernels"},
           "gpu_launches": sum(counts.values()),
           "launches_by_kernel": {"contract_tf32": counts[api.KC_CONTRACT_TF32],
                                  "prepass": counts[api.KC_PREPASS], "update": counts[api.KC_SPLIT]},
           "clocks": clk}
    if check is not None:
        rec["rel_err_vs_oracle"] = check
    return rec


def batch_check(probs, Us, steps, count=4):
    """The batch's states after `steps` steps from u0 against the oracle's run, on the
    smallest and the largest instance and two seeded others."""
    from oracle.integrators import OracleProblem, integrate, rel_err_inf
    sizes = [p.n[0] for p in probs]
    pick = {int(np.argmin(sizes)), int(np.argmax(sizes))}
    rng = np.random.default_rng(44)
    while len(pick) < min(count, len(probs)):
        pick.add(int(rng.integers(len(probs))))
    worst, rows = 0.0, []
    t0 = time.perf_counter()
    for j in sorted(pick):
        p = probs[j]
        ref = integrate(OracleProblem.from_problem(p, lmax=1), p.u0, p.scheme, steps)
        e = rel_err_inf(Us[j].cpu().numpy(), ref)
        worst = max(worst, e)
        rows.append({"n": p.n[0], "inf": e})
    return {"steps": steps, "instances": rows, "worst_inf": worst,
            "sample": f"{len(rows)} whole instances (smallest, largest, seeded others), "
                      f"oracle {time.perf_counter() - t0:.1f} s"}


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


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------

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
                         "sample": f"{args.warmup}+{args.steps} full steps of {args.workload} "
                                   f"(numpy float64, BLAS threads up to {cores})"},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def ours(args):
    import torch
    import torch.distributed as dist
    from paper_2304_02327_gb300 import api

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    api.lib()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    if args.workload in wl.BATCHED:
        # a batch as the headline (profiling runs of the batched stepper)
        prec = args.prec if args.prec != "fp64" else args.batch_prec
        rec = time_batched(api, args.workload, prec, args, flush, stream, world, local, rank,
                           do_check=not args.no_accuracy)
        if rank == 0:
            line = {"metric": METRIC, "value": rec["value"], "unit": METRIC, "n_gpus": world,
                    "steps": args.steps, "warmup": args.warmup, "ms_per_step": rec["ms_per_step"],
                    "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                    "dtype": rec["dtype"], "data": "synthetic",
                    "config": {"workload": args.workload, "precision": prec,
                               "l2": rec["l2"], "parallelism": f"LPT shard of instances x{world}"},
                    **{k: v for k, v in rec.items() if k not in ("value", "unit", "ms_per_step", "dtype",
                                                                 "workload", "l2")}}
            if not args.no_cpu_baseline:
                line["cpu_baseline"] = oracle_batch_sample(wl.batched_workload(args.workload),
                                                           args.cpu_seconds)
            print(json.dumps(line), flush=True)
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    p = wl.workload(args.workload)
    p.name_tag = args.workload
    head = time_single(api, p, args.prec, args, flush, stream, world, local, do_e2e=True)
    forms = [f for f in (x.strip() for x in args.mixed.split(",")) if f and f != "none" and f != args.prec]
    mixed = {}
    for prec in forms:
        r = time_single(api, p, prec, args, flush, stream, world, local, do_e2e=True)
        r["dtype"] = f"{prec}+f64" if prec != "fp64" else "f64"
        r["speedup_vs_headline"] = head["ms_per_step"] / r["ms_per_step"]
        mixed[prec] = r
    batched = None
    if args.batch and args.batch != "none":
        batched = time_batched(api, args.batch, args.batch_prec, args, flush, stream, world, local, rank,
                               do_check=not args.no_accuracy)
    others = {}
    if args.configs != "none":
        for name in OTHER_CONFIGS:
            if name != args.workload:
                others[name] = other_config(api, name, forms, args, flush, stream, world, local, rank)

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    line = {
        "metric": METRIC, "value": head["value"], "unit": METRIC, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.prec == "fp64" else f"{args.prec}+f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "n": p.n, "N": p.N,
                   "scheme": wl.SCHEME_NAMES[p.scheme], "tau": p.tau, "steps_of_workload": p.steps,
                   "precision": args.prec,
                   "l2": head["l2"],
                   "parallelism": f"replicas x{world}"},
        "plan_ms": head["plan_ms"],
        "roofline": head["roofline"],
        "e2e": head["e2e"],
        "gpu_launches": head["gpu_launches"],
        "kernel_ms_per_step": head["kernel_ms_per_step"],
        "launches_by_kernel": head["launches_by_kernel"],
        "graph": head["graph"],
        "clocks": head["clocks"],
        "library_gemm_tflops": library_gemm_tflops(),
    }
    if mixed:
        line["mixed"] = mixed
    if batched is not None:
        line["batched"] = batched
    if others:
        line["other_configs"] = others

    if not args.no_accuracy:
        errs, sample = accuracy_single(api, p, [args.prec] + forms)
        line["rel_err_vs_oracle"] = {"last_step_sampled": errs[args.prec]["last_step_sampled_vs_oracle"],
                                     "sample": sample,
                                     "full_run": "the FP64 form's whole runs are pinned to the oracle "
                                                 "at <= 1e-12 by the tests (100 steps at n = 128, 2 at "
                                                 "n = 320)" if args.prec == "fp64" else None}
        for prec in forms:
            mixed[prec]["rel_err"] = errs[prec]
    if not args.no_cpu_baseline:
        Uo, osteps, odt = run_oracle_sample(p, args.cpu_seconds)
        line["cpu_baseline"] = {"value": p.N * osteps / odt, "unit": METRIC, "cores": host_cores(),
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
