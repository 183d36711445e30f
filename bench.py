#!/usr/bin/env python3
"""Throughput of one multiple-shooting objective + gradient evaluation on GB300.

Workload: 4 transmons x 3 levels (N=81 rows, E=16 essential columns), all-pair cross-Kerr,
2 carriers per transmon with 40 B-spline coefficients each (d=640), QFT_16 target,
T=600 ns, 100000 implicit-midpoint steps, M windows (default 256), seeded synthetic controls
and non-unitary window states.  A step of this benchmark is one full evaluation
(controls, forward sweep of every window, terminal conditions, adjoint sweep with the fused
gradient, reductions).  The midpoint-state history (2 GB) is far larger than L2, so no L2
flush is needed between steps.

The default line also carries, measured in the same process:
  config3      the 4-transmon workload at every window count (64, 128, 256) and checkpoint
               interval (1, 64, 512), tiles from the library's model;
  solver_fp64  the benchmark workload with the all-FP64 step solver;
  batched      96 mixed problems (32 x 2q + 32 x 3q + 32 x 4q) in one graph-replayed batch
               against the same problems one after another;
  serving      a Poisson request stream over 64 sessions (2q/3q/4q/5q) served with continuous
               batching (arrival-order and throughput policies) against one request at a time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--windows M]
                  [--solver mixed|fp64] [--col-block CB] [--nsteps NT] [--no-cpu-baseline]
                  [--no-extras]

Prints one JSON line.  Under torchrun (N > 1) every rank evaluates its own independent
problem (weak scaling, no collective on the data path); rank 0 prints.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2407_13950_gb300 import synthetic as S  # noqa: E402

METRIC = "4-qubit QFT objective+gradient evals/s"
UNIT = "evals/s"


def flops_model(spec):
    """Algorithmic FP64 flops of one evaluation: one H-apply per implicit solve, the 2Ubar-U
    update, and the gradient inner products (8 flops per complex multiply-add)."""
    N, q, L, E, nt = spec.N, spec.q, spec.L, spec.E, spec.nsteps
    nnz = q * 2 * N * (L - 1) // L                 # ladder-term nonzeros per column
    f_step = 8 * nnz + 2 * N + 4 * N
    fwd = E * nt * f_step
    adj = E * nt * (f_step + 8 * nnz)
    return {"forward": fwd, "adjoint": adj, "total": fwd + adj}


class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
                for i, nm in enumerate(names):
                    if r[5 + i].lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


SWEEP_SOURCES = ["msqoc_sweep.cuh", "msqoc_sweep_pair.cuh", "msqoc_sweep_common.cuh", "msqoc_split.cuh",
                 "inst_sweep.cu", "msqoc_internal.h"]
PROFILES = os.path.join(ROOT, "profiles")
LAYOUTS = {"auto": 0, "fiber": 1, "pair": 2, "quad": 3, "lean": 4}


def sweep_traffic(kernel: str, windows: int, col_block: int, layout: int):
    """DRAM bytes per launch of a sweep kernel from a committed ncu summary of the same tiles
    (a `capture_config:` line naming windows, columns per tile and kernel family, and a
    `traffic_per_launch_bytes:` line), or None when there is none or the kernel sources changed
    since that capture (their digest differs)."""
    import glob
    import hashlib
    import re
    h = hashlib.sha256()
    for fn in SWEEP_SOURCES:
        h.update(fn.encode())
        with open(os.path.join(ROOT, "paper_2407_13950_gb300", "csrc", fn), "rb") as f:
            h.update(f.read())
    digest = h.hexdigest()[:16]
    want = f"capture_config: windows={windows} col_block={col_block} layout={layout}"
    for path in sorted(glob.glob(os.path.join(PROFILES, "k_sweep_4q_*.md"))):
        text = open(path).read()
        m = re.search(r"sources_sha256: ([0-9a-f]+)", text)
        t = re.search(rf"{kernel}=([0-9.e+]+)", text)
        if want in text and m and t and m.group(1) == digest:
            return float(t.group(1)), os.path.relpath(path, ROOT)
    return None, None


def max_over_ranks(value: float, dist, device) -> float:
    """The largest of every rank's value (timings: the job is as slow as its slowest rank)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_inputs(spec, rank: int):
    """Each rank evaluates its own independent problem: the seeded inputs of problem `rank`."""
    return S.random_alpha(spec, 1, problem=rank), S.random_W(spec, 1, problem=rank)


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_config(spec) -> dict:
    """The workload as both arms name it (implementation choices are reported separately)."""
    return {"workload": spec.name, "N": spec.N, "E": spec.E, "nsteps": spec.nsteps, "windows": spec.M,
            "T_ns": spec.T, "d": spec.d, "l2": "inputs larger than L2 (2 GB midpoint history per evaluation)"}


def cpu_baseline(spec, alpha, W):
    """The oracle, as it stands, on this host's cores: one whole evaluation (objective and
    gradient of every window; windows in parallel on all cores)."""
    import oracle
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.evaluate(spec, alpha, W, nthreads=cores)
    dt = time.perf_counter() - t0
    return {"value": 1.0 / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one whole evaluation ({spec.M} windows, forward+adjoint, {spec.nsteps} steps) on "
                      f"{cores} threads in {dt:.2f} s"}


def run_reference(args, spec):
    """The oracle as the reference arm: each step one whole evaluation of the same workload on
    every host core."""
    rank, world, _ = dist_info()
    if rank != 0:
        return
    alpha, W = S.random_alpha(spec, 1), S.random_W(spec, 1)
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    times = []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.evaluate(spec, alpha, W, nthreads=cores)
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
    per_eval = float(np.mean(times))
    value = 1.0 / per_eval
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_eval * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {**workload_config(spec), "parallelism": f"independent problem per GPU x{world}"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"each step one whole evaluation ({spec.M} windows, forward+adjoint) on "
                                       f"{cores} threads; {args.steps} timed steps after {args.warmup} warm-up"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_evaluations(prob, a_d, W_d, outs, stream, steps: int, warmup: int, kernel_times: bool = True):
    """ms per objective+gradient evaluation (CUDA events around `steps` back-to-back evaluations
    after `warmup`), and the library's per-kernel event times averaged over `steps` more."""
    import torch
    P_d, ga_d, gW_d = outs
    for _ in range(warmup):
        prob.eval_gradient_into(a_d, W_d, P_d, ga_d, gW_d, stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        prob.eval_gradient_into(a_d, W_d, P_d, ga_d, gW_d, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    kt = None
    if kernel_times:
        from paper_2407_13950_gb300 import msqoc
        kt = {k: 0.0 for k in msqoc.KERNEL_NAMES}
        for _ in range(steps):
            prob.eval_gradient_into(a_d, W_d, P_d, ga_d, gW_d, stream=stream)
            t = prob.kernel_times()
            for k in kt:
                kt[k] += t[k] / steps
    return ms, kt


FAMILY = {1: "one thread per fiber", 2: "lane pair per fiber", 3: "lane quad per fiber",
          4: "one thread per fiber, 168 registers"}


def config3_section(dev, stream, peak, steps: int = 5, warmup: int = 2) -> dict:
    """The 4-transmon workload at every window count and checkpoint interval of its
    configuration, with the library's own tile choice (no autotuning)."""
    import torch
    from paper_2407_13950_gb300 import msqoc
    out = {}
    for M in (64, 128, 256):
        spec = S.config_4q(M=M)
        alpha, W = S.random_alpha(spec, 1), S.random_W(spec, 1)
        a_d = torch.tensor(alpha, device=dev, dtype=torch.float64)
        W_d = torch.tensor(W, device=dev, dtype=torch.float64)
        outs = (torch.zeros(1, device=dev, dtype=torch.float64), torch.zeros(spec.d, device=dev, dtype=torch.float64),
                torch.zeros(spec.nW, device=dev, dtype=torch.float64))
        fl = flops_model(spec)
        for K in (1, 64, 512):
            with msqoc.Problem(spec, ckpt_interval=K, profile=True) as p:
                ms, kt = time_evaluations(p, a_d, W_d, outs, stream, steps, warmup)
                out[f"M{M}_K{K}"] = {
                    "evals_per_s": 1e3 / ms, "ms_per_eval": ms, "kernel_ms": kt,
                    "adjoint_frac_of_fp64_peak": fl["adjoint"] / (kt["adjoint"] * 1e-3) / 1e12 / peak,
                    "whole_eval_frac_of_fp64_peak": fl["total"] / (ms * 1e-3) / 1e12 / peak,
                    "tiles": f"{FAMILY[p.layout]} x {p.col_block} columns ({p.tiles} CTAs)",
                    "steps_per_sync": p.steps_per_sync,
                    "ckpt_interval": p.ckpt_interval, "device_bytes": p.device_bytes}
        del a_d, W_d, outs
        torch.cuda.empty_cache()
    return out


def solver_fp64_section(spec, dev, stream, peak, steps: int = 5, warmup: int = 2) -> dict:
    """The benchmark workload with the all-FP64 fixed-point step solver."""
    import torch
    from paper_2407_13950_gb300 import msqoc
    alpha, W = S.random_alpha(spec, 1), S.random_W(spec, 1)
    a_d = torch.tensor(alpha, device=dev, dtype=torch.float64)
    W_d = torch.tensor(W, device=dev, dtype=torch.float64)
    outs = (torch.zeros(1, device=dev, dtype=torch.float64), torch.zeros(spec.d, device=dev, dtype=torch.float64),
            torch.zeros(spec.nW, device=dev, dtype=torch.float64))
    fl = flops_model(spec)
    with msqoc.Problem(spec, solver=msqoc.SOLVER_FP64, profile=True) as p:
        ms, kt = time_evaluations(p, a_d, W_d, outs, stream, steps, warmup)
        achieved = fl["adjoint"] / (kt["adjoint"] * 1e-3) / 1e12
        return {"value": 1e3 / ms, "unit": UNIT, "ms_per_eval": ms, "kernel_ms": kt,
                "tiles": f"{FAMILY[p.layout]} x {p.col_block} columns ({p.tiles} CTAs)",
                "roofline": {"kernel": "k_sweep (adjoint)", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                             "frac": achieved / peak}}


def run_ours(args, spec):
    import torch
    from paper_2407_13950_gb300 import msqoc

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    alpha, W = rank_inputs(spec, rank)
    dev = torch.device("cuda", local)
    a_d = torch.tensor(alpha, device=dev, dtype=torch.float64)
    W_d = torch.tensor(W, device=dev, dtype=torch.float64)
    P_d = torch.zeros(1, device=dev, dtype=torch.float64)
    ga_d = torch.zeros(spec.d, device=dev, dtype=torch.float64)
    gW_d = torch.zeros(spec.nW, device=dev, dtype=torch.float64)
    stream = torch.cuda.current_stream(dev)
    solver = msqoc.SOLVER_FP64 if args.solver == "fp64" else msqoc.SOLVER_MIXED
    # tile width and kernel family: the library's model (0), a given width, or measured by the
    # autotuner (-1)
    layout = LAYOUTS[args.layout]
    tuned = tune_ms = None
    sps = args.steps_per_sync
    if args.col_block < 0:
        tuned, layout, sps, tune_ms = msqoc.autotune(spec, alpha=alpha, probe_steps=64, solver=solver, layout=layout,
                                                     steps_per_sync=args.steps_per_sync)
        fam = {1: "fiber", 2: "pair", 3: "quad", 4: "lean"}
        tune_ms = {f"{fam[lay]}-{cb}-s{dp}": v for (lay, cb, dp), v in tune_ms.items()}
    col_block = tuned if args.col_block < 0 else args.col_block
    prob = msqoc.Problem(spec, solver=solver, col_block=col_block, profile=True, layout=layout, steps_per_sync=sps)
    peak_tflops = msqoc.measure_fp64_peak()

    for _ in range(args.warmup):
        prob.eval_gradient_into(a_d, W_d, P_d, ga_d, gW_d, stream=stream)
    barrier()

    sampler = ClockSampler(local)
    sampler.start()
    # timed region: the evaluations back to back, no host synchronisation between them
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        prob.eval_gradient_into(a_d, W_d, P_d, ga_d, gW_d, stream=stream)
    e1.record(stream)
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, dev)
    value = world / (ms * 1e-3)
    # per-kernel CUDA-event times (the library's profiling events) over the same number of
    # evaluations right after: reading them synchronises every evaluation
    kt = {k: 0.0 for k in msqoc.KERNEL_NAMES}
    for _ in range(args.steps):
        prob.eval_gradient_into(a_d, W_d, P_d, ga_d, gW_d, stream=stream)
        t = prob.kernel_times()
        for k in kt:
            kt[k] += t[k]
    clocks = sampler.stop()

    # end to end through the C ABI with pinned host buffers (H2D of alpha and W, D2H of P and both
    # gradients inside the call, which returns once the results are on the host)
    pinned = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).pin_memory()
    a_h, W_h = pinned(alpha), pinned(W if spec.M > 1 else np.zeros(2))
    P_h, ga_h, gW_h = pinned(np.zeros(1)), pinned(np.zeros(spec.d)), pinned(np.zeros(max(spec.nW, 2)))
    e2e_times = []
    for it in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        prob.eval_gradient_into(a_h, W_h if spec.M > 1 else None, P_h, ga_h, gW_h if spec.M > 1 else None,
                                stream=stream)
        if it >= args.warmup:
            e2e_times.append(time.perf_counter() - t0)
    e2e_ms = max_over_ranks(float(np.mean(e2e_times)) * 1e3, dist, dev)

    fl = flops_model(spec)
    dom = max(("forward", "adjoint"), key=lambda k: kt[k])
    traffic, traffic_src = (sweep_traffic(dom, spec.M, prob.col_block, prob.layout) if spec.nsteps == 100000
                            else (None, None))
    dom_ms = kt[dom] / args.steps
    achieved = fl[dom] / (dom_ms * 1e-3) / 1e12
    launches_per_eval = 6 if spec.M > 1 else 5
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {**workload_config(spec), "parallelism": f"independent problem per GPU x{world}"},
        "implementation": {
            "solver": args.solver,
            "col_block": (f"autotuned ({prob.col_block})" if tuned else
                          col_block if col_block > 0 else f"model ({prob.col_block})"),
            "layout": FAMILY[prob.layout], "ctas": prob.tiles, "threads_per_cta": prob.threads,
            "steps_per_sync": prob.steps_per_sync,
            **({"autotune": {"best": tuned, "ms_per_probe_eval": tune_ms}} if tuned else {})},
        "roofline": {"bound": "alu", "kernel": f"k_sweep ({dom})", "achieved": achieved, "peak": peak_tflops,
                     "unit": "TFLOP/s", "frac": achieved / peak_tflops,
                     "traffic": traffic,
                     "traffic_note": (f"DRAM bytes per launch from {traffic_src} (ncu capture of the same "
                                      "tiles and sweep sources)" if traffic else
                                      "null: no ncu summary of these tiles for the current sweep sources"),
                     "peak_source": "measured FP64 FMA microbenchmark (msqoc_measure_fp64_peak), same run",
                     "peak_note": ("the method's FP64-defined flops against the native FP64 peak; the mixed "
                                   "solver computes part of that arithmetic in compensated FP32 (two-float "
                                   "sums), so the fraction is not one unit's occupancy and can exceed 1"),
                     "algorithmic_flops_per_launch": fl[dom], "avg_launch_ms": dom_ms},
        "kernel_ms": {k: v / args.steps for k, v in kt.items()},
        "whole_eval": {"algorithmic_tflops": fl["total"] / (ms * 1e-3) / 1e12,
                       "frac_of_fp64_peak": fl["total"] / (ms * 1e-3) / 1e12 / peak_tflops},
        "e2e": {"value": world / (e2e_ms * 1e-3), "unit": UNIT, "buffers": "pinned host",
                "h2d_bytes_per_step": 8 * (spec.d + spec.nW), "d2h_bytes_per_step": 8 * (1 + spec.d + spec.nW),
                # this rank's calls (host clock, ms): the value is from their mean
                "call_ms": {"min": min(e2e_times) * 1e3, "median": float(np.median(e2e_times)) * 1e3,
                            "max": max(e2e_times) * 1e3} if e2e_times else None},
        "gpu_launches": launches_per_eval * args.steps,
        "clocks": clocks,
    }
    prob.close()
    del a_d, W_d, P_d, ga_d, gW_d
    torch.cuda.empty_cache()
    if rank == 0 and not args.no_extras and spec.nsteps == 100000:
        # the other settings of the workload and the systems patterns, same process and box
        t_extra = time.perf_counter()
        line["config3"] = config3_section(dev, stream, peak_tflops)
        line["solver_fp64"] = solver_fp64_section(spec, dev, stream, peak_tflops)
        line["batched"] = batched_section(args, dev, stream, peak_tflops, steps=3, warmup=1)
        torch.cuda.empty_cache()
        line["serving"] = serving_section(args, peak_tflops, seconds=args.extra_serve_seconds)
        line["extras_seconds"] = time.perf_counter() - t_extra
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(spec, alpha, W)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def batched_section(args, dev, stream, peak, steps: int, warmup: int) -> dict:
    """The batched workload: 32 x 2 transmons + 32 x 3 + 32 x 4 (durations uniform in
    [0.5 T, 1.5 T] at the base step size, windows drawn from {8, 32, 64, 128}), one
    objective+gradient evaluation of all 96 per step, as one batch replayed from a CUDA graph,
    against the same problems evaluated one after another (one problem per launch sequence)."""
    import torch
    from paper_2407_13950_gb300 import msqoc

    specs = S.mixed_batch_specs(seed=1, n_per_shape=args.batch_per_shape,
                                shapes=[S.config_2q(), S.config_3q(), S.config_4q()])
    nprob = len(specs)
    probs = [msqoc.Problem(sp, layout=LAYOUTS[args.layout]) for sp in specs]
    host_in = [(S.random_alpha(sp, 1, problem=i), S.random_W(sp, 1, problem=i)) for i, sp in enumerate(specs)]
    dev_in = [(torch.tensor(a, device=dev, dtype=torch.float64), torch.tensor(W, device=dev, dtype=torch.float64))
              for a, W in host_in]
    outs = [(torch.zeros(1, device=dev, dtype=torch.float64), torch.zeros(p.d, device=dev, dtype=torch.float64),
             torch.zeros(max(p.nW, 2), device=dev, dtype=torch.float64)) for p in probs]
    batch = msqoc.Batch(probs, gradient=True, graph=True)
    fam = {1: "fiber", 2: "pair", 3: "quad", 4: "lean"}
    tile_mix = {}
    for sp, p in zip(specs, probs):       # how many problems run each (shape, family, width)
        key = f"{sp.q}q {fam[p.layout]} x{p.col_block} ({p.threads} threads)"
        tile_mix[key] = tile_mix.get(key, 0) + 1

    def batched_step():
        for i, (a, W) in enumerate(dev_in):
            batch.set_inputs(i, a, W, stream=stream)
        batch.eval_gradient(stream=stream)

    def plain_step(ev=None):
        for i, p in enumerate(probs):
            a, W = dev_in[i]
            P, ga, gW = outs[i]
            p.eval_gradient_into(a, W if p.spec.M > 1 else None, P, ga, gW if p.spec.M > 1 else None, stream=stream)
            if ev is not None:
                ev[i].record(stream)

    def timed(fn, n):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(n):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    for _ in range(warmup):
        batched_step()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    ms_b = timed(batched_step, steps)
    clocks = sampler.stop()
    for _ in range(warmup):
        plain_step()
    ms_p = timed(plain_step, steps)
    # completion times when all requests are submitted together: the batch finishes them all at
    # once; one after another, request i waits for the ones before it
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(nprob)]
    e0 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    plain_step(ev)
    torch.cuda.synchronize()
    done_p = np.array([e0.elapsed_time(e) for e in ev])
    # end to end through pinned host buffers: inputs copied from host memory, results read back
    pinned = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).pin_memory()
    res = [(pinned(np.zeros(1)), pinned(np.zeros(p.d)), pinned(np.zeros(max(p.nW, 1)))) for p in probs]
    host_pinned = [(pinned(a), pinned(W)) for a, W in host_in]

    def e2e_step():
        for i, (a, W) in enumerate(host_pinned):
            batch.set_inputs(i, a, W, stream=stream)
        batch.eval_gradient(stream=stream)
        for i, p in enumerate(probs):
            P, ga, gW = res[i]
            msqoc.load().msqoc_get_gradient(p.handle, msqoc._ptr(P), msqoc._ptr(ga),
                                           msqoc._ptr(gW) if p.spec.M > 1 else None, msqoc._stream_handle(stream))
        torch.cuda.synchronize()

    e2e_step()
    t0 = time.perf_counter()
    for _ in range(steps):
        e2e_step()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / steps
    h2d = sum(8 * (sp.d + (sp.nW if sp.M > 1 else 0)) for sp in specs)
    d2h = sum(8 * (1 + sp.d + (sp.nW if sp.M > 1 else 0)) for sp in specs)
    fl = sum(flops_model(sp)["total"] for sp in specs)
    out = {
        "workload": f"{nprob} problems: {args.batch_per_shape}x2q + {args.batch_per_shape}x3q + "
                    f"{args.batch_per_shape}x4q, durations U[0.5T,1.5T], windows in {{8,32,64,128}}",
        "launch": "one CUDA graph per step (shared sweep launches per shape and tile width)",
        "value": nprob / (ms_b * 1e-3), "unit": "evals/s", "ms_per_step": ms_b, "steps": steps, "warmup": warmup,
        "algorithmic_tflops": fl / (ms_b * 1e-3) / 1e12, "frac_of_fp64_peak": fl / (ms_b * 1e-3) / 1e12 / peak,
        "plain": {"value": nprob / (ms_p * 1e-3), "unit": "evals/s", "ms_per_step": ms_p,
                  "algorithmic_tflops": fl / (ms_p * 1e-3) / 1e12,
                  "launch": "one problem after another, each its own launch sequence"},
        "speedup_vs_plain": ms_p / ms_b,
        "latency_ms": {"batched": {"p50": ms_b, "p99": ms_b},
                       "plain": {"p50": float(np.percentile(done_p, 50)), "p99": float(np.percentile(done_p, 99))},
                       "note": "all 96 requests submitted at once; completion time of each (the batch "
                               "completes them together)"},
        "e2e": {"value": nprob / (e2e_ms * 1e-3), "unit": "evals/s", "buffers": "pinned host",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "clocks": clocks,
        "tiles": tile_mix,
    }
    batch.close()
    for p in probs:
        p.close()
    del dev_in, outs
    torch.cuda.empty_cache()
    return out


def run_batched(args):
    import torch
    from paper_2407_13950_gb300 import msqoc

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    sec = batched_section(args, dev, stream, msqoc.measure_fp64_peak(), steps=args.steps, warmup=args.warmup)
    line = {
        "metric": "mixed-batch objective+gradient evals/s", "value": sec["value"], "unit": "evals/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "batched-" + sec["workload"], "launch": sec["launch"],
                   "l2": "inputs larger than L2 (midpoint histories of GBs per step)"},
        **{k: v for k, v in sec.items() if k not in ("value", "unit", "ms_per_step", "workload", "launch")},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_sharded(args, spec):
    """One problem's windows spread over the ranks (shard.ShardedProblem): every rank evaluates
    its contiguous window range on its GPU, hands -2 Lambda across its boundary and joins one
    all-reduce of d + 1 doubles (NCCL).  Strong scaling: the value is evaluations per second of
    the one problem.  Host arrays in, host arrays out (the optimiser's replicated W)."""
    import torch
    from paper_2407_13950_gb300 import msqoc, shard

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl")
    else:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        os.environ.setdefault("MASTER_PORT", "29533")
        dist.init_process_group("gloo", rank=0, world_size=1)
    alpha, W = S.random_alpha(spec, 1), S.random_W(spec, 1)
    sp = shard.ShardedProblem(spec, dist)
    for _ in range(args.warmup):
        sp.eval_gradient(alpha, W)
    dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sp.eval_gradient(alpha, W)
    torch.cuda.synchronize()
    dt = max_over_ranks((time.perf_counter() - t0) / args.steps, dist if world > 1 else None,
                        torch.device("cuda", local))
    line = {"metric": METRIC + " (one problem, windows over ranks)", "value": 1.0 / dt, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {**workload_config(spec), "parallelism": f"windows of one problem over {world} ranks",
                       "windows_per_rank": [b - a + 1 for a, b in sp.ranges]},
            "e2e": {"value": 1.0 / dt, "unit": UNIT, "h2d_bytes_per_step": 8 * (spec.d + (sp.hi - sp.lo)),
                    "d2h_bytes_per_step": 8 * (1 + spec.d + (sp.hi - sp.lo))}}
    sp.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    dist.destroy_process_group()


def run_paper(args):
    """The paper's own test cases (Table 1-2: QFT-4/8/16 on 2/3/4 qubits with exchange coupling,
    full time grids): objective+gradient evaluations per second for each window count, and the
    speedup of the multiple-window evaluation over single shooting (M = 1), the quantity the
    paper reports (8x / 31x / 80x at M = 16 / 128 / 256 on 64 / 1024 / 4096 CPU processes)."""
    import torch
    from paper_2407_13950_gb300 import msqoc

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    out = {}
    cases = ((2, (1, 16)), (3, (1, 128)), (4, (1, 256)))
    if args.qft:
        cases = tuple(c for c in cases if 2 ** c[0] == args.qft)
    fam_names = {1: "fiber", 2: "pair", 3: "quad", 4: "lean"}
    for q, Ms in cases:
        row, tiles = {}, {}
        for M in Ms:
            spec = S.paper_qft_spec(q, M=M)
            alpha, W = S.random_alpha(spec, 1), S.random_W(spec, 1)
            a_d = torch.tensor(alpha, device=dev, dtype=torch.float64)
            W_d = torch.tensor(W if M > 1 else np.zeros(2), device=dev, dtype=torch.float64)
            P_d = torch.zeros(1, device=dev, dtype=torch.float64)
            ga_d = torch.zeros(spec.d, device=dev, dtype=torch.float64)
            gW_d = torch.zeros(max(spec.nW, 2), device=dev, dtype=torch.float64)
            with msqoc.Problem(spec, layout=LAYOUTS[args.layout]) as p:
                tiles[M] = f"{fam_names[p.layout]} x {p.col_block} columns"
                def step():
                    p.eval_gradient_into(a_d, W_d if M > 1 else None, P_d, ga_d, gW_d if M > 1 else None,
                                         stream=stream)
                for _ in range(args.warmup):
                    step()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                for _ in range(args.steps):
                    step()
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / args.steps
            row[M] = ms
        Mbig = Ms[-1]
        out[f"QFT-{2 ** q}"] = {"n_steps": S.PAPER_NSTEPS[q], "ms_per_eval": {str(k): v for k, v in row.items()},
                                "evals_per_s": {str(k): 1e3 / v for k, v in row.items()},
                                "tiles": {str(k): v for k, v in tiles.items()},
                                f"speedup_M{Mbig}_over_M1": row[1] / row[Mbig]}
    head = list(out)[-1]                       # QFT-16 unless --qft selects another case
    q16 = out[head]
    Mh = list(q16["evals_per_s"])[-1]
    line = {"metric": f"{head} objective+gradient evals/s (paper model, M={Mh})", "value": q16["evals_per_s"][Mh],
            "unit": "evals/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": q16["ms_per_eval"][Mh], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "paper's QFT-4/8/16 (Table 1 parameters, Table 2 step counts, exchange coupling)"},
            "cases": out,
            "paper_context": "paper: gradient-evaluation speedup over M=1 of 8x (QFT-4, 16 windows x 4 columns = 64 "
                             "processes), 31x (QFT-8, 1024 processes), 80x (QFT-16, 4096 processes) on Intel "
                             "Sapphire Rapids"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_optimize(args):
    """Time to solution of the paper's optimisation (Sec. 5 settings: amplitude box 25 MHz,
    Tikhonov 1e-3/d, energy 1e-3, window states scaled by sigma = 0.1, stop when the roll-out
    estimate is below 1e-3) on QFT-4 (or QFT-8 with --qft 8) with the paper's full time grid,
    from the paper's random initial guess (+-10 MHz): multiple shooting with 16 (QFT-8: 32)
    windows against single shooting, the
    single-shooting run stopped once its infidelity is below the roll-out infidelity reached
    with 2 windows (the paper's rule for a fair comparison).  Wall clock of whole optimiser runs
    (host-driven L-BFGS; every objective, gradient and regularization on the GPU)."""
    import torch
    from paper_2407_13950_gb300 import msqoc, optimize

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    q = {4: 2, 8: 3, 16: 4}[args.qft or 4]
    M_best, sigma = {2: 16, 3: 32, 4: 64}[q], 0.1      # the paper's best window counts (Table 3)
    if args.opt_windows > 0:
        M_best = args.opt_windows
    reps = max(1, min(args.steps, 3)) if q == 2 else 1

    def solve(M, tol):
        spec = S.paper_qft_spec(q, M=M)
        alpha0 = S.random_alpha(spec, 7, amp=S.PAPER_ALPHA0_AMP)
        st = optimize.paper_settings(spec)
        with msqoc.Problem(spec) as p:
            p.eval_gradient(alpha0, p.rollout(alpha0) if M > 1 else None)   # first-use allocations
            torch.cuda.synchronize()
            times, res = [], None
            for _ in range(reps):
                t0 = time.perf_counter()
                res = optimize.optimize(p, alpha0, tol=tol, max_iter=5000, bound=st["bound"],
                                        gamma_tik=st["gamma_tik"], gamma_energy=st["gamma_energy"],
                                        sigma=sigma if M > 1 else 1.0)
                torch.cuda.synchronize()
                times.append(time.perf_counter() - t0)
        with msqoc.Problem(spec.replace(M=1)) as p1:
            J_ro = p1.eval_objective(res.alpha)["J"]
        return {"M": M, "seconds": float(np.median(times)), "iterations": res.iterations,
                "evaluations": res.evaluations, "converged": bool(res.converged), "estimate": res.estimate,
                "rollout_infidelity": J_ro}

    if q == 4:
        # QFT-16: single shooting (a 0.85 s gradient, ~10^3 iterations) is left out of the bench
        two = single = None
    else:
        two = solve(2, 1e-3)
        single = solve(1, two["rollout_infidelity"])
    best = solve(M_best, 1e-3)
    d = S.paper_qft_spec(q).d
    name = f"QFT-{2 ** q}"
    paper_s = {2: 0.5, 3: 23.0, 4: 720.0}[q]
    line = {"metric": f"{name} optimisation time to solution (paper settings, M={M_best})", "value": best["seconds"],
            "unit": "s", "n_gpus": world, "steps": reps, "warmup": 1, "ms_per_step": best["seconds"] * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": best["seconds"] / paper_s,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{name} (paper Table 1-2 model and grid), Sec. 5 optimisation settings, "
                                   "sigma=0.1, seeded +-10 MHz initial guess"},
            "e2e": {"value": best["seconds"], "unit": "s", "h2d_bytes_per_step": 8 * d, "d2h_bytes_per_step": 8 * d},
            "runs": {"M2": two, "M1": single, f"M{M_best}": best},
            "speedup_over_single_shooting": single["seconds"] / best["seconds"] if single else None,
            "paper_context": {2: "paper Table 3: QFT-4 2.3 s (M=1) and 0.5 s (M=16, 64 CPU processes), 4.3x",
                              3: "paper Table 3: QFT-8 145 s (M=1) and 23 s (M=32, 256 CPU processes), 6.3x",
                              4: "paper Table 3: QFT-16 59 min (M=1) and 12 min (M=64, 1024 CPU processes), "
                                 "4.8x"}[q]}
    if rank == 0:
        print(json.dumps(line), flush=True)


def serving_summary(done, specs, seconds: float, peak: float) -> dict:
    """Completions, algorithmic FP64 throughput and latencies of one serving run, overall and
    by shape (requests of unequal cost are compared by their algorithmic flops)."""
    from paper_2407_13950_gb300 import serving
    fl = sum(serving.eval_flops(specs[r.session], r.gradient) for r in done)
    shapes = sorted({sp.q for sp in specs})
    by = {f"{q}q": [r for r in done if specs[r.session].q == q] for q in shapes}
    return {"evals_per_s": len(done) / seconds, "completed": len(done),
            "completed_by_shape": {k: len(v) for k, v in by.items()},
            "algorithmic_tflops": fl / seconds / 1e12, "frac_of_fp64_peak": fl / seconds / 1e12 / peak,
            "latency_ms": serving.latency_summary(done),
            "latency_by_shape_ms": {k: serving.latency_summary(v) for k, v in by.items() if v}}


def serving_section(args, peak, seconds: float) -> dict:
    """The serving workload: 16 sessions each of 2, 3, 4 and 5 transmons (the 5-transmon ones
    with checkpoint interval 64), a Poisson stream of `args.rate` requests/s (half gradients)
    for `seconds`, served with continuous batching under the arrival-order policy and the
    throughput policy, and one request at a time, on the same request stream."""
    import torch
    from paper_2407_13950_gb300 import serving

    per = args.sessions_per_shape
    shapes = [(S.config_2q(), 0), (S.config_3q(), 0), (S.config_4q(), 0), (S.config_5q(), 64)]
    free, _ = torch.cuda.mem_get_info()
    srv = serving.Server(device_budget_bytes=int(0.85 * free), lookahead=args.lookahead)
    specs, refused = [], 0
    for k in range(per):
        for base, K in shapes:
            try:
                srv.admit(base, ckpt_interval=K)
                specs.append(base)
            except serving.NotAdmitted:
                refused += 1
    # warm-up: an objective and a gradient request of one session per shape (kernel set-up)
    first = {}
    for i, sp in enumerate(specs):
        first.setdefault(sp.q, i)
    warm = [serving.Request(session=i, gradient=g, alpha=S.random_alpha(specs[i], 7, problem=i),
                            W=S.random_W(specs[i], 7, problem=i) if specs[i].M > 1 else None)
            for i in first.values() for g in (False, True)]
    srv.run(warm)
    out = {"workload": f"{len(specs)} sessions ({per} each of 2q, 3q, 4q, 5q; 5q with checkpoint interval 64), "
                       f"Poisson {args.rate:.0f} requests/s for {seconds:.0f} s per run, half gradients",
           "admitted": len(specs), "refused": refused, "budget_bytes": srv.budget, "used_bytes": srv.used,
           "lookahead": srv.lookahead,
           "latency_note": "from_ready: from the head of an idle session's queue (the previous request of "
                           "the session done) to the result; service: dispatch to result; from_arrival "
                           "includes the queue at the session (the offered load exceeds capacity); "
                           "below_capacity: a stream the GPU keeps up with, every request served, latencies "
                           "from arrival"}
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    for policy in ("fifo", "throughput"):
        srv.policy = policy
        reqs = serving.poisson_requests(specs, rate=args.rate, duration=seconds, seed=1)
        done = srv.run(reqs, duration=seconds)
        out["served_" + policy] = serving_summary(done, specs, seconds, peak)
    reqs = serving.poisson_requests(specs, rate=args.rate, duration=seconds, seed=1)
    done = srv.run_plain(reqs, duration=seconds)
    out["plain"] = serving_summary(done, specs, seconds, peak)
    # the same sessions below capacity (about 70% of the GPU one request at a time): latencies
    # are then the servers' own, not queueing at the sessions
    light = {"rate_per_s": args.light_rate, "seconds": args.light_seconds}
    for name, fn in (("served_fifo", srv.run), ("plain", srv.run_plain)):
        srv.policy = "fifo"
        reqs = serving.poisson_requests(specs, rate=args.light_rate, duration=args.light_seconds, seed=2)
        done = fn(reqs, duration=args.light_seconds + 5.0)
        light[name] = serving_summary(done, specs, args.light_seconds, peak)
        light[name]["offered"] = len(reqs)
    out["below_capacity"] = light
    out["clocks"] = sampler.stop()
    srv.close()
    fifo, plain = out["served_fifo"], out["plain"]
    out["fifo_vs_plain"] = {
        "completed_ratio_by_shape": {k: fifo["completed_by_shape"].get(k, 0) / max(v, 1)
                                     for k, v in plain["completed_by_shape"].items()},
        "tflops_ratio": fifo["algorithmic_tflops"] / max(plain["algorithmic_tflops"], 1e-30),
        "p99_from_ready_ms_by_shape": {k: [fifo["latency_by_shape_ms"].get(k, {}).get("from_ready", {}).get("p99"),
                                           v["from_ready"]["p99"]]
                                       for k, v in plain["latency_by_shape_ms"].items()}}
    torch.cuda.empty_cache()
    return out


def run_serving(args):
    import torch
    from paper_2407_13950_gb300 import msqoc

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    sec = serving_section(args, msqoc.measure_fp64_peak(), seconds=args.serve_seconds)
    fifo = sec["served_fifo"]
    line = {
        "metric": "served objective/gradient evals/s", "value": fifo["evals_per_s"], "unit": "evals/s",
        "n_gpus": world, "steps": 1, "warmup": 1, "ms_per_step": args.serve_seconds * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "serving: " + sec["workload"]},
        **{k: v for k, v in sec.items() if k != "workload"},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--windows", type=int, default=256,
                    help="4q workload: windows M (64, 128 or 256 in the workload's configuration)")
    ap.add_argument("--solver", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--col-block", type=int, default=-1,
                    help="columns per sweep tile: -1 = measured by the library's autotuner (default), "
                         "0 = the library's model")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--steps-per-sync", type=int, default=0,
                    help="time steps per history synchronisation of a sweep tile (0: measured by the autotuner "
                         "with --col-block -1, else one)")
    ap.add_argument("--no-extras", action="store_true",
                    help="4q workload: leave out the config3, solver_fp64, batched and serving sub-objects")
    ap.add_argument("--extra-serve-seconds", type=float, default=10.0,
                    help="4q workload: seconds of each serving run inside the default line")
    ap.add_argument("--light-rate", type=float, default=8.0,
                    help="serving: offered requests/s of the below-capacity stream")
    ap.add_argument("--light-seconds", type=float, default=12.0,
                    help="serving: seconds of arrivals of the below-capacity stream")
    ap.add_argument("--lookahead", type=int, default=16,
                    help="serving: requests the arrival-order policy may run ahead of the oldest one")
    ap.add_argument("--layout", choices=list(LAYOUTS), default="auto",
                    help="sweep kernel family: one thread, a lane pair or (2-level subsystems) a lane quad per fiber "
                         "(auto: the library's model)")
    ap.add_argument("--opt-windows", type=int, default=0,
                    help="optimize workload: window count of the multiple-shooting run (0 = the paper's best)")
    ap.add_argument("--nsteps", type=int, default=0,
                    help="shorter time grid with the same step size (small profiling case); 0 = 100000 steps")
    ap.add_argument("--workload", choices=["4q", "batched", "serving", "paper", "optimize", "sharded"], default="4q",
                    help="4q: the benchmark workload (one 4-transmon problem); batched: 96 mixed problems; "
                         "serving: continuous batching of a Poisson request stream; paper: the paper's QFT cases; "
                         "optimize: time to solution of the paper's QFT-4 optimisation; sharded: the 4q problem's "
                         "windows over the ranks (strong scaling)")
    ap.add_argument("--batch-per-shape", type=int, default=32)
    ap.add_argument("--sessions-per-shape", type=int, default=16)
    ap.add_argument("--rate", type=float, default=2000.0, help="serving: offered requests per second")
    ap.add_argument("--serve-seconds", type=float, default=20.0)
    ap.add_argument("--qft", type=int, choices=[4, 8, 16], default=None,
                    help="optimize: the QFT case (default 4; 16 runs only M=64); paper: only this case (default all)")
    args = ap.parse_args()
    if args.workload == "paper":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the paper workloads have no CPU reference run"}))
            return
        run_paper(args)
        return
    if args.workload == "optimize":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the optimisation workload has no CPU reference run"}))
            return
        run_optimize(args)
        return
    if args.workload == "serving":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the serving workload has no CPU reference run"}))
            return
        run_serving(args)
        return
    if args.workload == "batched":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the batched workload has no CPU reference run"}))
            return
        run_batched(args)
        return
    spec = S.config_4q(M=args.windows)
    if args.nsteps:
        spec = spec.replace(nsteps=args.nsteps, T=spec.T * args.nsteps / spec.nsteps,
                            name=f"{spec.name}-{args.nsteps}steps")
    if args.workload == "sharded":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the sharded workload has no CPU reference run"}))
            return
        run_sharded(args, spec)
        return
    if args.impl == "reference":
        run_reference(args, spec)
    else:
        run_ours(args, spec)


if __name__ == "__main__":
    main()
