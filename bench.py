#!/usr/bin/env python
"""Benchmark of the Sinkhorn-UOT hot path on GB300.

Default workload: one UOT problem N=M=16384 in FP32 (1 GiB plan), C = squared
distances of standard-Gaussian 64-D clouds divided by max(C), a/b Dirichlet(1)
times masses 1.0/2.0, reg 0.1, reg_m 0.5, 500 iterations.  A step is the
whole solve: P0 = exp(-C/reg), 500 fused iteration passes plus the finishing
sweep, and the FP64 transport cost.  ``value`` counts plan elements processed
per second (N*M*iters per step) with C, a, b already resident on the GPU;
``e2e`` repeats the same solve through the public API from pinned host
buffers (C, a, b copied in, plan and cost copied out inside the timed region;
steps double-buffered so one step's copies overlap its neighbours' solves).

``--impl reference`` times the FP64 CPU oracle on the same workload instead
(each step is a bounded sample: one oracle iteration on the full-size plan).

Other workloads print one JSON line of their own: ``--workload precision``
(N=M=32768, every storage form, accuracy at 8192^2 against the oracle),
``--workload batched`` (512 uneven problems in one set of launches against a
loop of single-problem launches) and ``--workload grad`` (32 problems of
2048^2, forward and adjoint in one CUDA graph).

Launch: ``python bench.py [--gpus N --steps K --warmup W]``; for N > 1 run it
under ``torch.distributed.run`` -- every rank then solves its own problem
(independent problems, no collective on the data path, weak scaling).
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
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "UOT Sinkhorn plan elems/s & HBM GB/s vs 8 TB/s; fused/bf16/batched vs plain FP32"
UNIT = "plan elems/s"
# The files that define the in-place fused pass itself (the template, its
# device helpers and its instantiation): the recorded DRAM traffic is trusted
# only while they are unchanged.  Host-side launch code and ABI declarations
# are left out so that unrelated additions do not discard the record.
KERNEL_SOURCES = ["paper_2412_11079_gb300/csrc/fused_kernel.cuh",
                  "paper_2412_11079_gb300/csrc/fused_inplace.cu",
                  "paper_2412_11079_gb300/csrc/uot_device.cuh"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "fused_pass_traffic.json")


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.proc = None
        self.path = None
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if bus_id:
                cmd += ["-i", bus_id]
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) == 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def bus_id_of(torch, dev):
    try:
        p = torch.cuda.get_device_properties(dev)
        return f"{p.pci_domain_id:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0"
    except Exception:
        return None


def make_problem(seed: int, args):
    from paper_2412_11079_gb300 import workloads
    return workloads.large_case(seed=seed, n=args.n, m=args.m, iters=args.iters)


def oracle_rate(p, iters: int):
    """FP64 oracle: plan elems/s over `iters` iterations of the full plan."""
    import oracle
    P = oracle.init_plan(p.C, p.reg)
    t0 = time.perf_counter()
    oracle.sinkhorn(P, p.a, p.b, p.reg, p.reg_m, iters)
    dt = time.perf_counter() - t0
    return p.C.size * iters / dt, dt


def run_reference(args, rank: int):
    if rank != 0:
        return
    p = make_problem(0, args)
    import oracle
    P = oracle.init_plan(p.C, p.reg)
    for _ in range(args.warmup):
        P = oracle.sinkhorn(P, p.a, p.b, p.reg, p.reg_m, 1).plan
    t0 = time.perf_counter()
    for _ in range(args.steps):
        P = oracle.sinkhorn(P, p.a, p.b, p.reg, p.reg_m, 1).plan
    dt = time.perf_counter() - t0
    value = p.C.size * args.steps / dt
    sample = (f"{args.steps} oracle iterations (1 per step) on the full {args.n}x{args.m} "
              f"plan, FP64 numpy, after {args.warmup} warm-up iterations")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(args, reference=True),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def roofline_of(kernel: str, alg_bytes_per_launch: float, launch_s: float, peak: float,
                peak_kind: str) -> dict:
    """Roofline sub-object of a comparison: algorithmic bytes of one launch of
    the dominant kernel over its event-timed duration, against the measured
    copy bandwidth."""
    achieved = alg_bytes_per_launch / launch_s / 1e9
    return {"bound": "hbm", "kernel": kernel, "alg_bytes_per_launch": alg_bytes_per_launch,
            "launch_ms": launch_s * 1e3, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_kind": peak_kind, "frac_of_8TBs": achieved / 8000.0}


def measure_precision(args, n: int, iters: int, acc_n: int, reps: int):
    """Reduced-precision workload: N=M=n (2-D uniform points, reg 0.1,
    reg_m 1.0, `iters` iterations) timed for every storage form with CUDA
    events around the iteration passes, and the error of each form against
    the FP64 oracle on the acc_n^2 instance of the same generator (0: none)."""
    import torch

    import oracle
    from paper_2412_11079_gb300 import uot, workloads

    dev = torch.device("cuda", 0)
    peak, peak_kind = measured_peaks()
    C, a, b, reg, reg_m, _ = workloads.uniform2d_device(0, n, n, dev, 0.1, 1.0, iters)
    # (name, storage form, dtype, K storage scale, dominant kernel)
    forms = [("f32", "inplace", torch.float32, 0, "fused_pass_kernel<float,512,8> (cluster of 2)"),
             ("f32", "kform", torch.float32, 0, "fused_pass_kernel<float,512,8,KF> (cluster of 2)"),
             ("bf16", "kform", torch.bfloat16, 0, "kform_pair_kernel<bf16> (cluster of 2)"),
             ("f16", "kform", torch.float16, 15, "kform_pair_kernel<f16> (cluster of 2)"),
             ("bf16", "inplace", torch.bfloat16, 0, "fused_pass_kernel<bf16,512,4> (cluster of 2)"),
             ("f16", "inplace", torch.float16, 0, "fused_pass_kernel<f16,512,4> (cluster of 2)")]
    out = {}
    for name, form, dt, scale, kern in forms:
        mat = torch.empty((n, n), dtype=dt, device=dev)
        opt = uot.options(uot.dtype_code(dt))
        ws = uot.workspace(n, n, opt, dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(); e1.record()
        opt.pass_events[0] = e0.cuda_event
        opt.pass_events[1] = e1.cuda_event
        U = torch.empty(n, device=dev)
        V = torch.empty(n, device=dev)
        times = []
        for rep in range(1 + reps):
            if form == "kform":
                uot.uot_init_kernel_scaled(C, mat, reg, scale, opt)
                uot.uot_sinkhorn_kform(mat, a, b, reg, reg_m, iters, 0.0, scale, U, V, ws, opt)
            else:
                uot.uot_init_kernel(C, mat, reg, opt)
                uot.uot_sinkhorn(plan=mat, a=a, b=b, reg=reg, reg_m=reg_m, iters=iters, ws=ws,
                                 opt=opt, check_status=False)
            torch.cuda.synchronize()
            if rep:
                times.append(e0.elapsed_time(e1) / iters)
        t = min(times)
        bytes_per = (2 if form == "inplace" else 1) * mat.element_size()
        out[f"{name}_{form}"] = {"ms_per_iter": t, "elems_per_s": n * n / (t * 1e-3),
                                 "bytes_per_elem_iter": bytes_per,
                                 "roofline": roofline_of(kern, bytes_per * n * n, t * 1e-3, peak,
                                                         peak_kind)}
        del mat, ws
        torch.cuda.empty_cache()
    del C
    torch.cuda.empty_cache()
    if acc_n:
        q = workloads.precision_case(seed=0, n=acc_n, m=acc_n, iters=iters)
        t0 = time.perf_counter()
        ref = oracle.sinkhorn(oracle.init_plan(q.C, q.reg), q.a, q.b, q.reg, q.reg_m,
                              q.iters).plan
        oracle_s = time.perf_counter() - t0
        ref_cost = oracle.transport_cost(ref, q.C)
        floor = 1e-6 * np.abs(ref).max()
        Cq = torch.from_numpy(q.C).to(dev)
        aq = torch.from_numpy(q.a).to(dev)
        bq = torch.from_numpy(q.b).to(dev)
        for name, form, dt, scale, _ in forms:
            mat = torch.empty(q.C.shape, dtype=dt, device=dev)
            opt = uot.options(uot.dtype_code(dt))
            if form == "kform":
                uot.uot_init_kernel_scaled(Cq, mat, q.reg, scale, opt)
                U, V, _ = uot.uot_sinkhorn_kform(mat, aq, bq, q.reg, q.reg_m, iters, 0.0, scale,
                                                 opt=opt)
                plan = uot.uot_kform_plan(mat, U, V)
                cost = uot.uot_kform_cost(mat, U, V, Cq).item()
            else:
                uot.uot_init_kernel(Cq, mat, q.reg, opt)
                uot.uot_sinkhorn(mat, aq, bq, q.reg, q.reg_m, iters, opt=opt, check_status=False)
                plan = mat
                cost = uot.uot_cost(mat, Cq).item()
            got = plan.double().cpu().numpy()
            err = float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), floor)))
            bar = 1e-5 if name == "f32" else 1e-2
            out[f"{name}_{form}"].update({
                f"plan_max_rel_err_{acc_n}": err,
                f"cost_rel_err_{acc_n}": abs(cost - ref_cost) / abs(ref_cost),
                "bar": bar, "meets_bar": bool(err <= bar and abs(cost - ref_cost) <= bar * abs(ref_cost))})
            del got, plan, mat
        del ref
    base = out["f32_inplace"]["elems_per_s"]
    for v in out.values():
        v["speedup_vs_f32_inplace"] = v["elems_per_s"] / base
    res = {"workload": f"precision N=M={n}, 2-D uniform points, reg 0.1, reg_m 1.0, "
                       f"{iters} iterations",
           "unit": UNIT, "forms": out}
    if acc_n:
        res["accuracy"] = (f"max relative plan-entry error (floor 1e-6 max) and cost error vs the "
                           f"FP64 oracle on the {acc_n}^2 instance, {iters} iterations "
                           f"(oracle {oracle_s:.0f} s on one host core)")
    return res


def measure_batched(args, nprob: int, iters: int, steps: int, warmup: int, compare: bool):
    """Batched workload: `nprob` problems, N and M log-uniform in [64, 4096],
    2-D uniform points, reg in [0.02, 0.2], reg_m log-uniform in [0.1, 10],
    `iters` iterations each; one persistent launch per engine (autotuned
    schedule, captured in a CUDA graph) against loops of single-problem
    launches on the same problems."""
    import torch

    from paper_2412_11079_gb300 import uot, workloads
    from paper_2412_11079_gb300.batch import Batch, autotune

    peak, peak_kind = measured_peaks()
    probs = workloads.batch_uneven(seed=0, count=nprob, iters=iters)
    B = Batch(probs)
    if args.tuning:
        st_, mt_, te_, rc_ = args.tuning.split(",")
        best, timings = uot.batch_tuning(int(st_), int(mt_), float(te_), int(rc_)), {}
        B.prepare(best)
    else:
        best, timings = autotune(B)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        B.init_plans(stream=stream)
        B.run(stream=stream)
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=stream):
            B.init_plans(stream=stream)
            B.run(stream=stream)
    cur = torch.cuda.current_stream()  # replay() launches on the current stream
    for _ in range(warmup):
        g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(cur)
    for _ in range(steps):
        g.replay()
    e1.record(cur)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    res = B.results()
    assert all(r.dev_status == 0 for r in res)
    elems = B.element_iterations
    place = B.placement()
    engines = {"on_chip_problems": sum(1 for c in place if c),
               "on_chip_elements": sum(int(pl.numel()) for pl, c in zip(B.plans, place) if c),
               "streaming_problems": sum(1 for c in place if not c),
               "cluster_sizes": {str(k): place.count(k) for k in sorted(set(place)) if k}}
    # Loops of single-problem launches on the same problems: the in-place
    # fused path, and the kernel form (what the batched engine runs).
    opt = uot.options()
    wss = [uot.workspace(*pl.shape, opt) for pl in B.plans]
    UV = [(torch.empty(pl.shape[0], device=pl.device), torch.empty(pl.shape[1], device=pl.device))
          for pl in B.plans]

    def loop_inplace():
        for p, C, pl, a, b, ws in zip(probs, B.C, B.plans, B.a, B.b, wss):
            uot.uot_init_kernel(C, pl, p.reg, opt)
            uot.uot_sinkhorn(pl, a, b, p.reg, p.reg_m, p.iters, 0.0, ws, opt, sync=False)

    def loop_kform():
        for p, C, pl, a, b, ws, (U, V) in zip(probs, B.C, B.plans, B.a, B.b, wss, UV):
            uot.uot_init_kernel(C, pl, p.reg, opt)
            uot.uot_sinkhorn_kform(pl, a, b, p.reg, p.reg_m, p.iters, 0.0, 0, U, V, ws, opt,
                                   sync=False)
            uot.uot_kform_plan(pl, U, V, pl)

    loop_ms = {}
    for name, fn in (("inplace", loop_inplace), ("kform", loop_kform)) if compare else ():
        fn()
        torch.cuda.synchronize()
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        loop_ms[name] = e0.elapsed_time(e1)
    # Algorithmic bytes: K read once per iteration, plus the init sweep (read
    # C, write K) and the final sweep (read K, write the plan) of every plan.
    alg_bytes = 4.0 * elems + 16.0 * B.elements
    out = {
        "workload": f"batched: {len(probs)} problems, N,M log-uniform [64,4096], "
                    f"{iters} iterations each, FP32",
        "unit": UNIT, "elements": B.elements, "element_iterations": elems,
        "value": elems / (ms * 1e-3), "ms_per_batch": ms,
        "roofline": roofline_of("batched_kernel + resident_kernel (whole batch, one graph)",
                                alg_bytes, ms * 1e-3, peak, peak_kind),
        "tuning": {"stages": best.stages, "max_team": best.max_team,
                   "target_elems": best.target_elems,
                   "resident_max_cluster": best.resident_max_cluster},
        "engines": engines,
        "looped_single_launches": {k: {"ms": v, "value": elems / (v * 1e-3)}
                                   for k, v in loop_ms.items()},
        "batched_over_loop": {k: v / ms for k, v in loop_ms.items()},
        "autotune_ms": {f"{k[0]}/{k[1]}/{k[2]:.0e}/{k[3]}": v for k, v in timings.items()},
    }
    del B
    torch.cuda.empty_cache()
    return out


def measure_grad(args, batch: int, n: int, iters: int, steps: int, warmup: int,
                 check_iters: int):
    """Differentiation workload: `batch` problems N=M=n (16-D Gaussian
    clouds, C/max, reg 0.05, reg_m 1.0), `iters` unrolled iterations, forward
    (kernel form with history) + adjoint backward of <P, C> w.r.t. C, a, b;
    the whole batch captured in one CUDA graph; the forward alone timed on
    the same graph branches."""
    import torch

    import oracle
    from paper_2412_11079_gb300 import uot, workloads

    dev = torch.device("cuda", 0)
    peak, peak_kind = measured_peaks()
    m = n
    probs = workloads.grad_batch(seed=0, count=batch, n=n, m=m, iters=iters)
    B = len(probs)
    ld = (m + 3) // 4 * 4
    # A uniform batch: [B, n, m] tensors, so the adjoint of the whole batch is
    # one set of launches (one reverse launch per step for all problems).
    C3 = torch.stack([torch.from_numpy(p.C) for p in probs]).to(dev)
    a2 = torch.stack([torch.from_numpy(p.a) for p in probs]).to(dev)
    b2 = torch.stack([torch.from_numpy(p.b) for p in probs]).to(dev)
    K3 = torch.empty((B, n, ld), device=dev)[:, :, :m]
    U2, V2 = torch.empty((B, n), device=dev), torch.empty((B, m), device=dev)
    hist2 = uot.grad_hist_batch(B, n, m, iters, dev)
    wss = [uot.workspace(n, m, None, dev) for _ in range(B)]
    dC3 = torch.empty((B, n, ld), device=dev)[:, :, :m]
    da2, db2 = torch.empty((B, n), device=dev), torch.empty((B, m), device=dev)
    cost = torch.empty(B, dtype=torch.float64, device=dev)
    per_problem = args.grad_backward == "per-problem"
    if per_problem:
        bwss = [uot.workspace_bytes(int(uot.load().uot_backward_workspace_size(n, m, iters)), dev)
                for _ in range(B)]
    else:
        bws = uot.workspace_bytes(
            int(uot.load().uot_backward_batch_workspace_size(B, n, m, iters)), dev)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    # The forward solves run as parallel branches (one stream each), every
    # launch limited to a share of the GPU, so the fixed cost of each 16 MB
    # pass overlaps with the other problems' passes.
    branches = [torch.cuda.Stream() for _ in range(min(args.grad_streams, B))]
    opt = uot.options(max_ctas=args.grad_max_ctas)
    bopt = uot.options(max_ctas=args.grad_bwd_max_ctas)
    reg, reg_m = probs[0].reg, probs[0].reg_m

    def step(s, backward=True):
        for br in branches:
            br.wait_stream(s)
        for i in range(B):
            bs = branches[i % len(branches)]
            uot.uot_init_kernel(C3[i], K3[i], reg, stream=bs)
            uot.uot_sinkhorn_kform_save(K3[i], a2[i], b2[i], reg, reg_m, iters, U2[i], V2[i],
                                        hist2[i], wss[i], bs, opt)
            if backward and per_problem:
                uot.uot_kform_cost(K3[i], U2[i], V2[i], C3[i], cost[i:i + 1], bs)
                uot.uot_sinkhorn_backward(K3[i], C3[i], a2[i], b2[i], reg, reg_m, iters,
                                          hist2[i], 1.0, dC3[i], da2[i], db2[i], bwss[i],
                                          bs, bopt)
        for br in branches:
            s.wait_stream(br)
        if backward and not per_problem:
            # The costs after the join: a full-grid cost launch on a branch
            # would hold up the other branches' narrow forward launches.
            for i in range(B):
                uot.uot_kform_cost(K3[i], U2[i], V2[i], C3[i], cost[i:i + 1], s)
            uot.uot_sinkhorn_backward_batch(K3, C3, a2, b2, reg, reg_m, iters, hist2, 1.0, dC3,
                                            da2, db2, bws, s)

    def timed_graph(backward):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(stream):
            step(stream, backward)
            torch.cuda.synchronize()
            with torch.cuda.graph(g, stream=stream):
                step(stream, backward)
        cur = torch.cuda.current_stream()
        for _ in range(warmup):
            g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(cur)
        for _ in range(steps):
            g.replay()
        e1.record(cur)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    ms = timed_graph(True)
    fwd_ms = timed_graph(False)
    elems = len(probs) * n * m * iters
    out = {
        "workload": f"grad: {len(probs)} problems N=M={n}, {iters} iterations, forward + adjoint",
        "unit": UNIT, "value": elems / (ms * 1e-3), "ms_per_step": ms,
        "forward_ms": fwd_ms, "backward_ms": ms - fwd_ms,
        "forward_value": elems / (fwd_ms * 1e-3),
        # Algorithmic bytes: K read once per forward iteration and once per
        # reverse step (4 + 4 B per element and iteration), plus per problem
        # the init (read C, write K), the adjoint's start (read K and C, write
        # and re-read dl) and the final contraction's epilogue (read K and C,
        # write dC): 8 + 16 + 12 B per element.
        "roofline": roofline_of("kform_pair_kernel<float> + reverse_pass_kernel + bw_gemm_kernel "
                                "(whole step)", elems * (4.0 + 4.0) + 36.0 * len(probs) * n * m,
                                ms * 1e-3, peak, peak_kind),
        "forward_branches": len(branches), "max_ctas_per_forward_launch": args.grad_max_ctas,
        "adjoint": ("per problem, on the forward's branches, launches of <= "
                    f"{args.grad_bwd_max_ctas} CTAs" if per_problem else
                    "batched: one reverse launch per step for all problems"),
    }
    del C3, K3, dC3, wss, hist2
    torch.cuda.empty_cache()
    if check_iters:
        # Gradient errors of the first problem at the full size against the
        # oracle's FP64 adjoint on a few iterations (the 200-iteration run is
        # covered by the GPU tests), per element against the magnitude of the
        # terms each entry sums (floor 1e-6 of the largest).
        q = workloads.grad_batch(seed=0, count=1, n=n, m=m, iters=check_iters)[0]
        Cq = torch.from_numpy(q.C).to(dev).requires_grad_(True)
        aq = torch.from_numpy(q.a).to(dev).requires_grad_(True)
        bq = torch.from_numpy(q.b).to(dev).requires_grad_(True)
        from paper_2412_11079_gb300.autograd import sinkhorn_cost
        sinkhorn_cost(Cq, aq, bq, q.reg, q.reg_m, q.iters).backward()
        rv, rdC, rda, rdb = oracle.sinkhorn_grad(q.C, q.a, q.b, q.reg, q.reg_m, q.iters)
        mC, ma, mb = oracle.sinkhorn_grad_magnitude(q.C, q.a, q.b, q.reg, q.reg_m, q.iters)

        def rel(x, r, mag):
            # per entry, against the magnitude of the terms the entry sums
            x = x.double().cpu().numpy()
            return float(np.max(np.abs(x - r) / np.maximum(mag, 1e-6 * mag.max())))

        out["grad_err_vs_term_magnitude"] = {
            "iters": q.iters, "dC": rel(Cq.grad, rdC, mC), "da": rel(aq.grad, rda, ma),
            "db": rel(bq.grad, rdb, mb), "bar": 1e-4}
    return out


def measure_small(args, n: int, iters: int, reps: int):
    """Small workload: N=M=n, 2-D uniform points, reg 0.05, reg_m 1.0,
    `iters` iterations, FP32 in place.  The plan (4 MiB at 1024^2) lives on
    chip, so the per-pass launch dominates: one launch per iteration against
    the persistent schedule (all iterations in one launch, rows held in
    shared memory).  Whole solves timed with CUDA events (init excluded)."""
    import torch

    from paper_2412_11079_gb300 import uot, workloads

    p = workloads.small_case(seed=0, n=n, m=n, iters=iters)
    C = torch.from_numpy(p.C).cuda()
    a = torch.from_numpy(p.a).cuda()
    b = torch.from_numpy(p.b).cuda()
    plan = torch.empty((n, n), device="cuda")
    out = {"workload": f"small: N=M={n}, 2-D uniform points, reg 0.05, reg_m 1.0, "
                       f"{iters} iterations, FP32 in place (plan held on chip)", "unit": UNIT}
    for name, sched in (("per_pass_launches", uot.UOT_SCHED_PASSES),
                        ("persistent", uot.UOT_SCHED_PERSISTENT)):
        opt = uot.options(schedule=sched)
        ws = uot.workspace(n, n, opt)
        best = float("inf")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for rep in range(reps + 1):
            uot.uot_init_kernel(C, plan, p.reg, opt)
            e0.record()
            uot.uot_sinkhorn(plan, a, b, p.reg, p.reg_m, iters, 0.0, ws, opt, sync=False)
            e1.record()
            torch.cuda.synchronize()
            if rep:
                best = min(best, e0.elapsed_time(e1))
        res = uot.uot_read_result(ws, n, n, opt)
        assert res.dev_status == 0 and res.iters_done == iters
        out[name] = {"us_per_iter": best * 1e3 / iters,
                     "value": float(n) * n * iters / (best * 1e-3)}
    out["persistent_over_per_pass"] = (out["persistent"]["value"] /
                                       out["per_pass_launches"]["value"])
    return out


def measure_tensor(args, n1: int, n: int, iters: int, reps: int):
    """Three-way workload: n1 x n x n FP32 plan (2048 x 256 x 256 = 512 MiB,
    larger than L2; a slice of n^2 entries is one row of the fused pass),
    three uniform 2-D point clouds, C = sum of the pairwise squared
    distances, reg 0.1, reg_m 1.0, `iters` iterations; one sweep of the plan
    per iteration plus two small launches forming the mode-2 and mode-3
    factors.  Roofline: one read and one write of the plan per iteration over
    the event-timed iterations (the small launches included)."""
    import torch

    from paper_2412_11079_gb300 import uot, workloads

    dev = torch.device("cuda", 0)
    peak, peak_kind = measured_peaks()
    C, a, b, c, reg, reg_m = workloads.tensor3_device(0, n1, n, n, dev)
    P = torch.empty((n1, n, n), device=dev)
    opt = uot.options()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(); e1.record()
    opt.pass_events[0] = e0.cuda_event
    opt.pass_events[1] = e1.cuda_event
    ws = uot.workspace_bytes(int(uot.load().uot_tensor3_workspace_size(n1, n, n)), dev)
    best = float("inf")
    for rep in range(reps + 1):
        uot.uot_init_kernel(C.view(n1, n * n), P.view(n1, n * n), reg)
        res = uot.uot_sinkhorn_tensor3(P, a, b, c, reg, reg_m, iters, ws, opt)
        assert res.dev_status == 0 and res.iters_done == iters
        if rep:
            best = min(best, e0.elapsed_time(e1) / iters)
    elems = float(n1) * n * n
    out = {"workload": f"three-way: {n1}x{n}x{n} FP32 plan, 2-D uniform points, C = sum of pairwise "
                       f"squared distances, reg 0.1, reg_m 1.0, {iters} iterations", "unit": UNIT,
           "ms_per_iter": best, "value": elems / (best * 1e-3),
           "roofline": roofline_of("fused_pass_kernel<float,512,8> over the mode-1 unfolding "
                                   "+ mode-2/3 factor launches", 8.0 * elems, best * 1e-3, peak,
                                   peak_kind)}
    del C, P
    torch.cuda.empty_cache()
    return out


def run_precision(args):
    import torch  # noqa: F401

    from paper_2412_11079_gb300 import build, uot
    build.build()
    uot.load()
    print(json.dumps(measure_precision(args, args.n, args.iters, args.acc_n, args.steps)),
          flush=True)


def run_batched(args):
    from paper_2412_11079_gb300 import build, uot
    build.build()
    uot.load()
    print(json.dumps(measure_batched(args, args.nprob, args.iters, args.steps, args.warmup,
                                     not args.no_compare)), flush=True)


def run_grad(args):
    from paper_2412_11079_gb300 import build, uot
    build.build()
    uot.load()
    print(json.dumps(measure_grad(args, args.batch, args.n, args.iters, args.steps, args.warmup,
                                  args.grad_check_iters)), flush=True)


def run_shard_rows(args, world: int, rank: int, local: int):
    """The large problem with its rows split over the ranks (Section 5.5):
    each rank holds N/world rows and the column sums are all-reduced (NCCL,
    on the device) between the sharded passes.  Strong scaling: the whole
    job is one problem.  With one rank the reduction is the identity."""
    import torch
    import torch.distributed as dist

    from paper_2412_11079_gb300 import build, shard, uot

    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    uot.load()
    p = make_problem(0, args)
    n, m, iters = args.n, args.m, args.iters
    lo, hi = rank * n // world, (rank + 1) * n // world
    C = torch.from_numpy(np.ascontiguousarray(p.C[lo:hi])).to(dev)
    a = torch.from_numpy(p.a[lo:hi].copy()).to(dev)
    b = torch.from_numpy(p.b).to(dev)
    plan = torch.empty((hi - lo, m), device=dev)
    allreduce = (lambda t: dist.all_reduce(t)) if world > 1 else (lambda t: None)

    def step():
        uot.uot_init_kernel(C, plan, p.reg)
        return shard.sinkhorn_rows(plan, a, b, p.reg, p.reg_m, iters, allreduce)

    for _ in range(args.warmup):
        assert step() == 0
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(bus_id_of(torch, dev)) if rank == 0 else None
    launches0 = uot.uot_launch_count()
    start.record()
    for _ in range(args.steps):
        step()
    stop.record()
    torch.cuda.synchronize()
    launches = uot.uot_launch_count() - launches0
    clocks = sampler.stop() if sampler else None
    ms = start.elapsed_time(stop)
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = t.item()
    value = float(n) * m * iters * args.steps / (ms * 1e-3)
    if rank == 0:
        cfg = config_of(args)
        cfg.update({"algo": "fused one-pass, plan in place, rows sharded over the ranks "
                            "(column sums all-reduced between passes)",
                    "parallelism": f"rows/{world}"})
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic", "config": cfg, "gpu_launches": launches,
            "clocks": clocks}), flush=True)
    if world > 1:
        dist.destroy_process_group()


def config_of(args, reference: bool = False):
    c = {"workload": f"single UOT problem N=M={args.n}" if args.n == args.m else
         f"single UOT problem {args.n}x{args.m}",
         "n": args.n, "m": args.m, "iters": args.iters, "reg": 0.1, "reg_m": 0.5,
         "cost": "squared distances of N(0, I_64) clouds / max",
         "marginals": "Dirichlet(1) x 1.0 / x 2.0"}
    if reference:
        c.update({"plan_dtype": "f64", "algo": "FP64 numpy oracle (row step, then column step)",
                  "sample": "one iteration per step on the full plan"})
    else:
        kform = getattr(args, "storage", "inplace") == "kform"
        c.update({"plan_dtype": "f32",
                  "algo": "fused one-pass, plan kept as K with FP32 scalings (kernel-form "
                          "storage), written once at the end" if kform else
                          "fused one-pass, plan in place",
                  "l2": "plan (1 GiB) larger than L2, no flush needed"})
    return c


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--m", type=int, default=16384)
    ap.add_argument("--iters", type=int, default=500)
    ap.add_argument("--oracle-iters", type=int, default=20)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--workload", default="large",
                    choices=["large", "precision", "batched", "grad", "small", "tensor"])
    ap.add_argument("--storage", default="inplace", choices=["inplace", "kform"],
                    help="large workload: how uot_sinkhorn keeps the plan (kform: the buffer "
                         "kept as K with FP32 scalings)")
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--nprob", type=int, default=512,
                    help="batched workload: number of problems")
    ap.add_argument("--tuning", default="",
                    help="batched workload: fixed schedule stages,max_team,target,cluster "
                         "(skips the autotuner)")
    ap.add_argument("--grad-check-iters", type=int, default=5)
    ap.add_argument("--no-extra", action="store_true",
                    help="default run: skip the precision, batched and gradient comparisons")
    ap.add_argument("--grad-streams", type=int, default=32)
    ap.add_argument("--grad-max-ctas", type=int, default=24)
    ap.add_argument("--grad-bwd-max-ctas", type=int, default=80,
                    help="CTA cap of the per-problem adjoint's launches")
    ap.add_argument("--grad-backward", choices=["batched", "per-problem"], default="batched")
    ap.add_argument("--acc-n", type=int, default=8192)
    ap.add_argument("--shard", default="", choices=["", "rows"],
                    help="rows: the large problem's rows split over the ranks, column sums "
                         "all-reduced between passes (strong scaling)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.shard == "rows":
        run_shard_rows(args, world, rank, local)
        return
    if args.workload == "grad":
        if args.n == 16384 and args.m == 16384:
            args.n = args.m = 2048
        if args.iters == 500:
            args.iters = 200
        run_grad(args)
        return
    if args.workload == "batched":
        if args.iters == 500:
            args.iters = 200
        run_batched(args)
        return
    if args.workload == "small":
        from paper_2412_11079_gb300 import build, uot
        build.build()
        uot.load()
        n = 1024 if args.n == 16384 else args.n
        print(json.dumps(measure_small(args, n, 100 if args.iters == 500 else args.iters,
                                       args.steps)), flush=True)
        return
    if args.workload == "tensor":
        from paper_2412_11079_gb300 import build, uot
        build.build()
        uot.load()
        print(json.dumps(measure_tensor(args, 2048, 256, 100 if args.iters == 500 else args.iters,
                                        args.steps)), flush=True)
        return
    if args.workload == "precision":
        if args.n == 16384 and args.m == 16384:
            args.n = args.m = 32768
        if args.iters == 500:
            args.iters = 300
        run_precision(args)
        return

    import torch
    import torch.distributed as dist

    from paper_2412_11079_gb300 import build, uot

    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    uot.load()

    p = make_problem(rank, args)
    n, m, iters = args.n, args.m, args.iters
    stream = torch.cuda.current_stream(dev)
    C = torch.from_numpy(p.C).to(dev)
    a = torch.from_numpy(p.a).to(dev)
    b = torch.from_numpy(p.b).to(dev)
    plan = torch.empty((n, m), dtype=torch.float32, device=dev)
    cost = torch.empty(1, dtype=torch.float64, device=dev)
    storage = uot.UOT_STORAGE_KFORM if args.storage == "kform" else uot.UOT_STORAGE_INPLACE
    opt = uot.options(storage=storage)
    ws = uot.workspace(n, m, opt, dev)

    def step(o):
        uot.uot_init_kernel(C, plan, p.reg, opt, stream)
        uot.uot_sinkhorn(plan, a, b, p.reg, p.reg_m, iters, 0.0, ws, o, stream, sync=False)
        uot.uot_cost(plan, C, cost, stream)

    for _ in range(args.warmup):
        step(opt)
    torch.cuda.synchronize()
    res = uot.uot_read_result(ws, n, m, opt)
    if res.dev_status != 0 or res.iters_done != iters:
        raise RuntimeError(f"solve failed: {res}")

    # Timed region: K steps, CUDA events on the launching stream; the fused
    # passes of each step are bracketed by their own event pair.
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    opts = []
    for e0, e1 in evs:
        e0.record(stream)  # torch creates the underlying cudaEvent on first record
        e1.record(stream)
        o = uot.options(storage=storage)
        o.pass_events[0] = e0.cuda_event
        o.pass_events[1] = e1.cuda_event
        opts.append(o)
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(bus_id_of(torch, dev)) if rank == 0 else None
    time.sleep(0.3 if sampler else 0.0)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = uot.uot_launch_count()
    start.record(stream)
    for k in range(args.steps):
        step(opts[k])
    stop.record(stream)
    torch.cuda.synchronize()
    launches = uot.uot_launch_count() - launches0
    clocks = sampler.stop() if sampler else None
    elapsed_ms = start.elapsed_time(stop)
    pass_ms = sum(e0.elapsed_time(e1) for e0, e1 in evs)
    if world > 1:
        t = torch.tensor([elapsed_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = t.item()
        dist.barrier()
    ms_step = elapsed_ms / args.steps
    elems = float(n) * m * iters * args.steps * world
    value = elems / (elapsed_ms * 1e-3)
    res = uot.uot_read_result(ws, n, m, opt)
    assert res.dev_status == 0 and res.iters_done == iters

    # Roofline of the dominant kernel (the fused pass): algorithmic bytes per
    # launch = one read and one write of the FP32 plan = 8*N*M (kernel-form
    # storage: one read, 4*N*M).
    per_launch_s = pass_ms * 1e-3 / (args.steps * iters)
    alg_bytes = (4.0 if args.storage == "kform" else 8.0) * n * m
    achieved = alg_bytes / per_launch_s / 1e9
    peak, peak_kind = measured_peaks()
    traffic = None
    if os.path.exists(TRAFFIC_FILE):
        with open(TRAFFIC_FILE) as fh:
            tr = json.load(fh)
        if tr.get("source_hash") == kernel_hash() and args.storage == "inplace":
            traffic = tr["bytes_per_elem"] * n * m

    # End to end through the public API from pinned host buffers: every step
    # copies its inputs in, solves (init, iterations, cost) and reads its plan
    # and cost back.  Steps are double-buffered on three streams, so one
    # step's copies overlap the neighbouring steps' solves.
    hC = torch.from_numpy(p.C).pin_memory()
    ha = torch.from_numpy(p.a).pin_memory()
    hb = torch.from_numpy(p.b).pin_memory()
    hplan = [torch.empty((n, m), dtype=torch.float32).pin_memory() for _ in range(2)]
    hcost = [torch.empty(1, dtype=torch.float64).pin_memory() for _ in range(2)]
    e2e_steps = max(2, args.steps)  # the same K steps as the device-timed line
    dC = [C, torch.empty_like(C)]
    dplan = [plan, torch.empty_like(plan)]
    da = [a, torch.empty_like(a)]
    db = [b, torch.empty_like(b)]
    dcost = [cost, torch.empty_like(cost)]
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def e2e_run(nsteps):
        ev_in = [torch.cuda.Event() for _ in range(nsteps)]
        ev_done = [torch.cuda.Event() for _ in range(nsteps)]
        ev_out = [torch.cuda.Event() for _ in range(nsteps)]
        for k in range(nsteps):
            j = k % 2
            with torch.cuda.stream(s_in):
                if k >= 2:
                    s_in.wait_event(ev_done[k - 2])  # buffers j free again
                dC[j].copy_(hC, non_blocking=True)
                da[j].copy_(ha, non_blocking=True)
                db[j].copy_(hb, non_blocking=True)
                ev_in[k].record(s_in)
            stream.wait_event(ev_in[k])
            if k >= 2:
                stream.wait_event(ev_out[k - 2])  # plan j read back
            uot.uot_init_kernel(dC[j], dplan[j], p.reg, opt, stream)
            uot.uot_sinkhorn(dplan[j], da[j], db[j], p.reg, p.reg_m, iters, 0.0, ws, opt, stream,
                             sync=False)
            uot.uot_cost(dplan[j], dC[j], dcost[j], stream)
            ev_done[k].record(stream)
            with torch.cuda.stream(s_out):
                s_out.wait_event(ev_done[k])
                hplan[j].copy_(dplan[j], non_blocking=True)
                hcost[j].copy_(dcost[j], non_blocking=True)
                ev_out[k].record(s_out)
        stream.wait_event(ev_out[nsteps - 1])

    e2e_run(2)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    s_in.wait_stream(stream)
    e2e_run(e2e_steps)
    s1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = s0.elapsed_time(s1)
    if world > 1:
        t = torch.tensor([e2e_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = t.item()
    e2e_value = float(n) * m * iters * e2e_steps * world / (e2e_ms * 1e-3)
    h2d = hC.numel() * 4 + ha.numel() * 4 + hb.numel() * 4
    d2h = hplan[0].numel() * 4 + 8
    res_e2e = float(hcost[(e2e_steps - 1) % 2].item())
    if not math.isfinite(res_e2e):
        raise RuntimeError("end-to-end solve returned a non-finite cost")
    del dC[1], dplan[1], da[1], db[1], dcost[1]

    compare = None
    if not args.no_compare and rank == 0:
        compare = {}
        q0 = torch.cuda.Event(enable_timing=True)
        q1 = torch.cuda.Event(enable_timing=True)

        def timed_solves(o, its, reps=2):
            uot.uot_init_kernel(C, plan, p.reg, o, stream)
            uot.uot_sinkhorn(plan, a, b, p.reg, p.reg_m, its, 0.0, ws_of(o), o, stream,
                             sync=False)
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(reps)]
            q0.record(stream)
            for e0, e1 in ev:
                e0.record(stream); e1.record(stream)
                oo = uot.options(algo=o.algo, storage=o.storage, deterministic=bool(o.deterministic))
                oo.pass_events[0] = e0.cuda_event
                oo.pass_events[1] = e1.cuda_event
                uot.uot_init_kernel(C, plan, p.reg, o, stream)
                uot.uot_sinkhorn(plan, a, b, p.reg, p.reg_m, its, 0.0, ws_of(o), oo, stream,
                                 sync=False)
            q1.record(stream)
            torch.cuda.synchronize()
            total_s = q0.elapsed_time(q1) * 1e-3
            pass_s = sum(e0.elapsed_time(e1) for e0, e1 in ev) * 1e-3 / (reps * its)
            return float(n) * m * its * reps / total_s, pass_s

        wss = {}

        def ws_of(o):
            key = bool(o.deterministic)
            if key not in wss:
                wss[key] = uot.workspace(n, m, o, dev)
            return wss[key]

        # Plain multi-pass FP32 on the same GPU and problem (3 reads + 2 writes
        # + 1 read of the plan per iteration).
        mp_iters = min(iters, 100)
        mp_value, mp_pass = timed_solves(uot.options(algo=uot.UOT_ALGO_MULTIPASS), mp_iters)
        compare["plain_fp32_multipass"] = {"value": mp_value, "unit": UNIT, "iters": mp_iters,
                                           "init_included": True}
        compare["fused_over_multipass"] = value / world / mp_value
        # The same solve with kernel-form storage: the buffer is read once per
        # iteration (4 bytes per element) and written once at the end.
        ks_value, ks_pass = timed_solves(uot.options(storage=uot.UOT_STORAGE_KFORM), iters)
        compare["fp32_kform_storage"] = {
            "value": ks_value, "unit": UNIT, "iters": iters, "init_included": True,
            "over_fused_in_place": ks_value / (value / world),
            "roofline": roofline_of("fused_pass_kernel<float,512,8,KF>", 4.0 * n * m, ks_pass,
                                    peak, peak_kind)}
        # Deterministic mode of the headline solve (static rows, ordered sums).
        dt_value, dt_pass = timed_solves(uot.options(deterministic=True), iters, reps=1)
        compare["fp32_in_place_deterministic"] = {
            "value": dt_value, "unit": UNIT, "iters": iters, "init_included": True,
            "over_fused_in_place": dt_value / (value / world),
            "roofline": roofline_of("fused_pass_kernel<float,512,8> + det_reduce_kernel",
                                    8.0 * n * m, dt_pass, peak, peak_kind)}
        # BF16 kernel form (read-only K, FP32 scalings) on the same problem.
        K16 = torch.empty((n, m), dtype=torch.bfloat16, device=dev)
        ko = uot.options(uot.UOT_BF16)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream); e1.record(stream)
        ko.pass_events[0] = e0.cuda_event
        ko.pass_events[1] = e1.cuda_event
        U = torch.empty(n, device=dev)
        V = torch.empty(m, device=dev)
        uot.uot_init_kernel_scaled(C, K16, p.reg, 0, ko)
        uot.uot_sinkhorn_kform(K16, a, b, p.reg, p.reg_m, iters, 0.0, 0, U, V, ws, ko, sync=False)
        torch.cuda.synchronize()
        q0.record(stream)
        for _ in range(2):
            uot.uot_sinkhorn_kform(K16, a, b, p.reg, p.reg_m, iters, 0.0, 0, U, V, ws, ko,
                                   sync=False)
        q1.record(stream)
        torch.cuda.synchronize()
        kf_value = float(n) * m * iters * 2 / (q0.elapsed_time(q1) * 1e-3)
        kf_pass = e0.elapsed_time(e1) * 1e-3 / iters
        del K16
        wss.clear()
        compare["bf16_kernel_form"] = {
            "value": kf_value, "unit": UNIT, "iters": iters,
            "over_fused_in_place": kf_value / (value / world),
            "roofline": roofline_of("kform_pair_kernel<bf16> (16384 columns per CTA)", 2.0 * n * m, kf_pass,
                                    peak, peak_kind)}
        if not args.no_extra:
            del dC, dplan, da, db, dcost
            torch.cuda.empty_cache()
            # The other workloads, bounded so the default run stays within a
            # few minutes: the small on-chip problem (N=M=1024), reduced
            # precision at N=M=32768 (accuracy at 8192^2), 512 uneven
            # problems, and 32 problems forward + adjoint.  Each reports its own elements/s against the plain
            # FP32 path and the roofline of its dominant kernel.
            t0 = time.perf_counter()
            compare["small_1024"] = measure_small(args, 1024, 100, 5)
            compare["tensor3_2048x256x256"] = measure_tensor(args, 2048, 256, 100, 2)
            compare["precision_32768"] = measure_precision(args, 32768, 300, args.acc_n, 2)
            compare["batched_512"] = measure_batched(args, 512, 200, 3, 3, True)
            compare["grad_32x2048"] = measure_grad(args, 32, 2048, 200, 3, 3,
                                                   args.grad_check_iters)
            compare["extra_wall_s"] = time.perf_counter() - t0

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rate, dt = oracle_rate(p, args.oracle_iters)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{args.oracle_iters} of {iters} iterations of the FP64 numpy oracle "
                         f"on the full {n}x{m} plan ({dt:.1f} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic", "config": config_of(args),
            "hbm_gbs_algorithmic": alg_bytes * iters * args.steps * world
            / (elapsed_ms * 1e-3) / 1e9,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_kind": peak_kind,
                         "kernel": "fused_pass_kernel<float,512,8>" +
                                   (",KF (kernel-form storage)" if args.storage == "kform" else ""),
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs: a device copy probe "
                                        "(read + write bytes over time), not a hard ceiling",
                         "frac_of_8TBs": achieved / 8000.0,
                         "launch_ms": per_launch_s * 1e3},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": e2e_steps,
                    "pipelining": "double-buffered: copies on two side streams overlap "
                                  "the neighbouring steps' solves"},
            "gpu_launches": launches, "clocks": clocks, "compare": compare,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
