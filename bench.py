#!/usr/bin/env python
"""Benchmark of the walk-on-ellipsoids operator build on GB300.

One step = the whole hot path on the two-geometry workload of anisotropic
2-D Cauchy problems: for the unit square and for the annulus r in [0.5, 1]
(K = [[1, .5], [.5, 2]], 256 boundary elements, 256 jittered interior
points, N = 1e5 walks per point, eps = 1e-5, FP32 walks): the Monte Carlo
operator build (MC-REM), the FP64 one-sided Jacobi SVD of the Gamma_1 block
and the TSVD reconstruction from measurements with 1 % Gaussian noise.

Prints one JSON line (metric, value = walks/s over all GPUs, roofline of the
walk kernel, CPU baseline = the FP64 oracle on the host cores, e2e = the same
through the public API with host buffers).  ``--impl reference`` times the
CPU oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = ("WoS walks/s and steps/s on 1 GB300 (% FP32/SFU roofline); "
          "served p50/p99 latency")
# ALU issue peak of one GB300: 152 SMs x 4 schedulers x 32 lanes per clock
# at the 2070 MHz maximum SM clock (lane-operations per second).
ALU_PEAK_GOPS = 152 * 4 * 32 * 2.070
# Algorithmic lane-operations of one step of the chain (FP32, 2-D, full S):
# Philox4x32-10 share 80/4 = 20, uniform 3, sin/cos 4, move 6, eps and cap
# tests 3, step counter 1, plus the distance: box 5, disc-minus-disc 9.
OPS_PER_STEP = {"box": 42, "annulus": 46}
PROFILE_NOTE = ROOT / "profiles" / "walk_kernel_square_annulus.md"


def _walk_kernel_hash() -> str:
    h = hashlib.sha256()
    for f in ("walk_kernel.cuh", "wos_device.cuh"):
        h.update((ROOT / "paper_2409_03686_gb300" / "csrc" / f).read_bytes())
    return h.hexdigest()[:16]


def _traffic_from_profile():
    """DRAM bytes per walk-kernel launch from the committed ncu summary, if it
    was taken on the current kernel source."""
    if not PROFILE_NOTE.exists():
        return None
    vals = {}
    for line in PROFILE_NOTE.read_text().splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_hash") != _walk_kernel_hash():
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def workload(name: str):
    from paper_2409_03686_gb300 import workloads as W
    if name == "square-annulus":
        return [W.square_config(), W.annulus_config()]
    if name == "small":  # for ncu captures: same kernels, smaller sizes
        return [W.square_config(N=20_000, grid=8), W.annulus_config(N=20_000, grid=8)]
    raise SystemExit(f"unknown workload {name}")


def describe(name: str) -> dict:
    if name == "square-annulus":
        return {"workload": ("2-D anisotropic Cauchy operator: unit square [-1/2,1/2]^2 "
                             "and annulus r in [0.5,1], K=[[1,0.5],[0.5,2]], 256 boundary "
                             "elements each (Gamma_1 = 128), 256 jittered interior points, "
                             "N=1e5 walks/point, eps=1e-5, FP32 walks; FP64 Jacobi SVD of "
                             "the 256x128 Gamma_1 block; TSVD of 1% noisy data"),
                "walks_per_step": 2 * 256 * 100_000,
                "l2": "flushed between timed steps (256 MiB write)",
                "parallelism": "replicas (one full workload per GPU)"}
    return {"workload": name}


# ----------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        self.path = None

    def start(self):
        try:
            out = ROOT / "gpurun_out"
            out.mkdir(exist_ok=True)
            self.path = out / f"clocks_gpu{self.gpu}.csv"
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# CPU oracle (the baseline and the reference arm)
# ----------------------------------------------------------------------------
def oracle_sample(insts, n_points: int, n_walks: int):
    """Times the oracle's MC-REM on the first n_points points with n_walks
    walks each, for every instance; returns (walks, steps, seconds)."""
    from oracle import oracle as O
    O.build()
    walks = steps = 0
    t0 = time.perf_counter()
    for inst in insts:
        sub = inst.replace(points=inst.points[:n_points], N=n_walks)
        C, U, s = O.build_counts(sub)
        walks += sub.M_D * sub.N
        steps += s
    return walks, steps, time.perf_counter() - t0


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    insts = workload(args.workload)
    n_pts, n_walks = 32, 100_000
    times, walks, steps = [], 0, 0
    for it in range(args.warmup + args.steps):
        w, s, dt = oracle_sample(insts, n_pts, n_walks)
        if it >= args.warmup:
            times.append(dt)
            walks += w
            steps += s
    total = sum(times)
    value = walks / total
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "walks/s",
        "steps_per_s": steps / total, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "config": describe(args.workload),
        "cpu_baseline": {"value": value, "unit": "walks/s", "cores": cores,
                         "kind": "oracle",
                         "sample": f"first {n_pts} points x {n_walks} walks of each "
                                   f"of the {len(insts)} instances per step (FP64 C "
                                   f"oracle, {cores} threads)"},
        "e2e": {"value": value, "unit": "walks/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ----------------------------------------------------------------------------
# the GPU arm
# ----------------------------------------------------------------------------
def pick_rank(S: np.ndarray) -> int:
    """Truncation at the first gap s_r / s_{r+1} >= 1.5 after s_r / s_1 < 1e-3
    (else the last gap before it)."""
    k = len(S)
    gaps = [r for r in range(1, k) if S[r] > 0 and S[r - 1] / S[r] >= 1.5]
    after = [r for r in gaps if S[r - 1] / S[0] < 1e-3]
    if after:
        return after[0]
    return gaps[-1] if gaps else k


def run_gpu(args, rank: int, world: int, dist):
    import torch
    from paper_2409_03686_gb300 import workloads as W
    from paper_2409_03686_gb300 import wos

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2409_03686_gb300 import build as B
    B.build()
    ctx = wos.Context(local)
    stream = torch.cuda.current_stream()
    insts = workload(args.workload)
    prep = []
    for inst in insts:
        meas = W.measurements(inst, noise=0.01, seed=3)
        sig = wos.wos_element_measures(inst.domain, inst.partition)
        p = dict(inst=inst,
                 points=torch.as_tensor(inst.points, dtype=torch.float64, device=dev),
                 sigma=torch.as_tensor(sig, device=dev),
                 uD=torch.as_tensor(meas.uD, device=dev),
                 u0=torch.as_tensor(meas.u0, device=dev),
                 ev=(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)),
                 host=dict(points=torch.as_tensor(inst.points).pin_memory(),
                           uD=torch.as_tensor(meas.uD).pin_memory(),
                           u0=torch.as_tensor(meas.u0).pin_memory()))
        for e in p["ev"]:
            e.record(stream)
        prep.append(p)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    streams = [torch.cuda.Stream(device=dev) for _ in prep]

    def one(p, timing_events=None, host_io=False, stream=None):
        inst = p["inst"]
        opts = wos.make_opts(precision=0, stream_id=inst.stream,
                             kernel_events=timing_events)
        if host_io:
            pts = p["host"]["points"].to(dev, non_blocking=True)
            uD = p["host"]["uD"].to(dev, non_blocking=True)
            u0 = p["host"]["u0"].to(dev, non_blocking=True)
        else:
            pts, uD, u0 = p["points"], p["uD"], p["u0"]
        sol = wos.solve_instance(ctx, inst, uD, u0, p["r"], points=pts, sigma=p["sigma"],
                                 opts=opts, stream=stream)
        if host_io:
            c = sol.counts.to("cpu", non_blocking=True)
            u1 = sol.u_gamma1.to("cpu", non_blocking=True)
            return sol, (c, u1)
        return sol, None

    # warm-up: truncation ranks from the spectra, step counts from stats
    steps_per_inst = []
    for p in prep:
        p["r"] = 1
        inst = p["inst"]
        c, u, st = wos.wos_build_operator(ctx, inst.domain, inst.K, p["points"],
                                          inst.partition, inst.N, inst.eps, inst.seed,
                                          opts=wos.make_opts(stream_id=inst.stream))
        U, S, V, sw = wos.wos_op_svd(ctx, c, inst.N, inst.partition.gamma1, p["sigma"])
        p["r"] = pick_rank(S.cpu().numpy())
        p["steps"] = st["steps"]
        p["kind"] = "box" if inst.domain.outer == "box" else "annulus"
        steps_per_inst.append(st["steps"])
    def step(timing=None, host_io=False, start_ev=None):
        """One step: every instance's pipeline on its own stream, joined on
        the current stream (instances overlap on the GPU)."""
        main = torch.cuda.current_stream()
        outs = []
        done = []
        for q, p in enumerate(prep):
            s = streams[q]
            if start_ev is not None:
                s.wait_event(start_ev)
            else:
                s.wait_stream(main)
            with torch.cuda.stream(s):
                outs.append(one(p, timing_events=timing[q] if timing else None,
                                host_io=host_io, stream=s))
                ev = torch.cuda.Event()
                ev.record(s)
                done.append(ev)
        for ev in done:
            main.wait_event(ev)
        return outs

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- device-timed steps --------------------------------------------------
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in prep] for _ in range(args.steps)]
    for row in kev:  # create the events; the library re-records them around the kernel
        for pair in row:
            for e in pair:
                e.record(stream)
    clocks = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = ctx.kernel_launches()
    clocks.start()
    t_wall = time.perf_counter()
    for it in range(args.steps):
        flush.zero_()
        starts[it].record(stream)
        step(timing=kev[it], start_ev=starts[it])
        ends[it].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    launches = ctx.kernel_launches() - launches0
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = sum(step_ms)
    if dist is not None:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    walks_per_step = sum(p["inst"].M_D * p["inst"].N for p in prep)
    steps_per_step = sum(steps_per_inst)
    value = world * walks_per_step * args.steps / (total_ms / 1e3)
    steps_per_s = world * steps_per_step * args.steps / (total_ms / 1e3)

    # roofline of the walk kernel: algorithmic lane-operations / kernel time.
    # The instances overlap on the GPU, so the kernel time of a step is the
    # union of its walk-kernel intervals (CUDA events on the launching
    # streams, placed relative to the step's start event).
    ops = sum(OPS_PER_STEP[p["kind"]] * p["steps"] for p in prep)
    unions = []
    for it in range(args.steps):
        iv = sorted((starts[it].elapsed_time(a), starts[it].elapsed_time(b))
                    for (a, b) in kev[it])
        tot, cur0, cur1 = 0.0, None, None
        for a, b in iv:
            if cur1 is None or a > cur1:
                if cur1 is not None:
                    tot += cur1 - cur0
                cur0, cur1 = a, b
            else:
                cur1 = max(cur1, b)
        tot += cur1 - cur0
        unions.append(tot)
    kernel_ms_step = float(np.mean(unions))
    achieved = ops / (kernel_ms_step / 1e3) / 1e9
    traffic = _traffic_from_profile()

    # ---- e2e: public API with host buffers and copies in the timed region ---
    e2e_s = torch.cuda.Event(enable_timing=True)
    e2e_e = torch.cuda.Event(enable_timing=True)
    h2d = sum(p["host"][k].numel() * 8 for p in prep for k in ("points", "uD", "u0"))
    d2h = 0
    torch.cuda.synchronize()
    e2e_s.record(stream)
    for it in range(args.steps):
        outs = step(host_io=True)
        d2h = sum(o[1][0].numel() * 4 + o[1][1].numel() * 8 for o in outs)
    e2e_e.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e2e_s.elapsed_time(e2e_e)
    if dist is not None:
        t = torch.tensor([e2e_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
    e2e_value = world * walks_per_step * args.steps / (e2e_ms / 1e3)

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "walks/s", "steps_per_s": steps_per_s,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": describe(args.workload),
        "steps_per_walk": steps_per_step / walks_per_step,
        "walk_kernel_ms_per_step": kernel_ms_step,
        "truncation_r": [p["r"] for p in prep],
        "roofline": {"bound": "alu", "achieved": achieved, "peak": ALU_PEAK_GOPS,
                     "unit": "Gop/s", "frac": achieved / ALU_PEAK_GOPS,
                     "traffic": traffic,
                     "peak_source": "152 SMs x 4 schedulers x 32 lanes x 2070 MHz "
                                    "(recipe unit counts and max clock)"},
        "gpu_launches": int(launches),
        "wall_s_timed": wall,
        "e2e": {"value": e2e_value, "unit": "walks/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "clocks": clk,
    }
    if not args.no_cpu_baseline and world == 1:
        n_pts, n_walks = 32, 100_000
        w, s, dt = oracle_sample([p["inst"] for p in prep], n_pts, n_walks)
        line["cpu_baseline"] = {
            "value": w / dt, "unit": "walks/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"first {n_pts} points x {n_walks} walks of each instance "
                      f"({w} walks, {dt:.1f} s, FP64 C oracle)"}
    print(json.dumps(line))


def run_batch(args, rank: int, world: int, dist):
    """Config 4: the 64-instance mixed batch (disc, annulus, square, L-shape,
    ball, box; log-uniform sizes and walks per point) in one autotuned
    persistent launch per dimension, against one plain launch per instance
    (default launch settings) on the same GPU.  Operator builds only."""
    import torch
    from paper_2409_03686_gb300 import build as B
    from paper_2409_03686_gb300 import workloads as W
    from paper_2409_03686_gb300 import wos
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.build()
    ctx = wos.Context(local)
    insts = W.mixed_batch(64, scale=args.batch_scale)
    pts = [torch.as_tensor(i.points, dtype=torch.float64, device=dev) for i in insts]
    walks = sum(i.M_D * i.N for i in insts)
    # sequential plain launches (no tuning in the context yet)
    counts_seq = []
    def sequential():
        out = []
        for inst, p in zip(insts, pts):
            c, u, _ = wos.wos_build_operator(ctx, inst.domain, inst.K, p, inst.partition,
                                             inst.N, inst.eps, inst.seed,
                                             opts=wos.make_opts(stream_id=inst.stream),
                                             stats=False)
            out.append(c)
        return out
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    def timed(fn, reps):
        ms = []
        for _ in range(reps):
            torch.cuda.synchronize()
            ev0.record()
            r = fn()
            ev1.record()
            torch.cuda.synchronize()
            ms.append(ev0.elapsed_time(ev1))
        return r, ms
    sequential()
    seq_out, seq_ms = timed(sequential, args.steps)
    # autotune each (dim, kind) class on its largest instance, then batch
    classes = {}
    for inst in insts:
        key = (inst.dim, inst.domain.outer, len(inst.domain.holes) > 0)
        if key not in classes or inst.M_D * inst.N > classes[key].M_D * classes[key].N:
            classes[key] = inst
    tunings = {str(k): wos.wos_autotune(ctx, v) for k, v in classes.items()}
    def batched():
        c, u, _ = wos.wos_build_operators_batched(ctx, insts, seed=insts[0].seed, points=pts,
                                                  stats=False)
        return c
    for _ in range(max(1, args.warmup)):
        batched()
    bat_out, bat_ms = timed(batched, args.steps)
    same = all(torch.equal(a, b) for a, b in zip(seq_out, bat_out))

    # small requests: 256 instances of 64..256 points x 1e3..1e4 walks
    small = W.mixed_batch(256, seed=17, m_lo=64, m_hi=256, n_lo=1e3, n_hi=1e4)
    spts = [torch.as_tensor(i.points, dtype=torch.float64, device=dev) for i in small]
    swalks = sum(i.M_D * i.N for i in small)
    def small_seq():
        return [wos.wos_build_operator(ctx, i.domain, i.K, p, i.partition, i.N, i.eps, i.seed,
                                       opts=wos.make_opts(stream_id=i.stream), stats=False)[0]
                for i, p in zip(small, spts)]
    def small_bat():
        return wos.wos_build_operators_batched(ctx, small, seed=small[0].seed, points=spts,
                                               stats=False)[0]
    small_seq()
    small_bat()
    s_seq, s_seq_ms = timed(small_seq, args.steps)
    s_bat, s_bat_ms = timed(small_bat, args.steps)
    s_same = all(torch.equal(a, b) for a, b in zip(s_seq, s_bat))
    if rank != 0:
        return
    t_seq = float(np.median(seq_ms)) / 1e3
    t_bat = float(np.median(bat_ms)) / 1e3
    ts_seq = float(np.median(s_seq_ms)) / 1e3
    ts_bat = float(np.median(s_bat_ms)) / 1e3
    print(json.dumps({
        "metric": METRIC, "value": walks / t_bat, "unit": "walks/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_bat,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"mixed batch of 64 instances (disc, annulus, square, L-shape, "
                               f"ball, box), {walks:.3g} walks, operator builds only",
                   "walks_per_step": walks},
        "sequential_walks_per_s": walks / t_seq, "batched_over_sequential": t_seq / t_bat,
        "batched_equals_sequential": bool(same), "tunings": tunings,
        "small_requests": {"instances": len(small), "walks": swalks,
                           "batched_walks_per_s": swalks / ts_bat,
                           "sequential_walks_per_s": swalks / ts_seq,
                           "batched_over_sequential": ts_seq / ts_bat,
                           "requests_per_s_batched": len(small) / ts_bat,
                           "requests_per_s_sequential": len(small) / ts_seq,
                           "batched_equals_sequential": bool(s_same)},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="square-annulus")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-scale", type=float, default=1.0,
                    help="walks-per-point scale of the batch workload")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as D
        D.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        dist = D
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "batch":
        run_batch(args, rank, world, dist)
    else:
        run_gpu(args, rank, world, dist)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
