#!/usr/bin/env python
"""Benchmark of the walk-on-ellipsoids operator build on GB300.

One step = the whole hot path on the 3-D workload of anisotropic Cauchy
problems (the default, ``--workload config3``): the unit ball and the cube
[-1, 1]^3, each with K = diag(1, 2, 4) and with a random SPD K (eigenvalues
log-uniform in [0.5, 4]); 1536 boundary patches (Gamma_1 = 768), 1024
interior points uniform in the inner half, N = 1e5 walks per point, eps =
1e-4, FP32 walks: the four Monte Carlo operator builds (MC-REM), the FP64
one-sided Jacobi SVDs of the four 1024 x 768 Gamma_1 blocks and the TSVD
reconstructions from measurements with 1 % Gaussian noise.
``--workload square-annulus`` is the 2-D workload (unit square and annulus,
K = [[1, .5], [.5, 2]], 256 elements and points, N = 1e5, eps = 1e-5).

The timed steps pipeline: step k + 1's walk launches overlap step k's SVD
and reconstructions, which run on high-priority SVD streams taken in turn;
``step_latency_ms`` is one step alone.  Prints one JSON line (metric, value =
walks/s over all GPUs, roofline of the dominant kernel by SM-time and of the
other one, measured pipe rates, CPU baseline = the FP64 oracle on the host
cores, e2e = the same steps through the public API with host buffers; on the
3-D workload also the served requests/s and p50 / p99 latency of a bounded
prefix of the seeded request stream against one-at-a-time plain launches,
and the batched / sequential ratio of the 64-instance mixed batch).
``--impl reference`` times the CPU oracle on a bounded sample of the same
workload instead.
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
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = ("WoS walks/s and steps/s on 1 GB300 (% FP32/SFU roofline); "
          "served p50/p99 latency")
# ALU issue peak of one GB300: 152 SMs x 4 schedulers x 32 lanes per clock
# at the 2070 MHz maximum SM clock (lane-operations per second).
ALU_PEAK_GOPS = 152 * 4 * 32 * 2.070
# Algorithmic lane-operations of one step of the chain (FP32, 2-D, full S),
# counted on the cheapest formulation known (absolute values are operand
# modifiers): Philox4x32-10 share 80/5 = 16 (a block of 80 operations serves
# five steps, one 23-bit window each), window 2 (shift, mask), angle and
# sine/cosine 4 (one FMA, the scaling to revolutions, two SFU operations),
# move 6 (S U and the update), eps test and step-length select 2, step
# counter 1, plus the distance: square 2 (max of |x_a|, subtraction from h),
# annulus 5 (two products, square root, |rho - mid| and its subtraction from
# the half-width).
OPS_PER_STEP = {"box": 33, "annulus": 36, "ball": 72, "cube": 70}
# FP32 3-D step, the same rules: Philox share 80/2 = 40 (a block of four
# words serves two steps of two 23-bit uniforms), uniforms 4 (shift and or
# per word), z = 3 - 2 f1 and the angle 2 pi f2 - 3 pi 2 (FMAs), sine/cosine
# 3 (scaling to revolutions, two SFU operations), 1 - z^2 and its square
# root 2, move 13 (d s, the three products of d U, the nine FMAs of S (d U)
# added to X), eps test and select 2, step counter 1, plus the distance:
# ball 5 (three products / FMAs for |x|^2, square root, R - rho), cube 3
# (two maxima of |x_a|, subtraction from h).
# FP64 peak of one GB300: 152 SMs x 2 FP64 FMA per clock (ncu:
# sm__sass_thread_inst_executed_op_dfma_pred_on.sum.peak_sustained = 304 per
# chip) x 2 flop x 2070 MHz, in GFLOP/s.
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.070
PROFILES = ROOT / "profiles"
CSRC = ROOT / "paper_2409_03686_gb300" / "csrc"


def _source_hash(files) -> str:
    h = hashlib.sha256()
    for f in files:
        h.update((CSRC / f).read_bytes())
    return h.hexdigest()[:16]


def _traffic_from_profile(note: str, hash_key: str, files, value_key: str):
    """DRAM bytes from a committed ncu summary (profiles/<note>), if it was
    taken on the current source of the kernel (its hash_key line equals the
    SHA-256 prefix of `files`); else None."""
    path = PROFILES / note
    if not path.exists():
        return None
    vals = {}
    for line in path.read_text().splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get(hash_key) != _source_hash(files):
        return None
    try:
        return float(vals[value_key])
    except (KeyError, ValueError):
        return None


def walk_traffic(dim: int):
    """DRAM bytes per walk-kernel launch (the 2-D or 3-D capture)."""
    note = "walk_kernel_ball_cube.md" if dim == 3 else "walk_kernel_square_annulus.md"
    return _traffic_from_profile(note, "kernel_source_hash",
                                 ("walk_kernel.cuh", "wos_device.cuh"), "dram_bytes_per_launch")


def svd_traffic():
    """DRAM bytes of the four 1024 x 768 factorisations of a 3-D step."""
    return _traffic_from_profile("jacobi_svd_fp64.md", "svd_source_hash", ("wos_svd.cu",),
                                 "dram_bytes_per_step")


def workload(name: str):
    from paper_2409_03686_gb300 import workloads as W
    if name == "config3":
        return W.config3_instances()
    if name == "config3-small":  # for ncu captures: same kernels, fewer walks
        return W.config3_instances(N=4_000, n_points=256)
    if name == "square-annulus":
        return [W.square_config(), W.annulus_config()]
    if name == "small":  # for ncu captures: same kernels, smaller sizes
        return [W.square_config(N=20_000, grid=8), W.annulus_config(N=20_000, grid=8)]
    raise SystemExit(f"unknown workload {name}")


def kind_of(inst) -> str:
    """Operation-count class of an instance's walk kernel."""
    if inst.dim == 3:
        return "cube" if inst.domain.outer == "box" else "ball"
    return "box" if inst.domain.outer == "box" else "annulus"


def describe(name: str) -> dict:
    if name == "config3":
        return {"workload": ("3-D anisotropic Cauchy operators: unit ball and cube "
                             "[-1,1]^3, each with K=diag(1,2,4) and a random SPD K "
                             "(eigenvalues log-uniform in [0.5,4]); 1536 boundary patches "
                             "(32x48 equal-area on the sphere, 6x16x16 on the cube; "
                             "Gamma_1 = 768), 1024 points uniform in the inner half, "
                             "N=1e5 walks/point, eps=1e-4, FP32 walks, uint32 counts; "
                             "FP64 Jacobi SVD of each 1024x768 Gamma_1 block; TSVD of 1% "
                             "noisy data"),
                "walks_per_step": 4 * 1024 * 100_000,
                "l2": ("flushed between consecutive steps' walks (256 MiB write on the "
                       "walk stream, inside the timed region; also in the e2e and "
                       "latency steps)"),
                "parallelism": "replicas (one full workload per GPU)"}
    if name == "square-annulus":
        return {"workload": ("2-D anisotropic Cauchy operator: unit square [-1/2,1/2]^2 "
                             "and annulus r in [0.5,1], K=[[1,0.5],[0.5,2]], 256 boundary "
                             "elements each (Gamma_1 = 128), 256 jittered interior points, "
                             "N=1e5 walks/point, eps=1e-5, FP32 walks; FP64 Jacobi SVD of "
                             "the 256x128 Gamma_1 block; TSVD of 1% noisy data"),
                "walks_per_step": 2 * 256 * 100_000,
                "l2": ("flushed between consecutive steps' walks (256 MiB write on the "
                       "walk stream, inside the timed region; also in the e2e and "
                       "latency steps)"),
                "parallelism": "replicas (one full workload per GPU)"}
    return {"workload": name}


def max_over_ranks(value: float, dist, device) -> float:
    """The largest of every rank's value (a job's time is its slowest
    rank's); the value itself without a process group."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


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
        self.temp = False

    def start(self):
        # samples go to $WOS_CLOCKS_CSV when set (to keep them), else to a
        # temporary file
        try:
            path = os.environ.get("WOS_CLOCKS_CSV")
            if path:
                self.path = Path(path)
            else:
                fd, name = tempfile.mkstemp(prefix=f"clocks_gpu{self.gpu}_", suffix=".csv")
                os.close(fd)
                self.path = Path(name)
                self.temp = True
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            if self.temp and self.path is not None:
                self.path.unlink(missing_ok=True)
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
        if self.temp:
            self.path.unlink(missing_ok=True)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# CPU oracle (the baseline and the reference arm)
# ----------------------------------------------------------------------------
def oracle_sample(insts, n_points: int, n_walks: int, passes: int = 1):
    """Times the oracle's MC-REM on the first n_points points with n_walks
    walks each, for every instance, `passes` times with independent walks
    (another Philox stream per pass); returns (walks, steps, seconds)."""
    from oracle import oracle as O
    O.build()
    walks = steps = 0
    t0 = time.perf_counter()
    for ps in range(passes):
        for inst in insts:
            sub = inst.replace(points=inst.points[:n_points], N=n_walks,
                               stream=inst.stream + 1000 * ps)
            C, U, s = O.build_counts(sub)
            walks += sub.M_D * sub.N
            steps += s
    return walks, steps, time.perf_counter() - t0


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    insts = workload(args.workload)
    n_pts, n_walks = (8 if insts[0].dim == 3 else 32), 100_000
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
        "dtype": "f64", "data": "synthetic",
        "config": dict(describe(args.workload),
                       l2="not applicable: the CPU oracle on the host cores"),
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
SVD_PATHS = {"auto": 0, "grid": 1, "fp64-sweeps": 3}


def qr_flop(m: int, n: int) -> int:
    """FP64 flop of the Householder QR of an m x n matrix (m >= n): 2mn^2 -
    2n^3/3 (the column-pivoting norm updates are O(mn))."""
    return 2 * m * n * n - (2 * n ** 3) // 3


def fp32_preconditioned(n: int, svd_path: str) -> bool:
    """Whether the library runs FP32 sweeps before the FP64 ones for a worked
    matrix of n columns: above 256 (the sizes the cluster kernel cannot take)
    and up to 768 columns (a lane's registers), unless FP64 sweeps alone are
    asked for."""
    return 256 < n <= 768 and svd_path != "fp64-sweeps"


def ns_flop(n: int) -> int:
    """FP64 flop between the FP32 and the FP64 sweeps: two symmetric products
    Q^T Q (n^3 each, one triangle) and X Q (2 n^3); the two correction
    products run in FP32."""
    return 4 * n ** 3


def svd_fp64_flop(m: int, n: int, sweeps: int, svd_path: str) -> int:
    """FP64 flop of one factorisation of an m x n worked matrix: the QR
    (n >= 32), the Newton-Schulz products of the FP32-preconditioned path,
    and the FP64 sweeps (sweeps = the FP64 sweeps the library reports)."""
    fl = jacobi_flop(m, n, sweeps) + (qr_flop(m, n) if n >= 32 else 0)
    return fl + (ns_flop(n) if fp32_preconditioned(n, svd_path) else 0)


def jacobi_flop(m: int, n: int, sweeps: int) -> int:
    """FP64 flop of the Jacobi sweeps of one SVD of an m x n worked matrix
    (m >= n) as the library runs it (on X = R^T, n x n, when n >= 32): every
    pair visit counted as rotated.  Up to 256 columns the sweeps accumulate V
    (three dot products 6l, column updates 6l + 6n); above, they do not,
    carry the norms and scale the columns (one dot product 2l, column
    updates 4l: one FMA per row and column)."""
    rows = n if n >= 32 else m
    if n > 256:
        return sweeps * (n * (n - 1) // 2) * (6 * rows)
    return sweeps * (n * (n - 1) // 2) * (12 * rows + 6 * n)


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
    wos.wos_set_svd_path(ctx, SVD_PATHS[args.svd_path])
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

    # the SVD stream runs at high priority: when a step's walk launch drains,
    # the block scheduler places the SVD's clusters before the next step's
    # walk blocks, which fill the rest of the GPU (steps pipeline)
    # several SVD streams, taken in turn by the steps, so that consecutive
    # steps' SVDs overlap each other too: four for the 2-D configuration
    # (each SVD a latency-bound cluster launch on a few SMs), two for the
    # 3-D one (its SVDs take longer than its walks; more streams only pile
    # them up: 3.36 / 3.37e9 walks/s with four against 3.50 / 3.54e9)
    if args.svd_streams <= 0:
        args.svd_streams = 2 if args.workload.startswith("config3") else 4
    streams = [torch.cuda.Stream(device=dev, priority=-1) for _ in range(args.svd_streams)]
    build_stream = torch.cuda.Stream(device=dev)
    # the project's autotuner picks the launch configuration of each
    # instance's class (precision, dimension, kernel kind) on a bounded sample
    # of its walks, before anything is timed; later builds use it
    tunings = ({inst_p["inst"].name: wos.wos_autotune(ctx, inst_p["inst"])
                for inst_p in prep} if not args.no_autotune else {})
    # --walk-blocks-per-sm caps the walk launches' resident blocks per SM
    # (the tuned configuration otherwise), leaving room beside them for the
    # previous step's SVD kernels
    walk_launch = {}
    if args.walk_blocks_per_sm > 0:
        for p in prep:
            t = tunings.get(p["inst"].name, {})
            walk_launch[p["inst"].name] = dict(
                block_size=int(t.get("block_size", 256)),
                blocks_per_sm=(min(int(t["blocks_per_sm"]), args.walk_blocks_per_sm)
                               if t.get("blocks_per_sm", 0) > 0 else args.walk_blocks_per_sm),
                tiles_per_warp=int(t.get("tiles_per_warp", 0)),
                hist_slots=int(t.get("hist_slots", 0)),
                refill_min=int(t.get("refill_min", 0)))
    # measured pipe throughputs of this GPU (microbenchmark kernels, a few ms)
    pipes = wos.wos_measure_pipes(ctx)
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
        p["sweeps"] = sw
        M_1 = int(inst.partition.gamma1.sum())
        p["svd_mn"] = (max(inst.M_D, M_1), min(inst.M_D, M_1))
        p["steps"] = st["steps"]
        p["kind"] = kind_of(inst)
        steps_per_inst.append(st["steps"])
    def step(timing=None, host_io=False, start_ev=None, svd_timing=None, jac_timing=None,
             join=True, index=0):
        """One step: the operator builds back to back on the build stream (a
        persistent walk launch fills the GPU), then both instances' SVDs in
        one batched call and their reconstructions on the SVD stream.  With
        join, the current stream waits for the step; without, the step's
        completion events are returned and the next step's walks (on the
        build stream) overlap this step's SVD."""
        main = torch.cuda.current_stream()
        bs = build_stream
        if start_ev is not None:
            bs.wait_event(start_ev)
        else:
            bs.wait_stream(main)
        built = []
        with torch.cuda.stream(bs):
            # L2 flushed between consecutive steps' walks: the build stream
            # runs the walks in order, so the write sits after the previous
            # step's walk launches and before this step's
            flush.zero_()
            for q, p in enumerate(prep):
                inst = p["inst"]
                if host_io:
                    pts = p["host"]["points"].to(dev, non_blocking=True)
                    uD = p["host"]["uD"].to(dev, non_blocking=True)
                    u0 = p["host"]["u0"].to(dev, non_blocking=True)
                else:
                    pts, uD, u0 = p["points"], p["uD"], p["u0"]
                opts = wos.make_opts(precision=0, stream_id=inst.stream,
                                     kernel_events=timing[q] if timing else None,
                                     **walk_launch.get(inst.name, {}))
                c, _, _ = wos.wos_build_operator(ctx, inst.domain, inst.K, pts,
                                                 inst.partition, inst.N, inst.eps, inst.seed,
                                                 opts=opts, stats=False, stream=bs)
                built.append((c, uD, u0))
        ev_built = torch.cuda.Event()
        ev_built.record(bs)
        # both instances' SVDs in one batched call, then their TSVDs
        s = streams[index % len(streams)]
        s.wait_event(ev_built)
        for c, uD, u0 in built:
            for t in (c, uD, u0):
                t.record_stream(s)
        outs, done = [], []
        with torch.cuda.stream(s):
            if svd_timing is not None:
                svd_timing[0][0].record(s)
            svds = wos.wos_op_svd_batched(
                ctx, [(built[q][0], p["inst"].N, p["inst"].partition.gamma1, p["sigma"])
                      for q, p in enumerate(prep)], sync=False, stream=s,
                jacobi_events=jac_timing)
            if svd_timing is not None:
                svd_timing[0][1].record(s)
            for q, p in enumerate(prep):
                inst = p["inst"]
                c, uD, u0 = built[q]
                U, S, V, _ = svds[q]
                u1, _ = wos.wos_reconstruct(ctx, U, S, V, c, inst.N, inst.partition.gamma1,
                                            p["sigma"], uD, p["r"], u0=u0, stream=s)
                if host_io:
                    outs.append((c.to("cpu", non_blocking=True),
                                 u1.to("cpu", non_blocking=True)))
                else:
                    outs.append((c, u1))
            e = torch.cuda.Event()
            e.record(s)
            done.append(e)
        if not join:
            return outs, done
        for e in done:
            main.wait_event(e)
        return outs

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # latency of one step on its own (nothing overlapped)
    # (the walk and factorisation launches are timed in these steps too: the
    # kernels' own rates, with nothing overlapping them)
    def new_pairs(n):
        out = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(n)]
        for pair in out:  # create the events; the library re-records them
            for e in pair:
                e.record(stream)
        return out

    lat_ms, lat_starts, lat_kev, lat_jev = [], [], [], []
    for _ in range(3):
        l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        kv, jv = new_pairs(len(prep)), new_pairs(1)[0]
        l0.record(stream)
        step(start_ev=l0, timing=kv, jac_timing=jv)
        l1.record(stream)
        torch.cuda.synchronize()
        lat_ms.append(l0.elapsed_time(l1))
        lat_starts.append(l0)
        lat_kev.append(kv)
        lat_jev.append(jv)
    step_latency_ms = float(np.median(lat_ms))

    # ---- device-timed steps --------------------------------------------------
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in prep] for _ in range(args.steps)]
    for row in kev:  # create the events; the library re-records them around the kernel
        for pair in row:
            for e in pair:
                e.record(stream)
    sev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))]
           for _ in range(args.steps)]
    jev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    for pair in jev:  # create the events; the library re-records them
        for e in pair:
            e.record(stream)
    clocks = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = ctx.kernel_launches()
    clocks.start()
    t_wall = time.perf_counter()
    t_first = torch.cuda.Event(enable_timing=True)
    t_last = torch.cuda.Event(enable_timing=True)
    pending = []
    t_first.record(stream)
    for it in range(args.steps):
        starts[it].record(stream)
        _, done = step(timing=kev[it], start_ev=starts[it], svd_timing=sev[it],
                       jac_timing=jev[it], join=False, index=it)
        pending.extend(done)
    for e in pending:
        stream.wait_event(e)
    t_last.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    launches = ctx.kernel_launches() - launches0
    total_ms = t_first.elapsed_time(t_last)
    total_ms = max_over_ranks(total_ms, dist, dev)
    walks_per_step = sum(p["inst"].M_D * p["inst"].N for p in prep)
    steps_per_step = sum(steps_per_inst)
    value = world * walks_per_step * args.steps / (total_ms / 1e3)
    steps_per_s = world * steps_per_step * args.steps / (total_ms / 1e3)

    # roofline of the walk kernel: algorithmic lane-operations / kernel time.
    # The instances overlap on the GPU, so the kernel time of a step is the
    # union of its walk-kernel intervals (CUDA events on the launching
    # streams, placed relative to the step's start event).
    ops = sum(OPS_PER_STEP[p["kind"]] * p["steps"] for p in prep)

    def union_ms(start, pairs):
        iv = sorted((start.elapsed_time(a), start.elapsed_time(b)) for (a, b) in pairs)
        tot, cur0, cur1 = 0.0, None, None
        for a, b in iv:
            if cur1 is None or a > cur1:
                if cur1 is not None:
                    tot += cur1 - cur0
                cur0, cur1 = a, b
            else:
                cur1 = max(cur1, b)
        return tot + cur1 - cur0

    # pipelined steps (the walks share the SMs with the previous step's SVD)
    kernel_ms_step = float(np.mean([union_ms(starts[it], kev[it]) for it in range(args.steps)]))
    achieved_ov = ops / (kernel_ms_step / 1e3) / 1e9
    # the same launches in the steps run alone: the kernel's own rate
    walk_ms_alone = float(np.median([union_ms(l0, kv) for l0, kv in zip(lat_starts, lat_kev)]))
    achieved = ops / (walk_ms_alone / 1e3) / 1e9
    traffic = walk_traffic(prep[0]["inst"].dim)
    walk_roof = {"kernel": "walk_kernel", "bound": "alu", "achieved": achieved,
                 "peak": ALU_PEAK_GOPS, "unit": "Gop/s", "frac": achieved / ALU_PEAK_GOPS,
                 "traffic": traffic,
                 "timing": "the walk launches of the steps run alone (CUDA events on the "
                           "build stream, union per step, median of three steps)",
                 "ms_per_step": walk_ms_alone,
                 "overlapped": {"ms_per_step": kernel_ms_step, "achieved": achieved_ov,
                                "frac": achieved_ov / ALU_PEAK_GOPS,
                                "note": "the timed pipelined steps: the walks share the "
                                        "SMs with the previous step's factorisation"},
                 "measured_issue_peak": pipes["issue"] / 1e9,
                 "frac_of_measured_issue": achieved / (pipes["issue"] / 1e9),
                 "peak_source": "152 SMs x 4 schedulers x 32 lanes x 2070 MHz "
                                "(recipe unit counts and max clock)",
                 "unit_of_work": "one step of the chain: 33 (2-D square) / 36 (2-D "
                                 "annulus) / 72 (3-D ball) / 70 (3-D cube) algorithmic "
                                 "lane-operations",
                 "ops_per_step": {p["inst"].name: OPS_PER_STEP[p["kind"]] for p in prep}}
    # the Jacobi launch of a step's batched SVD (both instances): FP64
    # roofline with every pair visit counted as rotated, an upper bound on the
    # work; the whole SVD call (form_B, QR, Jacobi, left vectors, finalize) is
    # reported beside it
    svd_ms_sum = float(np.mean([sum(a.elapsed_time(b) for (a, b) in row) for row in sev]))
    jac_ms_ov = float(np.mean([a.elapsed_time(b) for (a, b) in jev]))
    jac_ms = float(np.median([a.elapsed_time(b) for (a, b) in lat_jev]))
    walk_ms_sum = float(np.mean([sum(a.elapsed_time(b) for (a, b) in row) for row in kev]))
    flop = sum(svd_fp64_flop(p["svd_mn"][0], p["svd_mn"][1], p["sweeps"], args.svd_path)
               for p in prep)
    mixed = all(fp32_preconditioned(p["svd_mn"][1], args.svd_path) for p in prep)
    svd_achieved = flop / (jac_ms / 1e3) / 1e9
    svd_achieved_ov = flop / (jac_ms_ov / 1e3) / 1e9
    sweeps64 = ("jacobi_group_kernel" if not mixed and
                sum(p["svd_mn"][1] for p in prep) > 2 * 3 * 152 else "jacobi_lean_kernel")
    svd_roof = {"kernel": ("svd_cluster_kernel" if args.svd_path == "auto" and
                           all(p["svd_mn"][1] <= 256 for p in prep)
                           else ("qrs_kernel + pc32_sweeps_kernel + pc32_replay_kernel + "
                                 "dgemm_kernel + " + sweeps64 if mixed
                                 else "qrcp_kernel + " + sweeps64)
                           if all(p["svd_mn"][1] > 256 for p in prep)
                           else "qrcp_kernel + jacobi_kernel"),
                "bound": "alu", "pipe": "fp64", "achieved": svd_achieved,
                "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                "frac": svd_achieved / FP64_PEAK_GFLOPS,
                "traffic": svd_traffic() if args.workload == "config3" else None,
                "peak_source": "152 SMs x 2 FP64 FMA/clk (ncu dfma peak_sustained 304 "
                               "per chip) x 2 flop x 2070 MHz",
                "unit_of_work": "one factorisation's FP64 flop: the Householder QR (2mn^2 - "
                                "2n^3/3, n >= 32; pivoted, or in decreasing-norm order "
                                "before FP32 sweeps), the Newton-Schulz and X Q products "
                                "after FP32 sweeps (4 n^3; 256 < n <= 768), and every pair "
                                "visit of every FP64 sweep (12 l + 6n flop with V "
                                "accumulated, n <= 256; 6 l without, n > 256; l = rows of "
                                "the matrix Jacobi works on: n after the QR, m without; every "
                                "visit counted as rotated).  The FP32 sweeps run on the FP32 "
                                "pipe and are not counted",
                "sweeps": [p["sweeps"] for p in prep],
                "problems_per_launch": len(prep),
                "timing": "the factorisation launches (QR and sweeps) of the steps run "
                          "alone (CUDA events on the SVD stream, median of three steps)",
                "ms_per_step": jac_ms,
                "overlapped": {"ms_per_step": jac_ms_ov, "achieved": svd_achieved_ov,
                               "frac": svd_achieved_ov / FP64_PEAK_GFLOPS,
                               "svd_call_ms": svd_ms_sum,
                               "note": "the timed pipelined steps: the factorisation shares "
                                       "the SMs with the next step's walks"}}
    # the dominant kernel is the one with the larger share of the GPU's
    # SM-time per step (device time x SMs it holds): the walk launches hold
    # every SM, a cluster factorisation 16 SMs per problem (the grid-wide
    # kernels up to every SM); the steps pipeline, so device times overlap
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    cluster = svd_roof["kernel"] == "svd_cluster_kernel"
    svd_sms = min(sms, 16 * len(prep)) if cluster else sms
    walk_roof["sm_ms_per_step"] = walk_ms_alone * sms
    svd_roof["sm_ms_per_step"] = jac_ms * svd_sms
    if jac_ms * svd_sms > walk_ms_alone * sms:
        roof, roof2 = svd_roof, walk_roof
    else:
        roof, roof2 = walk_roof, svd_roof

    # ---- e2e: public API with host buffers and copies in the timed region ---
    e2e_s = torch.cuda.Event(enable_timing=True)
    e2e_e = torch.cuda.Event(enable_timing=True)
    h2d = sum(p["host"][k].numel() * 8 for p in prep for k in ("points", "uD", "u0"))
    d2h = 0
    torch.cuda.synchronize()
    e2e_s.record(stream)
    pending = []
    for it in range(args.steps):
        outs, done = step(host_io=True, join=False, index=it)
        pending.extend(done)
        d2h = sum(o[0].numel() * 4 + o[1].numel() * 8 for o in outs)
    for e in pending:
        stream.wait_event(e)
    e2e_e.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e2e_s.elapsed_time(e2e_e)
    e2e_ms = max_over_ranks(e2e_ms, dist, dev)
    e2e_value = world * walks_per_step * args.steps / (e2e_ms / 1e3)

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "walks/s", "steps_per_s": steps_per_s,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "schedule": "pipelined: step k+1's walk launches (build stream) overlap step k's "
                    "SVD and reconstructions (%d high-priority SVD streams taken in turn); "
                    "L2 flushed before every step's walks" % args.svd_streams,
        "step_latency_ms": step_latency_ms,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": describe(args.workload),
        "steps_per_walk": steps_per_step / walks_per_step,
        "walk_kernel_ms_per_step": kernel_ms_step,
        "truncation_r": [p["r"] for p in prep],
        "roofline": roof,
        "roofline_secondary": roof2,
        "device_ms_per_step": {"alone": {"walk_kernels": walk_ms_alone,
                                         "svd_factorisation": jac_ms},
                               "pipelined": {"walk_kernels": walk_ms_sum,
                                             "svd_factorisation": jac_ms_ov,
                                             "svd_call": svd_ms_sum}},
        "gpu_launches": int(launches),
        "autotuned": {k: {f: v[f] for f in ("block_size", "blocks_per_sm", "tiles_per_warp",
                                             "hist_slots", "refill_min", "best_ms",
                                             "default_ms")} for k, v in tunings.items()},
        "wall_s_timed": wall,
        "e2e": {"value": e2e_value, "unit": "walks/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "clocks": clk,
        "pipe_peaks": {"unit": "lane-ops/s (measured; per SM per clock at 2070 MHz beside)",
                       **{k: v for k, v in pipes.items()},
                       "per_sm_clk": {k: v / (sms * 2.07e9) for k, v in pipes.items()}},
    }
    if args.workload == "config3" and not args.no_extras:
        # the metric's served latency (a bounded prefix of the config-5
        # stream) and the config-4 batched / sequential ratio, each in a
        # context of its own, after the timed steps
        sv = measure_serve(args, local)
        line["served"] = {"workload": sv["workload"], "requests": sv["requests"],
                          **sv["served"], "one_at_a_time": sv["one_at_a_time"],
                          "served_over_one_at_a_time": sv["served_over_one_at_a_time"],
                          "served_equals_alone": sv["served_equals_alone"]}
        bt = measure_batch(args, local, reps=3)
        line["batched"] = {"workload": "config 4: 64 mixed 2-D / 3-D instances "
                                       f"({bt['walks']:.3g} walks), operator builds only, "
                                       "median of 3 calls each",
                           "batched_walks_per_s": bt["batched_walks_per_s"],
                           "sequential_walks_per_s": bt["sequential_walks_per_s"],
                           "batched_over_sequential": bt["batched_over_sequential"],
                           "batched_equals_sequential": bt["batched_equals_sequential"],
                           "small_requests": bt["small_requests"]}
    if not args.no_cpu_baseline and world == 1:
        insts = [p["inst"] for p in prep]
        if insts[0].dim == 3:
            n_pts, n_walks, passes = 96, insts[0].N, 1
            what = (f"the first {n_pts} of {insts[0].M_D} points x {n_walks} walks of each "
                    f"of the {len(insts)} instances")
        else:
            n_pts, n_walks, passes = insts[0].M_D, insts[0].N, 2
            what = (f"the whole workload (all {n_pts} points x {n_walks} walks of both "
                    f"instances) twice with independent walks")
        w, s, dt = oracle_sample(insts, n_pts, n_walks, passes=passes)
        line["cpu_baseline"] = {
            "value": w / dt, "unit": "walks/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{what}: {w} walks, {dt:.1f} s, FP64 C oracle on "
                      f"{os.cpu_count()} threads"}
    print(json.dumps(line))


def measure_batch(args, local: int, reps: int) -> dict:
    """Config 4: the 64-instance mixed batch (disc, annulus, square, L-shape,
    ball, box; log-uniform sizes and walks per point) in one autotuned
    persistent launch per dimension, against one plain launch per instance
    (default launch settings) on the same GPU, `reps` timed calls each (a
    context of its own, so the plain launches use no tuning).  Operator
    builds only."""
    import torch
    from paper_2409_03686_gb300 import build as B
    from paper_2409_03686_gb300 import workloads as W
    from paper_2409_03686_gb300 import wos
    dev = torch.device("cuda", local)
    B.build()
    ctx = wos.Context(local)
    wos.wos_set_svd_path(ctx, SVD_PATHS[args.svd_path])
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
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    def timed(fn, reps):
        ms = []
        for _ in range(reps):
            flush.zero_()  # L2 flushed before every timed call
            torch.cuda.synchronize()
            ev0.record()
            r = fn()
            ev1.record()
            torch.cuda.synchronize()
            ms.append(ev0.elapsed_time(ev1))
        return r, ms
    sequential()
    seq_out, seq_ms = timed(sequential, reps)
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
    bat_out, bat_ms = timed(batched, reps)
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
    s_seq, s_seq_ms = timed(small_seq, reps)
    s_bat, s_bat_ms = timed(small_bat, reps)
    s_same = all(torch.equal(a, b) for a, b in zip(s_seq, s_bat))
    t_seq = float(np.median(seq_ms)) / 1e3
    t_bat = float(np.median(bat_ms)) / 1e3
    ts_seq = float(np.median(s_seq_ms)) / 1e3
    ts_bat = float(np.median(s_bat_ms)) / 1e3
    ctx.close()
    return {
        "walks": walks, "t_bat": t_bat, "t_seq": t_seq,
        "batched_walks_per_s": walks / t_bat,
        "sequential_walks_per_s": walks / t_seq, "batched_over_sequential": t_seq / t_bat,
        "batched_equals_sequential": bool(same), "tunings": tunings,
        "small_requests": {"instances": len(small), "walks": swalks,
                           "batched_walks_per_s": swalks / ts_bat,
                           "sequential_walks_per_s": swalks / ts_seq,
                           "batched_over_sequential": ts_seq / ts_bat,
                           "requests_per_s_batched": len(small) / ts_bat,
                           "requests_per_s_sequential": len(small) / ts_seq,
                           "batched_equals_sequential": bool(s_same)},
    }


def run_batch(args, rank: int, world: int, dist):
    """Config 4 alone (see measure_batch), ``--steps`` timed calls each."""
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    r = measure_batch(args, local, args.steps)
    if rank != 0:
        return
    walks, t_bat = r.pop("walks"), r.pop("t_bat")
    r.pop("t_seq")
    print(json.dumps({
        "metric": METRIC, "value": walks / t_bat, "unit": "walks/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_bat,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"mixed batch of 64 instances (disc, annulus, square, L-shape, "
                               f"ball, box), {walks:.3g} walks, operator builds only",
                   "walks_per_step": walks,
                   "l2": "flushed before every timed call (256 MiB write, outside it)"},
        **r,
    }))


def measure_serve(args, local: int) -> dict:
    """Serving: a prefix of the seeded 10,000-request Poisson stream of 3-D
    ball / cube requests (operator build + FP64 SVD + truncation + TSVD
    reconstruction each, host inputs and outputs) through the request queue,
    against one-at-a-time plain launches of the same requests on the same
    GPU.  Throughput with every request submitted at once; latency with
    Poisson arrivals at 70 % of the served throughput (the one-at-a-time
    latency at the same arrivals follows from its measured service times,
    first come first served).  A context of its own."""
    import threading

    import torch
    from paper_2409_03686_gb300 import build as B
    from paper_2409_03686_gb300 import workloads as W
    from paper_2409_03686_gb300 import wos
    dev = torch.device("cuda", local)
    B.build()
    ctx = wos.Context(local)
    wos.wos_set_svd_path(ctx, SVD_PATHS[args.svd_path])
    reqs = W.serve_stream(first=args.serve_requests)
    seed = reqs[0].inst.seed
    meas = [W.measurements(r.inst, noise=r.noise, seed=r.index) for r in reqs]
    sig = {}

    def alone(r, m):
        """One request with plain launches: inputs to the device, build, SVD,
        singular values to the host, truncation, TSVD, result to the host."""
        inst = r.inst
        key = (inst.domain.outer, inst.M_tot)
        if key not in sig:
            sig[key] = wos.wos_element_measures(inst.domain, inst.partition)
        pts = torch.as_tensor(inst.points, dtype=torch.float64).pin_memory().to(
            dev, non_blocking=True)
        sigma = torch.as_tensor(sig[key]).pin_memory().to(dev, non_blocking=True)
        uD = torch.as_tensor(m.uD).pin_memory().to(dev, non_blocking=True)
        u0 = torch.as_tensor(m.u0).pin_memory().to(dev, non_blocking=True)
        c, _, _ = wos.wos_build_operator(ctx, inst.domain, inst.K, pts, inst.partition,
                                         inst.N, inst.eps, inst.seed,
                                         opts=wos.make_opts(stream_id=inst.stream),
                                         stats=False)
        g1 = inst.partition.gamma1
        U, S, V, _ = wos.wos_op_svd(ctx, c, inst.N, g1, sigma, sync=False)
        r_use = pick_rank(S.cpu().numpy())
        u1, _ = wos.wos_reconstruct(ctx, U, S, V, c, inst.N, g1, sigma, uD, r_use, u0=u0,
                                    want_uD_hat=False)
        return u1.cpu().numpy(), r_use

    alone(reqs[0], meas[0])  # warm-up (module load, pools)
    seq_t, seq_u1 = [], []
    for r, m in zip(reqs, meas):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        u1, _ = alone(r, m)
        seq_t.append(time.perf_counter() - t0)
        seq_u1.append(u1)

    def make_queue():
        return wos.wos_queue_create(ctx, seed=seed, precision=0,
                                    side_streams=args.serve_side,
                                    slice_walks=args.serve_slice)

    # warm-up of the queue path
    q = make_queue()
    for r, m in zip(reqs[:4], meas[:4]):
        wos.wos_wait(q, wos.wos_submit(q, r.inst, m.uD, m.u0))
    wos.wos_queue_destroy(q)

    # throughput: everything submitted at once
    q = make_queue()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tickets = [wos.wos_submit(q, r.inst, m.uD, m.u0) for r, m in zip(reqs, meas)]
    for t in tickets:
        wos.wos_wait(q, t)
    t_sat = time.perf_counter() - t0
    qst = wos.wos_queue_get_stats(q)
    wos.wos_queue_destroy(q)
    same = all(np.array_equal(t.u_gamma1, u) for t, u in zip(tickets, seq_u1))

    # latency: Poisson arrivals at 70 % of the served throughput
    rate = 0.7 * len(reqs) / t_sat
    arrive = np.array([r.arrival for r in reqs]) / rate
    done = [None] * len(reqs)
    live = {}
    lock = threading.Lock()
    stop = threading.Event()
    q = make_queue()

    def poller():
        while not stop.is_set() or live:
            with lock:
                items = list(live.items())
            for i, t in items:
                if wos.wos_poll(q, t):
                    done[i] = time.perf_counter()
                    with lock:
                        del live[i]
            time.sleep(0.0002)

    th = threading.Thread(target=poller)
    th.start()
    t_start = time.perf_counter()
    sub = []
    for i, (r, m) in enumerate(zip(reqs, meas)):
        while time.perf_counter() - t_start < arrive[i]:
            time.sleep(max(0.0, min(0.001, arrive[i] - (time.perf_counter() - t_start))))
        sub.append(time.perf_counter())
        t = wos.wos_submit(q, r.inst, m.uD, m.u0)
        with lock:
            live[i] = t
    stop.set()
    th.join()
    wos.wos_queue_destroy(q)
    lat = np.array([d - s for d, s in zip(done, sub)]) * 1e3
    # one-at-a-time at the same arrivals: FIFO single server
    fin, seq_lat = 0.0, []
    for a, sv in zip(arrive, seq_t):
        fin = max(fin, a) + sv
        seq_lat.append((fin - a) * 1e3)
    seq_lat = np.array(seq_lat)
    ctx.close()
    walks = sum(r.inst.M_D * r.inst.N for r in reqs)
    t_seq = float(np.sum(seq_t))
    pct = lambda a, p: float(np.percentile(a, p))
    return {
        "requests": len(reqs), "walks": walks, "t_sat": t_sat,
        "workload": f"first {len(reqs)} requests of a seeded 10,000-request "
                    "Poisson stream: 3-D unit ball / cube, 1536 patches, "
                    "K = diag(1,2,4) or random SPD, 256-1024 points, "
                    "N = 1e5, eps in {1e-3, 1e-4}, noise 0.1-5 %; "
                    "build + SVD + TSVD per request",
        "served": {"requests_per_s": len(reqs) / t_sat, "walks_per_s": walks / t_sat,
                   "latency_ms_p50": pct(lat, 50), "latency_ms_p99": pct(lat, 99),
                   "arrival_rate_per_s": rate, "slices": qst["slices"]},
        "one_at_a_time": {"requests_per_s": len(reqs) / t_seq, "walks_per_s": walks / t_seq,
                          "latency_ms_p50": pct(seq_lat, 50),
                          "latency_ms_p99": pct(seq_lat, 99),
                          "service_ms_p50": pct(np.array(seq_t) * 1e3, 50)},
        "served_over_one_at_a_time": t_seq / t_sat,
        "served_equals_alone": bool(same),
        "h2d_bytes": int(sum(r.inst.points.nbytes + m.uD.nbytes + m.u0.nbytes
                             for r, m in zip(reqs, meas))),
        "d2h_bytes": int(sum(8 * int(r.inst.partition.gamma1.sum()) for r in reqs)),
    }


def run_serve(args, rank: int, world: int, dist):
    """Serving alone (see measure_serve)."""
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    r = measure_serve(args, local)
    if rank != 0:
        return
    print(json.dumps({
        "metric": METRIC, "value": r["requests"] / r["t_sat"], "unit": "requests/s",
        "n_gpus": world, "steps": 1, "warmup": 1, "ms_per_step": 1e3 * r["t_sat"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 walks, f64 SVD/TSVD", "data": "synthetic",
        "config": {"workload": r["workload"], "walks": r["walks"],
                   "side_streams": args.serve_side, "slice_walks": args.serve_slice},
        "served": r["served"], "one_at_a_time": r["one_at_a_time"],
        "served_over_one_at_a_time": r["served_over_one_at_a_time"],
        "served_equals_alone": r["served_equals_alone"],
        "e2e": {"value": r["requests"] / r["t_sat"], "unit": "requests/s",
                "h2d_bytes_per_step": r["h2d_bytes"], "d2h_bytes_per_step": r["d2h_bytes"]},
    }))


def run_svd(args, rank: int, world: int, dist):
    """The FP64 SVD alone (QR preconditioning + Jacobi on R^T + left vectors)
    on seeded operator-shaped count matrices of the two operator sizes of
    the paper's 2-D experiments (M_D x M_1 = 256 x 128 and 1024 x 768),
    one wos_op_svd call per shape per step.  factorisation = the QR and the
    Jacobi sweeps (the cluster kernel; or the grid-wide QR, X and Jacobi
    launches, with the FP32 sweeps, their replay and the Newton-Schulz
    products between them above 256 columns)."""
    import torch
    from paper_2409_03686_gb300 import build as B
    from paper_2409_03686_gb300 import workloads as W
    from paper_2409_03686_gb300 import wos
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.build()
    ctx = wos.Context(local)
    wos.wos_set_svd_path(ctx, SVD_PATHS[args.svd_path])
    N = 100_000
    shapes = [(256, 256, 128), (1024, 1536, 768)]
    probs = []
    for M_D, M_tot, M_1 in shapes:
        C = torch.as_tensor(W.synthetic_counts(M_D, M_tot, N, seed=M_D).astype(np.int32),
                            device=dev)
        g1 = np.zeros(M_tot, np.uint8)
        g1[:M_1] = 1
        sg = torch.full((M_tot,), 2 * np.pi / M_tot, dtype=torch.float64, device=dev)
        probs.append((C, N, g1, sg))
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in probs]
    for e in evs:  # create the events; the library re-records e[1], e[2]
        for x in e:
            x.record()
    res = [dict(call=[], jac=[], sweeps=0) for _ in probs]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for it in range(args.warmup + args.steps):
        for q, pb in enumerate(probs):
            e = evs[q]
            flush.zero_()  # L2 flushed before every timed call
            torch.cuda.synchronize()
            e[0].record()
            out = wos.wos_op_svd_batched(ctx, [pb], jacobi_events=(e[1], e[2]))
            e[3].record()
            torch.cuda.synchronize()
            if it >= args.warmup:
                res[q]["call"].append(e[0].elapsed_time(e[3]))
                res[q]["jac"].append(e[1].elapsed_time(e[2]))
            res[q]["sweeps"] = out[0][3]
    if rank != 0:
        return
    per = []
    for (M_D, M_tot, M_1), r in zip(shapes, res):
        call, jac = float(np.median(r["call"])), float(np.median(r["jac"]))
        fl = svd_fp64_flop(M_D, M_1, r["sweeps"], args.svd_path)
        per.append({"shape": f"{M_D}x{M_1}", "ms_per_call": call, "factorisation_ms": jac,
                    "sweeps": r["sweeps"], "factorisation_gflops": fl / jac / 1e6,
                    "factorisation_frac_fp64_peak": fl / jac / 1e6 / FP64_PEAK_GFLOPS})
    total = sum(p["ms_per_call"] for p in per)
    print(json.dumps({
        "metric": "fp64_svd_ms", "value": total, "unit": "ms", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "svd_path": args.svd_path,
        "config": {"workload": "FP64 SVD of seeded operator-shaped counts, 256x128 and "
                               "1024x768 (M_D x M_1), N = 1e5, one call per shape per step",
                   "l2": "flushed before every timed call (256 MiB write, outside it)"},
        "per_shape": per,
    }))


def run_chains(args, rank: int, world: int, dist):
    """The paper's eps and the mapped chains, measured (operator builds
    only, median of 3 timed builds after one warm-up, L2 flushed before each):
    * Ex. 5.4 (perforated disc) and Ex. 5.2 (annulus, extrinsic Voronoi
      cells) at the paper's N = 1e6 and eps = 1e-10 with FP64 walks: ms per
      build, walks/s, steps per walk and the averaged measure of Gamma_1
      (printed 0.1126 for Ex. 5.4; ln 0.95 / ln 0.5 = 0.0740 for Ex. 5.2);
    * the benchmark instances with the paper's chain and with the mapped
      chain (wos_opts.mapped: exact distance in y = S^{-1} x for the square
      and the cube, the quadric lower bound for the annulus and the balls),
      FP32: ms per build and steps per walk."""
    import torch
    from paper_2409_03686_gb300 import build as B
    from paper_2409_03686_gb300 import workloads as W
    from paper_2409_03686_gb300 import wos
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.build()
    ctx = wos.Context(local)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def timed_build(inst, mapped=False):
        pts = torch.as_tensor(inst.points, dtype=torch.float64, device=dev)
        opts = wos.make_opts(precision=int(inst.fp64), stream_id=inst.stream, mapped=mapped)
        ms, st, c = [], None, None
        for it in range(4):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            c, _, st = wos.wos_build_operator(ctx, inst.domain, inst.K, pts, inst.partition,
                                              inst.N, inst.eps, inst.seed, opts=opts)
            e1.record()
            torch.cuda.synchronize()
            if it:
                ms.append(e0.elapsed_time(e1))
        walks = inst.M_D * inst.N
        m = float(np.median(ms))
        return {"ms_per_build": m, "walks_per_s": walks / (m / 1e3),
                "steps_per_walk": st["steps"] / walks, "unterminated": st["unterminated"]}, c

    out = {}
    for name, inst, ref in (
            ("ex5.4 perforated disc, FP64, eps=1e-10, N=1e6",
             W.perforated_disc_config(), 0.1126),
            ("ex5.2 annulus (Voronoi cells), FP64, eps=1e-10, N=1e6",
             W.annulus_voronoi_config(), math.log(0.95) / math.log(0.5))):
        r, c = timed_build(inst)
        g1 = torch.as_tensor(inst.partition.gamma1.astype(bool), device=dev)
        r["avg_mu_gamma1"] = float((c[:, g1].sum(1).double() / inst.N).mean())
        r["reference_value"] = ref
        out[name] = r
    cmp = {}
    insts = [W.square_config(), W.annulus_config()] + W.config3_instances()
    for inst in insts:
        a, _ = timed_build(inst)
        b, _ = timed_build(inst, mapped=True)
        cmp[inst.name + ("-randK" if inst.dim == 3 and inst.K[0, 1] != 0 else "")] = {
            "paper_chain": a, "mapped_chain": b,
            "speedup": a["ms_per_build"] / b["ms_per_build"]}
    if rank == 0:
        print(json.dumps({"metric": "operator build ms (paper eps; mapped chains)",
                          "value": out, "mapped_vs_paper_chain": cmp, "unit": "ms",
                          "higher_is_better": False, "n_gpus": world,
                          "data": "synthetic"}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 30 on config3, 100 on the 2-D workloads)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="config3",
                    help="config3 (default), square-annulus, small, config3-small, "
                         "batch, serve, svd, chains")
    ap.add_argument("--no-extras", action="store_true",
                    help="config3 without the served-latency and batching measurements")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--svd-path", choices=list(SVD_PATHS), default="auto",
                    help="SVD factorisation kernels: auto (cluster kernel when the "
                         "operator fits it) or grid (grid-wide kernels)")
    ap.add_argument("--walk-blocks-per-sm", type=int, default=0,
                    help="cap on the walk launches' resident blocks per SM (0: as tuned)")
    ap.add_argument("--svd-streams", type=int, default=0,
                    help="SVD streams the pipelined steps alternate over (0: two for the "
                         "3-D configuration, whose SVDs take longer than its walks; four "
                         "for the 2-D one)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="default launch configuration (profiling: no trial launches)")
    ap.add_argument("--batch-scale", type=float, default=1.0,
                    help="walks-per-point scale of the batch workload")
    ap.add_argument("--serve-requests", type=int, default=128,
                    help="prefix of the served request stream")
    ap.add_argument("--serve-side", type=int, default=8,
                    help="concurrent SVD / reconstruction pipelines of the queue")
    ap.add_argument("--serve-slice", type=int, default=4096,
                    help="walks per point per batched slice of the queue")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 30 if args.workload.startswith("config3") else 100
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
    elif args.workload == "serve":
        run_serve(args, rank, world, dist)
    elif args.workload == "svd":
        run_svd(args, rank, world, dist)
    elif args.workload == "chains":
        run_chains(args, rank, world, dist)
    else:
        run_gpu(args, rank, world, dist)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
