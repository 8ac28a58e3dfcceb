"""Benchmark: delta-tracking walk on spheres on the 3D manufactured workload.

Workload (one "step" = one full solve): unit cube, u = e^{x/2} sin(pi y) cos(pi z),
alpha = 1 + 0.3 |x|^2, sigma = 1 + x y, drift omega = alpha grad(Phi) with
Phi = x sin(2 pi y) + sin(2 pi z)/(2 pi) + z/2, f from eq. 1, g = u, eps = 1e-4;
64^3 = 262,144 cell-centre points x 1024 walks, FP32 walk state, FP64 per-point
accumulators.  Metric: walk-steps/s (one step = one distance query + one
Green's-function sample).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

`--impl reference` times the FP64 CPU oracle (the only reference of this
method here) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "walk-steps/s"
UNIT = "steps/s"
GRID = 64
WALKS = 1024
DEFAULT_WALKS = WALKS  # the other workloads use their own walk counts unless --walks is given
EPS = 1e-4
SEED = 0
SIGMA_LATTICE = 64
# Algorithmic work of one walk step of this workload, for a minimal implementation of the
# step with the fields as code: FP32/INT32 lane operations -- one Philox block 80, the six
# 21-bit uniforms (split 12, conversions 18) 30, directions 16, box distance 17, Green's
# norm 14, radius (table start + one Newton step of the radial CDF) 62, coefficients
# (alpha, Phi, sigma, u_m with value / gradient / Laplacian, f, the transform) 74, update
# 12 -> 305; special-function (MUFU) operations -- directions 6, Green's norm 3, radius 6,
# coefficients 12 -> 27.  Every warp instruction takes one issue slot whatever its pipe, and
# the lanes issue at the FP32 lane rate, so the step needs 332 issue slots; the MUFU pipe
# (its own rate) is a separate, looser bound.
LANE_OPS_PER_STEP = 305
MUFU_OPS_PER_STEP = 27
ISSUE_OPS_PER_STEP = LANE_OPS_PER_STEP + MUFU_OPS_PER_STEP
RMS_TARGET = 1e-2
L2_FLUSH_BYTES = 512 << 20
# DRAM bytes (read + write) of one launch of the specialised walk kernel on the 64^3-point
# workload, from the ncu capture summarised in profiles/wos_walk_spec_kernel_cube3d.md:
# 9.51 MB read, 0 written, at 64 walks per point.  The bytes are per point (the points, the
# accumulators, the radial table); walk state stays in registers, so the 1024-walk launch
# moves the same bytes.  Reported for 64^3 points only; re-take it whenever the kernel changes.
TRAFFIC_BYTES_PER_LAUNCH = 9.50784e6


def measure_unit_peaks(ctx):
    """Measured rates of the units the walk kernel uses (library micro-benchmarks, CUDA events)."""
    lanes, lanes_ms = ctx.measure_peak("fp32_lanes")
    mufu, mufu_ms = ctx.measure_peak("mufu")
    l2, l2_ms = ctx.measure_peak("l2_read", 32 << 20)
    return {"fp32_lanes_per_s": lanes, "mufu_ops_per_s": mufu, "l2_read_bytes_per_s": l2,
            "how": "wos_measure_peak: FFMA / rsqrt.approx chains at 32 warps per SM; 16-byte cache-global "
                   "loads of a 32 MiB buffer; 5 launches after one warm-up, CUDA events"}


def mesh_l2_record(ctx, args, l2_peak):
    """L2 roofline of the mesh walk (the displaced icosphere with 128^3 noise grids, distance
    queries with tolerance 0.1): algorithmic L2 bytes per step from the kernel's node and
    triangle counters plus the field taps, over the kernel time, against the measured L2
    read rate.  16,384 interior points x 64 walks, three timed solves."""
    import torch
    desc = W.mesh_noise_problem(level=7, tol=0.1)
    prob = make_problem(ctx, desc, args)
    sb = ctx.sigma_bar(prob, 48)[0]
    pts = torch.from_numpy(W.mesh_interior_points(16384, seed=0)).cuda()
    ctx.solve(prob, pts, 64, 1e-4, sb, seed=0)
    torch.cuda.synchronize()
    ms, st = [], None
    for i in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _, st = ctx.solve(prob, pts, 64, 1e-4, sb, seed=1 + i)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    import paper_2201_13240_gb300 as wos
    sd = wos.stats_dict(st)
    t = sum(ms) / len(ms)
    nodes, tris = sd["mesh_nodes"] / sd["steps"], sd["mesh_tris"] / sd["steps"]
    bps = 128.0 * nodes + 48.0 * tris + 4.0 * (64 + 8 + 8)
    rate = bps * sd["steps"] / (t * 1e-3)
    prob.close()
    return {"workload": "displaced icosphere (327,680 triangles), 128^3 noise grids, 16384 interior points x 64 "
                        "walks, eps 1e-4, distance-query tolerance 0.1",
            "steps_per_s": sd["steps"] / (t * 1e-3), "steps_per_walk": sd["steps"] / sd["walks"],
            "nodes_per_step": nodes, "triangles_per_step": tris, "bytes_per_step": bps,
            "gb_per_s": rate / 1e9, "peak_gb_per_s": l2_peak / 1e9, "frac": rate / l2_peak,
            "basis": "BVH nodes x 128 B + triangles x 48 B (kernel counters) + alpha B-spline 64 and sigma, f "
                     "multilinear 8 taps x 4 B per step; peak: wos_measure_peak L2 read (32 MiB buffer)"}


def walks_for_rms(ctx, prob, pts, exact, sb, n_guess, stream, seed):
    """The smallest tried walks-per-point whose normalised RMS against the exact solution is at
    most RMS_TARGET: geometric steps of 10% up from 0.8 x the noise-model guess; each try is one
    solve (fresh accumulators, device-timed with CUDA events)."""
    import torch
    npts = pts.shape[1]
    acc = ctx.new_accum(npts)
    n = max(256, int(math.ceil(0.8 * n_guess / 256.0)) * 256)
    tries = []
    for _ in range(8):
        for t in acc:
            t.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.solve(prob, pts, n, EPS, sb, seed=seed, accum=acc)
        m, _, _ = ctx.finalize(acc)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        rms = float(np.linalg.norm(m.cpu().numpy() - exact) / np.linalg.norm(exact))
        tries.append([n, rms, ms])
        if rms <= RMS_TARGET:
            return {"walks_per_point": n, "normalised_rms": rms, "solve_ms": ms,
                    "points_per_s": npts / (ms * 1e-3), "tries": tries, "seed": seed}
        n = int(math.ceil(1.1 * n / 256.0)) * 256
    return {"walks_per_point": None, "tries": tries, "seed": seed}


def workload_config(extra=None):
    cfg = {"workload": f"cube3d_drift_manufactured: {GRID}^3 points x {WALKS} walks, eps 1e-4, FP32 walks, "
                       "FP64 sums",
           "points": GRID ** 3, "walks_per_point": WALKS, "eps": EPS, "seed": SEED,
           "l2": "flushed between timed steps (512 MiB write)"}
    if extra:
        cfg.update(extra)
    return cfg


JIT = {"compile_s": 0.0}


def make_problem(ctx, desc, args, variants=("plain",)):
    """Upload a problem; with --kernel specialised (the default) also compile and load the walk
    kernels specialised to its fields (the compile time is reported, outside the timed region)."""
    t0 = time.perf_counter()
    prob = ctx.problem(desc, specialize=(("fp32",), variants) if args.kernel == "specialised" else None)
    if args.kernel == "specialised":
        JIT["compile_s"] += time.perf_counter() - t0
    return prob


def kernel_label(args):
    return ("wos_walk_spec_kernel<3,float>: the walk kernel specialised to the problem's fields (NVRTC, sm_103a)"
            if args.kernel == "specialised" else "wos_walk_kernel<3,float> (generic field interpreter)")


def rank_info():
    r = int(os.environ.get("RANK", "0"))
    w = int(os.environ.get("WORLD_SIZE", "1"))
    lr = int(os.environ.get("LOCAL_RANK", "0"))
    return r, w, lr


# ---------------------------------------------------------------------------
# clocks sampled with nvidia-smi while the timed region runs
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"wos_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
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
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline leg and the reference arm)
# ---------------------------------------------------------------------------
def oracle_rate(desc, sb, npoints, walks, seed):
    import oracle
    oracle.build()
    pts = W.cell_centres(3, GRID)[:, W.seeded_subset(GRID ** 3, npoints, 77 + seed)]
    t0 = time.perf_counter()
    _, st = oracle.solve(desc, pts, walks, seed=seed, eps=EPS, sigma_bar=sb)
    dt = time.perf_counter() - t0
    return st["steps"], dt


def run_reference(args):
    r, world, _ = rank_info()
    if r != 0:
        return 0
    import oracle
    oracle.build()
    desc = W.cube3d_problem()
    sb = oracle.sigma_bar(desc, SIGMA_LATTICE)[0]
    npoints = 96  # per step: 96 points x 1024 walks (a bounded sample of the workload)
    for i in range(args.warmup):
        oracle_rate(desc, sb, npoints, WALKS, seed=1000 + i)
    tot_steps, tot_t = 0, 0.0
    for i in range(args.steps):
        s, dt = oracle_rate(desc, sb, npoints, WALKS, seed=i)
        tot_steps += s
        tot_t += dt
    value = tot_steps / tot_t
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config({"sample": f"{npoints} seeded points x {WALKS} walks "
                                                                      "per step"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{npoints} seeded points x {WALKS} walks per step, FP64, OpenMP"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch

    rank, world, local_rank = rank_info()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_2201_13240_gb300 as wos

    ctx = wos.Context(local_rank)
    desc = W.cube3d_problem()
    prob = make_problem(ctx, desc, args)
    sb, smin, smax = ctx.sigma_bar(prob, SIGMA_LATTICE)
    pts_np = W.cell_centres(3, GRID)
    npts = pts_np.shape[1]
    pts = torch.from_numpy(pts_np).cuda()
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    acc = ctx.new_accum(npts)
    stats = ctx.new_stats()
    mean = torch.empty(npts, dtype=torch.float64, device="cuda")
    # disjoint walk ids per rank: the ranks' walks would merge into one estimate
    offset = rank * WALKS

    def step(seed):
        for t in acc:
            t.zero_()
        ctx.solve(prob, pts, WALKS, EPS, sb, seed=seed, walk_offset=offset, accum=acc, stats=stats)
        m, v, se = ctx.finalize(acc)
        return m, se

    for i in range(max(args.warmup, 0)):
        step(SEED)
    torch.cuda.synchronize()
    stats.zero_()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        for i in range(args.steps):
            flush.fill_(float(i))      # evict L2 between timed steps (outside the events)
            ev[i][0].record(stream)
            m, se = step(SEED)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    times = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(times)
    st = wos.stats_dict(stats)
    # the same steps through the generic kernel (field interpreter), for comparison
    generic = None
    if args.kernel == "specialised":
        gprob = ctx.problem(desc)
        gacc, gst = ctx.new_accum(npts), ctx.new_stats()
        ctx.solve(gprob, pts, WALKS, EPS, sb, seed=SEED, walk_offset=offset, accum=gacc, stats=gst)
        torch.cuda.synchronize()
        gst.zero_()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        gms = 0.0
        for i in range(args.steps):
            for t in gacc:
                t.zero_()
            flush.fill_(float(i))
            g0.record(stream)
            ctx.solve(gprob, pts, WALKS, EPS, sb, seed=SEED, walk_offset=offset, accum=gacc, stats=gst)
            ctx.finalize(gacc)
            g1.record(stream)
            torch.cuda.synchronize()
            gms += g0.elapsed_time(g1)
        generic = {"value": wos.stats_dict(gst)["steps"] / (gms * 1e-3), "unit": UNIT, "ms_per_step": gms / args.steps}
        gprob.close()
    if dist is not None:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        s = torch.tensor([st["steps"]], dtype=torch.float64, device="cuda")
        dist.all_reduce(s)
        all_steps = float(s.item())
    else:
        all_steps = float(st["steps"])
    value = all_steps / (total_ms * 1e-3)
    ms_per_step = total_ms / args.steps
    steps_per_walk = st["steps"] / max(st["walks"], 1)

    # accuracy of the last estimate against the manufactured solution
    exact = W.cube3d_exact(*pts_np.astype(np.float64))
    m_np = m.cpu().numpy()
    rms = float(np.linalg.norm(m_np - exact) / np.linalg.norm(exact))
    # the ranks walked disjoint walk ids of the same points: their accumulators merge into
    # one estimate with world x WALKS walks per point (one all-reduce of sum, sumsq, count)
    rms_merged = rms
    if dist is not None:
        from paper_2201_13240_gb300 import multi
        multi.merge_accumulators(acc)
        mm = ctx.finalize(acc)[0].cpu().numpy()
        rms_merged = float(np.linalg.norm(mm - exact) / np.linalg.norm(exact))
    se_np = se.cpu().numpy()
    # walks per point for normalised RMS 1e-2 (noise part scales as 1/sqrt(N))
    noise = float(np.sqrt(np.mean(se_np ** 2)) / np.sqrt(np.mean(exact ** 2)))
    walks_for_1e2 = int(math.ceil(WALKS * (noise / 1e-2) ** 2))

    # end to end through the C interface with HOST buffers (copies inside the timed region)
    pin_pts = torch.from_numpy(pts_np).pin_memory()
    out = (torch.empty(npts, dtype=torch.float64).pin_memory(), torch.empty(npts, dtype=torch.float64).pin_memory(),
           torch.empty(npts, dtype=torch.float64).pin_memory(),
           torch.zeros(wos.STATS_WORDS, dtype=torch.int64).pin_memory())
    e2e_steps = 0
    ctx.solve_host(prob, pin_pts, WALKS, EPS, sb, seed=SEED, walk_offset=offset, out=out)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        ctx.solve_host(prob, pin_pts, WALKS, EPS, sb, seed=SEED, walk_offset=offset, out=out)
        e2e_steps += int(out[3][0])
    e2e_t = time.perf_counter() - t0
    if dist is not None:
        t = torch.tensor([e2e_t], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_t = float(t.item())
        e2e_steps *= world
    e2e = {"value": e2e_steps / e2e_t, "unit": UNIT, "h2d_bytes_per_step": 3 * 4 * npts,
           "d2h_bytes_per_step": 3 * 8 * npts + 8 * wos.STATS_WORDS}

    # roofline of the walk kernel (ALU bound): algorithmic issue slots / kernel time, against
    # the lane rate measured in this run (and each pipe against its own measured rate)
    peaks = measure_unit_peaks(ctx)
    # kernel time: the solve dominates the step; finalize and memsets are timed separately below
    fe0, fe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fe0.record(stream)
    for _ in range(5):
        ctx.finalize(acc)
    fe1.record(stream)
    torch.cuda.synchronize()
    finalize_ms = fe0.elapsed_time(fe1) / 5
    kernel_ms = ms_per_step - finalize_ms
    steps_per_s_kernel = (st["steps"] / args.steps) / (kernel_ms * 1e-3)
    achieved = ISSUE_OPS_PER_STEP * steps_per_s_kernel
    peak_lanes = peaks["fp32_lanes_per_s"]
    captured = args.kernel == "specialised" and GRID == 64
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_lanes / 1e12, "unit": "Tops/s",
                "frac": achieved / peak_lanes, "traffic": TRAFFIC_BYTES_PER_LAUNCH if captured else None,
                "traffic_unit": "bytes per launch (dram read + write, ncu)",
                "kernel": kernel_label(args), "ops_per_step": ISSUE_OPS_PER_STEP,
                "peak_basis": "measured in this run: FP32 FMA lane operations per second (wos_measure_peak); "
                              "one issue slot per lane operation",
                "pipes": {"fp32_int_lanes": {"ops_per_step": LANE_OPS_PER_STEP,
                                             "frac": LANE_OPS_PER_STEP * steps_per_s_kernel / peak_lanes},
                          "mufu": {"ops_per_step": MUFU_OPS_PER_STEP,
                                   "frac": MUFU_OPS_PER_STEP * steps_per_s_kernel / peaks["mufu_ops_per_s"]}},
                "measured_peaks": peaks}

    # points/s at normalised RMS 1e-2, measured: the smallest tried walk count that reaches it
    rms_run = walks_for_rms(ctx, prob, pts, exact, sb, walks_for_1e2, stream, SEED + 1000) if rank == 0 else None
    mesh_l2 = mesh_l2_record(ctx, args, peaks["l2_read_bytes_per_s"]) if rank == 0 else None

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    # CPU baseline: the oracle on a bounded sample on this host's cores
    cpu = None
    if not args.no_cpu_baseline:
        cpu_pts = 512
        o_steps, o_t = oracle_rate(desc, sb, cpu_pts, WALKS, seed=SEED)
        cpu = {"value": o_steps / o_t, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{cpu_pts} seeded points of the workload x {WALKS} walks, FP64 oracle, OpenMP, "
                         f"{o_t:.1f} s"}
    clocks = clk.summary()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config({"sigma_bar": sb, "parallelism": f"points replicated, disjoint walk ids, "
                                                                        f"{world} GPU(s)",
                                       "kernel": args.kernel}),
            "specialise_compile_s": JIT["compile_s"], "generic_kernel": generic,
            "points_per_s": world * npts / (ms_per_step * 1e-3),
            "walks_per_s": world * npts * WALKS / (ms_per_step * 1e-3),
            "steps_per_walk": steps_per_walk, "normalised_rms_at_1024_walks": rms,
            "normalised_rms_merged_over_ranks": rms_merged,
            "noise_model_walks_for_rms_1e-2": walks_for_1e2,
            "points_per_s_at_rms_1e-2": rms_run.get("points_per_s"), "rms_1e-2_run": rms_run,
            "capped_walks": st["capped"], "nonfinite_walks": st["nonfinite"],
            "e2e": e2e, "gpu_launches": 2 * args.steps, "roofline": roofline, "mesh_l2": mesh_l2,
            "cpu_baseline": cpu,
            "clocks": clocks}
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_other(args):
    """Measurements of the other workloads (one GPU): walk-steps/s of each, and for the
    inverse problem the adjoint (gradient) rate against the forward rate."""
    import torch

    import paper_2201_13240_gb300 as wos

    ctx = wos.Context(0)
    wl = args.workload
    extra = {}

    def timed(fn, reps):
        fn(0)
        torch.cuda.synchronize()
        ms = []
        for i in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            out = fn(i + 1)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return out, sum(ms) / len(ms)

    if wl == "square2d":
        desc = W.square2d_problem()
        prob = make_problem(ctx, desc, args)
        sb = ctx.sigma_bar(prob, 256)[0]
        pts_np = W.cell_centres(2, 32)
        pts = torch.from_numpy(pts_np).cuda()
        walks = args.walks if args.walks != DEFAULT_WALKS else 256
        (acc, st), ms = timed(lambda i: ctx.solve(prob, pts, walks, 1e-3, sb, seed=i), args.steps)
        m, v, se = (t.cpu().numpy() for t in ctx.finalize(acc))
        exact = W.square2d_exact(*pts_np.astype(np.float64))
        extra["normalised_rms"] = float(np.linalg.norm(m - exact) / np.linalg.norm(exact))
        cfg = {"workload": f"square2d_manufactured: 32^2 points x {walks} walks, eps 1e-3", "sigma_bar": sb}
        npts = pts_np.shape[1]
    elif wl == "grad":
        desc = W.cube3d_problem()
        prob = make_problem(ctx, desc, args, ("plain", "grad"))
        sb = ctx.sigma_bar(prob, 64)[0]
        pts_np = W.cell_centres(3, GRID)
        pts = torch.from_numpy(pts_np).cuda()
        npts = pts_np.shape[1]
        (acc, gacc, st), ms = timed(lambda i: ctx.solve_grad(prob, pts, WALKS, 1e-4, sb, seed=i), args.steps)
        (acc0, st0), ms0 = timed(lambda i: ctx.solve(prob, pts, WALKS, 1e-4, sb, seed=i), args.steps)
        gm, gv, gse = (t.cpu().numpy() for t in ctx.finalize_grad(gacc, acc[2]))
        exact = W.cube3d_exact_grad(*pts_np.astype(np.float64))
        # the first ball of a point at distance d weights by ~1/d: near the boundary the
        # gradient estimate is far noisier, so the error is reported for d >= 0.1 too
        dist = np.minimum(pts_np, 1.0 - pts_np).min(axis=0)
        inner = dist >= 0.1
        extra["grad_normalised_rms"] = float(np.linalg.norm(gm - exact) / np.linalg.norm(exact))
        extra["grad_normalised_rms_d_ge_0.1"] = float(np.linalg.norm((gm - exact)[:, inner]) /
                                                      np.linalg.norm(exact[:, inner]))
        extra["value_only_ms"] = ms0
        extra["grad_over_value_time"] = ms / ms0
        cfg = {"workload": f"cube3d_drift_manufactured with grad u (Supplemental Sec. 2): {GRID}^3 points x "
                           f"{WALKS} walks, eps 1e-4", "sigma_bar": sb}
    elif wl == "nf":
        # next-flight (Sec. 5.2) against delta tracking on the 3D workload: balls (distance
        # queries) and inner iterations per walk, and the time for the same walks
        desc = W.cube3d_problem()
        prob = ctx.problem(desc)
        sb = ctx.sigma_bar(prob, 64)[0]
        pts_np = W.cell_centres(3, GRID)
        pts = torch.from_numpy(pts_np).cuda()
        npts = pts_np.shape[1]
        nser = args.nf_series
        exact = W.cube3d_exact(*pts_np.astype(np.float64))

        def rms_of(acc_):
            m_, v_, se_ = (t.cpu().numpy() for t in ctx.finalize(acc_))
            return float(np.linalg.norm(m_ - exact) / np.linalg.norm(exact)), float(np.mean(se_))
        # the series kernels (N terms), then the printed approximations and delta tracking
        (acc, st), ms = timed(lambda i: ctx.solve_nf(prob, pts, WALKS, 1e-4, sb, seed=i, series_terms=nser),
                              args.steps)
        rms, mse = rms_of(acc)
        (acc_a, st_a), ms_a = timed(lambda i: ctx.solve_nf(prob, pts, WALKS, 1e-4, sb, seed=i, series_terms=0),
                                    args.steps)
        rms_a, mse_a = rms_of(acc_a)
        (acc0, st0), ms0 = timed(lambda i: ctx.solve(prob, pts, WALKS, 1e-4, sb, seed=i), args.steps)
        rms0, mse0 = rms_of(acc0)
        sd, sa, s0 = wos.stats_dict(st), wos.stats_dict(st_a), wos.stats_dict(st0)
        extra["series_terms"] = nser
        extra["inner_per_walk"] = sd["inner"] / max(sd["walks"], 1)
        extra["inner_per_s"] = sd["inner"] / (ms * 1e-3)
        extra["normalised_rms"] = rms
        extra["mean_stderr_over_delta_tracking"] = mse / mse0
        extra["approximate_kernels"] = {"ms": ms_a, "normalised_rms": rms_a, "mean_stderr_over_delta_tracking":
                                        mse_a / mse0, "inner_per_walk": sa["inner"] / max(sa["walks"], 1)}
        extra["delta_tracking_ms"] = ms0
        extra["delta_tracking_steps_per_walk"] = s0["steps"] / max(s0["walks"], 1)
        extra["delta_tracking_normalised_rms"] = rms0
        # Sec. 5.2's point: next-flight walks take one distance query per ball, flat in
        # sigma_bar, where delta tracking takes one per step.  On the triangle mesh (the
        # manufactured problem on the displaced icosphere, certified radii) at the problem's
        # sigma_bar and at 8 times it
        if not args.no_nf_mesh:
            dm = W.mesh_manufactured_problem(level=7, tol=args.mesh_tol)
            pm = ctx.problem(dm)
            pm.specialize(("fp32",), ("plain",))
            sbm = ctx.sigma_bar(pm, 48)[0]
            pts_m_np = W.mesh_interior_points(16384, seed=0)
            pts_m = torch.from_numpy(pts_m_np).cuda()
            exm = W.cube3d_exact(*pts_m_np.astype(np.float64))
            wm = 256
            mesh_leg = {"points": 16384, "walks": wm, "mesh_tol": args.mesh_tol}
            for fac in (1, 8):
                (a_nf, s_nf), ms_nf = timed(lambda i: ctx.solve_nf(prob=pm, pts=pts_m, walks=wm, eps=1e-4,
                                                                   sigma_bar=fac * sbm, seed=i, series_terms=nser),
                                            args.steps)
                (a_dt, s_dt), ms_dt = timed(lambda i: ctx.solve(pm, pts_m, wm, 1e-4, fac * sbm, seed=i), args.steps)
                dn, dd_ = wos.stats_dict(s_nf), wos.stats_dict(s_dt)
                mn = ctx.finalize(a_nf)[0].cpu().numpy()
                md = ctx.finalize(a_dt)[0].cpu().numpy()
                mesh_leg[f"sigma_bar_x{fac}"] = {
                    "sigma_bar": fac * sbm,
                    "next_flight": {"ms": ms_nf, "balls_per_walk": dn["steps"] / max(dn["walks"], 1),
                                    "inner_per_walk": dn["inner"] / max(dn["walks"], 1),
                                    "normalised_rms": float(np.linalg.norm(mn - exm) / np.linalg.norm(exm))},
                    "delta_tracking": {"ms": ms_dt, "steps_per_walk": dd_["steps"] / max(dd_["walks"], 1),
                                       "normalised_rms": float(np.linalg.norm(md - exm) / np.linalg.norm(exm))}}
            extra["mesh"] = mesh_leg
        cfg = {"workload": f"cube3d_drift_manufactured, next-flight walks (off-centred G, P as the series of "
                           f"{nser} terms): {GRID}^3 points x {WALKS} walks, eps 1e-4; steps count balls",
               "sigma_bar": sb}
    elif wl == "c2literal":
        # config 2 with its literal, non-conservative drift (the extra-drift walk)
        desc = W.cube3d_literal_problem()
        prob = make_problem(ctx, desc, args)
        sb = ctx.sigma_bar(prob, 64)[0]
        pts_np = W.cell_centres(3, GRID)
        pts = torch.from_numpy(pts_np).cuda()
        npts = pts_np.shape[1]
        (acc, st), ms = timed(lambda i: ctx.solve(prob, pts, WALKS, 1e-4, sb, seed=i), args.steps)
        m, v, se = (t.cpu().numpy() for t in ctx.finalize(acc))
        exact = W.cube3d_exact(*pts_np.astype(np.float64))
        rms = float(np.linalg.norm(m - exact) / np.linalg.norm(exact))
        # a heavy tail of the walk's weights shows as a few points with large errors: the RMS
        # over all points against the RMS without the worst 0.1% measures it (the mixture ball
        # sample and the per-ball bounds of the drift walk bound its weights)
        err = np.abs(m - exact)
        keep = err <= np.quantile(err, 0.999)
        trimmed = float(np.linalg.norm((m - exact)[keep]) / np.linalg.norm(exact[keep]))
        extra["normalised_rms_without_worst_0.1pct_points"] = trimmed
        extra["rms_all_over_trimmed"] = rms / trimmed
        extra["median_abs_z"] = float(np.median(err / se))
        noise = float(np.sqrt(np.median(se ** 2)) / np.sqrt(np.mean(exact ** 2)))
        walks_1e2 = int(math.ceil(WALKS * (noise / 1e-2) ** 2))
        extra["normalised_rms"] = rms
        extra["walks_per_point_for_rms_1e-2"] = walks_1e2
        extra["points_per_s_at_rms_1e-2"] = npts / (ms * 1e-3) * WALKS / max(walks_1e2, 1)
        cfg = {"workload": f"cube3d with the literal drift omega = (sin 2 pi y, cos 2 pi z, 0.5): {GRID}^3 points x "
                           f"{WALKS} walks, eps 1e-4 (extra-drift walk; not in the paper)", "sigma_bar": sb}
    elif wl == "slice":
        # the interactive path (Sec. 7.2): one walk per slice point per frame plus the
        # sphere-traced image of the CSG scene cut by the slice plane
        desc = W.csg_variable_problem()
        prob = make_problem(ctx, desc, args)
        sb = ctx.sigma_bar(prob, 64)[0]
        res = args.points if args.points != 16384 else 512
        v = wos.view([-1.3, -1.3, 0.05], [2.6, 0, 0], [0, 2.6, 0], res, res, 1280, 720, (-3.0, 3.0),
                     eye=(2.5, 2.0, 3.5), look=(0, 0, 0))
        sv = wos.SliceView(ctx, prob, v, 1e-4, sb)
        for _ in range(3):
            sv.frame(1)
        torch.cuda.synchronize()
        nfr = max(args.steps, 1) * 10
        stats0 = wos.stats_dict(sv.stats)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(nfr):
            img = sv.frame(1)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / nfr
        s1 = wos.stats_dict(sv.stats)
        # per-frame statistics (the line's rates are per frame time)
        st = torch.tensor([(s1[k] - stats0[k]) // nfr for k in ("steps", "walks", "capped", "nonfinite", "outside",
                                                                "inner", "mesh_nodes", "mesh_tris", "exhausted")],
                          dtype=torch.int64)
        extra["frames_per_s"] = 1e3 / ms
        extra["frames"] = nfr
        npts = res * res
        if args.write_image:
            wos.write_ppm(args.write_image, img)
        cfg = {"workload": f"CSG scene (rounded box, capsule, sphere and torus cuts, half-space) with variable "
                           f"coefficients: {res}^2 slice points x 1 walk per frame + 1280x720 sphere-traced view, "
                           "eps 1e-4", "sigma_bar": sb}
    elif wl == "mesh":
        # distance queries with a certified-radius tolerance (the default walk of this line) and
        # with exact radii, on the same points, walks and seed; query work read from the
        # kernel's node and triangle counters
        l2_peak = ctx.measure_peak("l2_read", 32 << 20)[0]
        npts = args.points
        pts = torch.from_numpy(W.mesh_interior_points(npts, seed=0)).cuda()
        walks = args.walks if args.walks != DEFAULT_WALKS else 512
        sb = None
        runs, head_ms_st = {}, {}
        tols = (args.mesh_tol, 0.0) if args.mesh_tol > 0 else (0.0,)
        if args.no_mesh_exact and args.mesh_tol > 0:
            tols = (args.mesh_tol,)
        for tol in tols:
            desc = W.mesh_noise_problem(level=7, tol=tol)
            t0 = time.perf_counter()
            prob = ctx.problem(desc)
            build_s = time.perf_counter() - t0
            if args.kernel == "specialised":
                prob.specialize(("fp32",), ("plain",))
            if sb is None:
                sb = ctx.sigma_bar(prob, 48)[0]
            (acc, st), ms = timed(lambda i: ctx.solve(prob, pts, walks, 1e-4, sb, seed=i), args.steps)
            sd = wos.stats_dict(st)  # statistics of the last timed solve
            steps, walks_n = sd["steps"], sd["walks"]
            nodes, tris = sd["mesh_nodes"] / sd["steps"], sd["mesh_tris"] / sd["steps"]
            # bytes one step reads from L2: BVH nodes (128 B), triangles (3 x 16 B), and the
            # coefficient taps at y (alpha B-spline 64 x 4 B, sigma and f multilinear 8 x 4 B each)
            bps = 128.0 * nodes + 48.0 * tris + 4.0 * (64 + 8 + 8)
            m, v, se = ctx.finalize(acc)
            head_ms_st[tol] = (ms, st)
            runs[tol] = {"ms": ms, "steps_per_s": steps / (ms * 1e-3), "points_per_s": npts / (ms * 1e-3),
                         "steps_per_walk": steps / walks_n, "nodes_per_step": nodes, "triangles_per_step": tris,
                         "exhausted": sd["exhausted"], "bvh_build_s": build_s,
                         "l2": {"bytes_per_step": bps, "gb_per_s": bps * steps / (ms * 1e-3) / 1e9,
                                "peak_gb_per_s": l2_peak / 1e9, "frac": bps * steps / (ms * 1e-3) / l2_peak,
                                "basis": "algorithmic bytes of the visited nodes, tested triangles and field taps "
                                         "per step (kernel counters) / kernel time; peak: wos_measure_peak L2 read"},
                         "_mean": m.cpu().numpy(), "_se": se.cpu().numpy()}
        ms, st = head_ms_st[args.mesh_tol if args.mesh_tol > 0 else 0.0]
        extra["mesh_tol"] = args.mesh_tol
        for tol, r in runs.items():
            extra[f"tol_{tol}"] = {k: v for k, v in r.items() if not k.startswith("_")}
        if args.mesh_tol > 0 and 0.0 in runs:
            a, b = runs[args.mesh_tol], runs[0.0]
            extra["speedup_over_exact_radii"] = b["ms"] / a["ms"]
            extra["mean_abs_z_vs_exact_radii"] = float(np.mean(np.abs(a["_mean"] - b["_mean"]) /
                                                               np.sqrt(a["_se"] ** 2 + b["_se"] ** 2)))
        if args.dist_grid > 0:
            # the same problem with a distance grid: conservative radii away from the boundary
            # and exact queries nearer to it (with the certified-radius query there instead:
            # 580 ms against 485 ms, 10 % smaller balls where exact queries are cheap)
            dg = W.mesh_noise_problem(level=7, dist_grid=args.dist_grid)
            t0 = time.perf_counter()
            probg = make_problem(ctx, dg, args)
            torch.cuda.synchronize()
            build_g = time.perf_counter() - t0
            (accg, stg), msg = timed(lambda i: ctx.solve(probg, pts, walks, 1e-4, sb, seed=i), args.steps)
            sg = wos.stats_dict(stg)
            extra[f"dist_grid_{args.dist_grid}"] = {
                "ms": msg, "steps_per_walk": sg["steps"] / max(sg["walks"], 1),
                "steps_per_s": sg["steps"] / (msg * 1e-3), "points_per_s": npts / (msg * 1e-3),
                "build_s": build_g,
                "speedup_over_exact_radii": runs[0.0]["ms"] / msg if 0.0 in runs else None,
                "speedup_over_tol_alone": (runs[args.mesh_tol]["ms"] / msg) if args.mesh_tol in runs else None}
        cfg = {"workload": f"displaced icosphere (327,680 triangles), 128^3 noise grids: {npts} interior points "
                           f"x {walks} walks, eps 1e-4, distance-query tolerance {args.mesh_tol}", "sigma_bar": sb}
    elif wl == "batch":
        probs, pts_np, offs, walks_np = W.batch_problems(args.problems, seed=7)
        t0 = time.perf_counter()
        hp = [ctx.problem(p) for p in probs]
        sbs = [ctx.sigma_bar(h, 64)[0] for h in hp]
        batch = ctx.batch(hp, offs, sbs)
        extra["setup_s"] = time.perf_counter() - t0
        if args.kernel == "specialised":
            # the batched kernel with the fields every problem shares compiled in (before the
            # autotuner, whose trials then run it)
            t0 = time.perf_counter()
            batch.specialize(("fp32",))
            JIT["compile_s"] += time.perf_counter() - t0
            extra["shared_fields_mask"] = batch.specialized()[1]
        pts = torch.from_numpy(pts_np).cuda()
        wt = torch.from_numpy(walks_np).cuda()
        acc = ctx.new_accum(pts.shape[1])
        stt = ctx.new_stats()
        if not args.no_autotune:
            # launch schedule (chunk, register cap) from trial launches at 1/16 of the walks
            t0 = time.perf_counter()
            sched, best_ms, default_ms = ctx.batch_autotune(batch, pts, wt, 1e-3, seed=1, trial_shift=4)
            extra["autotune"] = {"schedule": sched, "trial_ms": best_ms, "default_trial_ms": default_ms,
                                 "tune_s": time.perf_counter() - t0}
        graph = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            ctx.solve_batch(batch, pts, wt, 1e-3, seed=0, accum=acc, stats=stt, stream=s)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=s):
            for t in acc:
                t.zero_()
            stt.zero_()
            ctx.solve_batch(batch, pts, wt, 1e-3, seed=0, accum=acc, stats=stt, stream=s)

        def run(i):
            graph.replay()
            return acc, stt
        (acc, st), ms = timed(run, args.steps)
        npts = pts.shape[1]
        if args.kernel == "specialised":
            # the same launch through the generic (field-interpreting) batched kernel
            gb = ctx.batch(hp, offs, sbs)
            gb.set_schedule(**batch.schedule())
            (_, gst), gms = timed(lambda i: ctx.solve_batch(gb, pts, wt, 1e-3, seed=0), args.steps)
            extra["generic_kernel"] = {"ms": gms, "steps_per_s": wos.stats_dict(gst)["steps"] / (gms * 1e-3)}
        # L2 roofline of the batched step: the grid taps it reads per step (alpha and Phi cubic
        # B-splines with derivatives, 16 taps each; sigma and f bilinear, 4 each; 4 B a tap)
        # over the kernel time, against the L2 read rate measured here
        l2_peak = ctx.measure_peak("l2_read", 32 << 20)[0]
        bps = 4.0 * (16 + 16 + 4 + 4)
        steps_b = wos.stats_dict(st)["steps"]
        extra["l2"] = {"bytes_per_step": bps, "gb_per_s": bps * steps_b / (ms * 1e-3) / 1e9,
                       "peak_gb_per_s": l2_peak / 1e9, "frac": bps * steps_b / (ms * 1e-3) / l2_peak,
                       "basis": "algorithmic bytes of the grid taps per step / kernel time; peak: "
                                "wos_measure_peak L2 read (ncu reads ~625 B per step of 32-byte sectors)"}
        cfg = {"workload": f"{args.problems} 2D problems (disk/annulus/rounded box, 64^2 noise grids), "
                           f"{npts} points, {int(walks_np.sum())} walks, one launch in a CUDA graph, eps 1e-3"}
    elif wl == "inverse":
        sig = W.inverse_sigma_grid()
        sig_t = torch.from_numpy(sig).cuda()
        desc = W.inverse_problem(sig)
        desc["sigma"] = dict(desc["sigma"], data=sig_t)
        # the forward walk and both replay adjoints compiled for the problem's fields
        prob = make_problem(ctx, desc, args, ("plain", "adjoint"))
        sb = ctx.sigma_bar(prob, 48)[0]
        npts = 4096
        pts = torch.from_numpy(W.inverse_sensors(npts)).cuda()
        walks = args.walks if args.walks != DEFAULT_WALKS else 1024
        gu = torch.ones(npts, dtype=torch.float64, device="cuda")
        grad = torch.zeros(sig.size, dtype=torch.float64, device="cuda")
        (acc, st), ms = timed(lambda i: ctx.solve(prob, pts, walks, 1e-4, sb, seed=i), args.steps)

        def adj(i):
            grad.zero_()
            stt = ctx.new_stats()
            ctx.adjoint_sigma(prob, pts, walks, gu, grad, 1e-4, sb, seed=i, stats=stt)
            return grad, stt
        (_, sta), ms_adj = timed(adj, args.steps)
        grad_a = torch.zeros(W.inverse_alpha_grid().size, dtype=torch.float64, device="cuda")

        def adj_alpha(i):
            grad_a.zero_()
            ctx.adjoint_alpha(prob, pts, walks, gu, grad_a, 1e-4, sb, seed=i)
            return grad_a
        _, ms_adj_a = timed(adj_alpha, args.steps)
        extra["adjoint_alpha_ms"] = ms_adj_a
        extra["adjoint_alpha_grads_per_s_over_forward_solves_per_s"] = ms / ms_adj_a
        if args.kernel == "specialised":
            # the generic (field-interpreting) adjoint kernels on the same walks, for comparison
            gprob = ctx.problem(desc)
            _, ms_g = timed(lambda i: (grad.zero_(), ctx.adjoint_sigma(gprob, pts, walks, gu, grad, 1e-4, sb,
                                                                       seed=i)), args.steps)
            _, ms_ga = timed(lambda i: (grad_a.zero_(), ctx.adjoint_alpha(gprob, pts, walks, gu, grad_a, 1e-4, sb,
                                                                          seed=i)), args.steps)
            extra["generic_adjoint_ms"] = {"sigma": ms_g, "alpha": ms_ga}
        extra["adjoint_ms"] = ms_adj
        extra["forward_solves_per_s"] = 1e3 / ms
        extra["adjoint_grads_per_s"] = 1e3 / ms_adj
        extra["adjoint_grads_per_s_over_forward_solves_per_s"] = ms / ms_adj
        cfg = {"workload": f"inverse sigma: 32^3 multilinear sigma, 16^3 B-spline alpha, {npts} sensors x {walks} "
                           "walks, eps 1e-4", "sigma_bar": sb}
    else:
        raise SystemExit(f"unknown workload {wl}")
    stv = wos.stats_dict(st)
    line = {"metric": METRIC, "value": stv["steps"] / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": 1, "ms_per_step": ms, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": cfg, "steps_per_walk": stv["steps"] / max(stv["walks"], 1),
            "points_per_s": npts / (ms * 1e-3), "walks_per_s": stv["walks"] / (ms * 1e-3),
            "capped_walks": stv["capped"], "nonfinite_walks": stv["nonfinite"],
            "kernel": args.kernel if wl != "nf" else "generic", "specialise_compile_s": JIT["compile_s"]}
    line.update(extra)
    print(json.dumps(line))
    return 0


def main():
    global GRID, WALKS
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--grid", type=int, default=GRID, help="points per axis (profiling runs use a smaller case)")
    ap.add_argument("--walks", type=int, default=WALKS, help="walks per point (profiling runs use fewer)")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle leg (profiling runs)")
    ap.add_argument("--workload", default="cube3d", choices=["cube3d", "square2d", "mesh", "batch", "inverse", "grad", "nf", "slice", "c2literal"],
                    help="cube3d is the benchmark; the others print supplementary measurements")
    ap.add_argument("--points", type=int, default=16384, help="mesh workload: interior points")
    ap.add_argument("--problems", type=int, default=4096, help="batch workload: problems")
    ap.add_argument("--write-image", default="", help="slice workload: write the last frame as a PPM file")
    ap.add_argument("--no-autotune", action="store_true", help="batch workload: keep the default launch schedule")
    ap.add_argument("--no-nf-mesh", action="store_true", help="nf workload: skip the triangle-mesh leg")
    ap.add_argument("--nf-series", type=int, default=8,
                    help="nf workload: terms of the off-centred kernels' series (1..64)")
    ap.add_argument("--kernel", default="specialised", choices=["specialised", "generic"],
                    help="walk kernel: compiled for the problem's fields (default) or the generic field interpreter")
    ap.add_argument("--mesh-tol", type=float, default=0.1,
                    help="mesh workload: certified-radius tolerance of the distance queries (0: exact radii only)")
    ap.add_argument("--no-mesh-exact", action="store_true",
                    help="mesh workload: skip the exact-radius comparison (sweeps)")
    ap.add_argument("--dist-grid", type=int, default=128,
                    help="mesh workload: also time walks with an n^3 distance grid (0: exact radii only)")
    args = ap.parse_args()
    GRID, WALKS = args.grid, args.walks
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "cube3d":
        return run_other(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
