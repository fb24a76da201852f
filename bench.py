"""Benchmark: receiver-sun-steps per second of shadow accumulation on one GB300.

Workload (default `district`): 2,000 synthetic convex buildings (~60k triangles), a
2048 x 2048 ground raster at 1 m plus 1,000,000 facade samples, one day 09:00-17:00 at
1-minute steps (481 sun directions).  One step = one full accumulation of every receiver
over every sun step with the shadow-accrual method (ground grid: accrual raster; facades:
light-space accrual map), inputs resident on the device.  The per-step baselines (per-step
ray sweep, per-step raster) are timed on the same workload and reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload NAME]

Under torchrun (`--multi problems`, the default) every rank accumulates a district of its
own (the same distribution, its own seed): independent problems, no data collective, weak
scaling, value = all ranks' receiver-steps / the slowest rank's time.  `--multi shard`
splits one district's receivers instead (bands of grid rows, ranges of facade points; the
scene and its BVH on every rank) and gathers the results on rank 0: strong scaling, value
= the district's receiver-steps / the slowest rank's time.
`--impl reference` times the FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "receiver·sun-steps/s shadow-accumulated (accrual vs per-step sweep), 1 GB300"
UNIT = "receiver-steps/s"


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, path: str):
        self.path = path
        self.proc = None
        try:
            self.f = open(path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}",
                                          f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                                          "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1].split()[0]))
                smax.append(float(p[2].split()[0]))
            except ValueError:
                continue
            for n, v in zip(names[1:], p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------ multi-rank
def slowest_rank_ms(ms: float, dist=None, device=None) -> float:
    """Max of the per-rank step times over all ranks (the job is as slow as its slowest
    replica); ms itself when not distributed."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(units_per_rank: int, world: int, ms_max: float) -> float:
    """Whole-job throughput: every rank processes its own copy of the workload."""
    return world * units_per_rank / (ms_max * 1e-3)


# ------------------------------------------------------------------------ workload
def make_workload(name: str, rank: int = 0):
    """The named workload; under `--multi problems` rank r > 0 takes a district of its own
    (the same distribution, its own seed: an independent problem, not a copy)."""
    from synth import configs
    if name == "district":
        return configs.district(seed_off=2 + 1000 * rank) if rank else configs.district()
    if name == "district_1k":
        # the district's city with a 1024 x 1024 ground grid over its centre and 250k
        # facade samples: a quarter-size case for detailed profiles
        w = configs.district(n_facade=250_000)
        from synth.city import GroundGrid
        w.ground = GroundGrid(x0=512.0, y0=512.0, dx=1.0, nx=1024, ny=1024)
        return w
    if name == "district_small":
        return configs.district_small()
    if name == "boxes16":
        return configs.boxes16()
    raise SystemExit(f"unknown workload {name}")


def workload_config(args, w) -> dict:
    """The workload part of the JSON line's config, the same for both arms."""
    g = w.ground
    nf = 0 if w.facade_pos is None else int(w.facade_pos.shape[0])
    return {"workload": f"{args.workload}: {w.city.B} buildings, {w.mesh.T} triangles, "
                        f"{g.nx}x{g.ny} ground @ {g.dx} m + {nf} facade samples, {w.sun.S} sun steps",
            "receivers": int(w.R), "sun_steps": int(w.sun.S), "block_len": args.block_len or 60}


def cpu_oracle_sample(w, seconds_hint: float = 15.0, seed: int = 0):
    """Time the FP64 oracle on a bounded receiver sample of the workload (all steps)."""
    import oracle
    rng = np.random.default_rng(seed)
    t9, tb = w.mesh.tri9(), w.mesh.tri_building
    # calibrate on a small sample (after a warm-up call that loads the library and starts
    # its threads), then size the sample to ~seconds_hint of work
    pos_all = w.ground.positions() if w.ground is not None else None
    oracle.shadow_bits(t9, tb, pos_all[:16], None, w.sun.dirs)
    n_g = 512
    sel = rng.choice(pos_all.shape[0], n_g, replace=False)
    t0 = time.perf_counter()
    oracle.shadow_bits(t9, tb, pos_all[sel], None, w.sun.dirs)
    dt = max(time.perf_counter() - t0, 1e-3)
    per_rx = dt / n_g
    n_total = int(max(64, min(50_000, seconds_hint / per_rx)))
    R = w.R
    frac_f = (0 if w.facade_pos is None else w.facade_pos.shape[0]) / R
    n_f = int(round(n_total * frac_f))
    n_g = n_total - n_f
    sel_g = rng.choice(pos_all.shape[0], n_g, replace=False)
    t0 = time.perf_counter()
    oracle.shadow_bits(t9, tb, pos_all[sel_g], None, w.sun.dirs)
    if n_f:
        sel_f = rng.choice(w.facade_pos.shape[0], n_f, replace=False)
        oracle.shadow_bits(t9, tb, w.facade_pos[sel_f], w.facade_nrm[sel_f], w.sun.dirs)
    el = time.perf_counter() - t0
    value = (n_g + n_f) * w.sun.S / el
    return {"value": value, "unit": UNIT, "cores": oracle.default_threads(), "kind": "oracle",
            "sample": f"{n_g} ground + {n_f} facade receivers (seeded uniform sample) x all "
                      f"{w.sun.S} steps, FP64 brute force with per-building box pre-test",
            "seconds": el}


def cpu_oracle_configs(seconds_each: float = 4.0):
    """The FP64 oracle on the other workloads, each on a bounded seeded sample: the 16-box
    sweep case in full, the season (50,000 buildings; its first day), one batched variant
    (its region, the first day of the summer interval), and the park (all steps)."""
    import oracle
    from synth import configs
    rng = np.random.default_rng(5)
    out = {}

    cores = oracle.default_threads()

    def timed_sample(t9, tb, pos, dirs, label, full=False, steps_note="all"):
        # calibrate on two receivers per thread, then size the sample to ~seconds_each
        n = pos.shape[0] if full else min(pos.shape[0], 2 * cores)
        t0 = time.perf_counter()
        oracle.shadow_bits(t9, tb, pos[:n], None, dirs)
        dt = max(time.perf_counter() - t0, 1e-4)
        if not full:
            n = int(max(n, min(pos.shape[0], n * seconds_each / dt)))
            t0 = time.perf_counter()
            oracle.shadow_bits(t9, tb, pos[:n], None, dirs)
            dt = time.perf_counter() - t0
        return {"value": n * dirs.shape[0] / dt, "unit": UNIT, "cores": cores,
                "kind": "oracle", "seconds": dt,
                "sample": f"{n} {label} receivers x {steps_note} {dirs.shape[0]} steps"
                          + ("" if full else " (seeded uniform sample)")}

    def first_day(sun):
        return sun.dirs[int(sun.day_start[0]):int(sun.day_start[1])]

    w = configs.boxes16()
    out["boxes16"] = timed_sample(w.mesh.tri9(), w.mesh.tri_building, w.ground.positions(),
                                  w.sun.dirs, "ground (every cell)", full=True)
    w = configs.season()
    pos = w.ground.positions()[rng.choice(w.ground.R, 2000, replace=False)]
    out["season"] = timed_sample(w.mesh.tri9(), w.mesh.tri_building, pos, first_day(w.sun), "ground",
                                 steps_note="the first day's")
    sc = configs.scenarios(n_variants=1, days=31)
    t9, tb = sc.variant_mesh(0)
    ix0, iy0, nx, ny = (int(x) for x in sc.regions[0])
    gg = sc.base.ground
    loc = rng.choice(nx * ny, 2000, replace=False)
    pos = gg.positions()[(iy0 + loc // nx) * gg.nx + (ix0 + loc % nx)]
    out["batch_variant"] = timed_sample(t9, tb, pos, first_day(sc.intervals[1]), "variant-region ground",
                                        steps_note="the first day's")
    w = configs.park()
    pos = w.ground.positions()[rng.choice(w.ground.R, 20000, replace=False)]
    out["park"] = timed_sample(w.mesh.tri9(), w.mesh.tri_building, pos, w.sun.dirs, "park")
    return out


# ------------------------------------------------------------------------ GPU arm
def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_1907_04435_gb300 import binding as B

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    sharded = world > 1 and args.multi == "shard"
    w = make_workload(args.workload, rank if (world > 1 and not sharded) else 0)
    st = w.sun
    # resident inputs
    # the synthetic buildings are closed, outward-wound prisms
    scene = B.Scene(w.mesh.verts, w.mesh.tris, w.mesh.tri_building, w.city.B, closed=True)
    sun = B.Sun(st.dirs, st.day_start, args.block_len)
    g = w.ground
    if sharded:
        from paper_1907_04435_gb300 import shard
        bx0, by0, bdx, bnx, brows, _ = shard.grid_band((g.x0, g.y0, g.dx, g.nx, g.ny), rank, world)
        grid = B.Receivers.ground_grid(bx0, by0, bdx, bnx, brows)
        fa, fb = shard.split(0 if w.facade_pos is None else w.facade_pos.shape[0], rank, world)
        fac = B.Receivers.points(w.facade_pos[fa:fb], w.facade_nrm[fa:fb]) if fb > fa else None
    else:
        grid = B.Receivers.ground_grid(g.x0, g.y0, g.dx, g.nx, g.ny)
        fac = B.Receivers.points(w.facade_pos, w.facade_nrm) if w.facade_pos is not None else None
    R = grid.R + (fac.R if fac else 0)
    units = R * st.S
    job_units = w.R * st.S if sharded else world * units
    out_g = [torch.zeros(grid.R, dtype=torch.int32, device=dev),
             torch.empty(grid.R, dtype=torch.float32, device=dev),
             torch.zeros(grid.R, dtype=torch.int32, device=dev)]
    out_f = ([torch.zeros(fac.R, dtype=torch.int32, device=dev),
              torch.empty(fac.R, dtype=torch.float32, device=dev),
              torch.zeros(fac.R, dtype=torch.int32, device=dev)] if fac else None)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(method_ground, method_fac, ev=None):
        if ev is not None:
            ev[0].record(stream)
        B.sa_accumulate(scene, grid, sun, st.step_minutes, method_ground,
                        gross=out_g[0], minutes=out_g[1], continuous=out_g[2])
        if ev is not None:
            ev[1].record(stream)
        if fac:
            B.sa_accumulate(scene, fac, sun, st.step_minutes, method_fac,
                            gross=out_f[0], minutes=out_f[1], continuous=out_f[2])
        if ev is not None:
            ev[2].record(stream)

    def timed(method_ground, method_fac, steps, warmup, kernel_times=None, median=False):
        """Mean (or median) ms per step (whole step, ground call, facade call).  With
        kernel_times (a dict) the library also times each launch of its main kernels on the
        stream it launches on, and the per-class (total ms, launches) of the timed steps
        land there."""
        for _ in range(warmup):
            step(method_ground, method_fac)
        torch.cuda.synchronize()
        if kernel_times is not None:
            B.sa_kernel_times()
            B.sa_set_option(B.SA_OPT_KERNEL_TIMING, 1)
        tot, tg, tf = [], [], []
        for _ in range(steps):
            flush.fill_(1.0)                     # evict L2 between timed iterations
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            step(method_ground, method_fac, ev)
            torch.cuda.synchronize()
            tg.append(ev[0].elapsed_time(ev[1]))
            tf.append(ev[1].elapsed_time(ev[2]))
            tot.append(ev[0].elapsed_time(ev[2]))
        if kernel_times is not None:
            B.sa_set_option(B.SA_OPT_KERNEL_TIMING, 0)
            kernel_times.update(B.sa_kernel_times())
        f = statistics.median if median else statistics.fmean
        return f(tot), f(tg), f(tf)

    if args.only_step:
        # profiling mode: W warm-up steps and K timed steps of one method only
        ms, ms_g, ms_f = timed(args.method, args.method, args.steps, args.warmup)
        if rank == 0:
            print(json.dumps({"only_step": True, "workload": args.workload, "method": args.method,
                              "ms_per_step": ms, "ground_ms": ms_g, "facade_ms": ms_f}))
        return

    # ---- headline: shadow accrual (ground accrual raster + facade ray-traced accrual)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    csv_dir = args.clocks_dir or tempfile.gettempdir()
    clocks = ClockSampler(local, os.path.join(csv_dir, f"clocks_rank{rank}.csv"))
    ktimes = {}
    ms, ms_g, ms_f = timed("accrual_sam", "accrual_sam", args.steps, args.warmup, ktimes)
    clk = clocks.stop()
    torch.cuda.synchronize()
    if world > 1:
        ms = slowest_rank_ms(ms, dist, dev)
        dist.barrier()
    value = job_units / (ms * 1e-3)
    gathered = None
    if sharded:
        from paper_1907_04435_gb300 import shard
        parts = [t.cpu().numpy() for t in out_g] + ([t.cpu().numpy() for t in out_f] if fac else
                                                    [np.zeros(0, np.int32), np.zeros(0, np.float32),
                                                     np.zeros(0, np.int32)])
        got = shard.gather_to_root(parts, dist)
        if rank == 0:
            gathered = {"ground_receivers": int(got[0].size), "facade_receivers": int(got[3].size),
                        "gross_sum": int(got[0].sum()) + int(got[3].sum())}

    # ---- per-step baselines and the other exact method on the same workload
    methods = {"accrual_sam": {"ms": ms, "ground_ms": ms_g, "facade_ms": ms_f,
                               "value": units / (ms * 1e-3)}}
    if not args.skip_baselines:
        for mg, mf, name in (("accrual_trace", "accrual_trace", "accrual_trace"),
                             ("sweep_raster", "sweep_trace", "sweep_raster+sweep_trace"),
                             ("sweep_trace", "sweep_trace", "sweep_trace")):
            m_ms, m_g, m_f = timed(mg, mf, args.baseline_steps, 1, median=True)
            methods[name] = {"ms": m_ms, "ground_ms": m_g, "facade_ms": m_f,
                             "value": units / (m_ms * 1e-3),
                             "timing": f"median of {args.baseline_steps} steps after 1 warm-up"}
        sweep = methods["sweep_trace"]["value"]
        for v in methods.values():
            v["speedup_vs_sweep_trace"] = v["value"] / sweep
        # the inverse accrual map (approximate, ground receivers only: Sec. 5) beside the
        # exact methods' ground calls
        gsteps = grid.R * st.S
        iam_ms = _event_ms(lambda: B.sa_accumulate(scene, grid, sun, st.step_minutes, "iam",
                                                   gross=out_g[0], minutes=out_g[1],
                                                   continuous=out_g[2]), 3)
        methods["iam_ground_only"] = {
            "ground_ms": iam_ms, "ground_value": gsteps / (iam_ms * 1e-3),
            "note": "approximate (3 source levels, 1 m acne rule); accuracy in the IAM tests",
            "speedup_vs_sweep_trace_ground": methods["sweep_trace"]["ground_ms"] / iam_ms}

    # ---- roofline of the dominant kernel (instrumented work counters)
    roof, roof_all = roofline(B, scene, grid, fac, sun, ktimes, args.steps, args.workload)

    # ---- end to end through the C ABI from host buffers (a rank's own district; the split
    # mode reports its device-timed value only)
    e2e = (end_to_end(B, w, args, dev) if not sharded else
           {"value": None, "unit": UNIT, "note": "not measured when one district is split"})

    # ---- batched scenarios (development variants x seasonal intervals)
    batch = None if args.skip_batch else bench_batch(B, w, args)

    # ---- the other workloads (small sweep case, season, height gradient)
    other = None if (args.skip_configs or world > 1) else bench_configs(B)

    # ---- analysis measures over the central 1024 x 1024 m of the district (Sec. 7.2)
    analysis = None
    if not args.skip_configs and world == 1:
        gross, _, _ = B.sa_accumulate(scene, grid, sun, st.step_minutes, "accrual_sam")
        xa, ya = g.x0 + 512 * g.dx, g.y0 + 512 * g.dx
        xb, yb = xa + 1024 * g.dx, ya + 1024 * g.dx
        poly = np.array([[xa, ya], [xb, ya], [xb, yb], [xa, yb]], np.float32)
        area_ms = _event_ms(lambda: B.sa_shadow_area(grid, gross, st.S, poly), 5)
        contrib_ms = _event_ms(lambda: B.sa_building_contribution(scene, grid, sun, poly), 3)
        casting, nearest, stats = B.sa_building_contribution(scene, grid, sun, poly)
        analysis = {"region": "central 1024 x 1024 cells of the ground grid",
                    "shadow_area_ms": area_ms, "shadow_area_m2": B.sa_shadow_area(grid, gross, st.S, poly),
                    "building_contribution_ms": contrib_ms,
                    "buildings_casting": int((casting > 0).sum()),
                    "nearest_sum_m2": float(nearest.sum()), "unattributed_cell_steps": stats[1]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong" if sharded else "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(workload_config(args, w),
                           method="accrual_sam: ground accrual raster + facade light-space accrual map",
                           l2="flushed (256 MB write) before every timed iteration",
                           parallelism=(f"receivers split over {world} ranks, gathered on rank 0"
                                        if sharded else f"independent districts x{world}"
                                        if world > 1 else "one GPU")),
            "methods": methods,
            "roofline": roof,
            "roofline_kernels": roof_all,
            "e2e": e2e,
            "gpu_launches": count_launches(scene, sun, grid, fac),
            "gathered": gathered,
            "batch": batch,
            "other_workloads": other,
            "analysis": analysis,
            "clocks": clk,
        }
        if world == 1 and not args.skip_cpu:
            line["cpu_baseline"] = cpu_oracle_sample(w, args.cpu_seconds)
            if not args.skip_configs:
                line["cpu_baseline_other_workloads"] = cpu_oracle_configs()
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def count_launches(scene, sun, grid, fac):
    """Kernels of one timed step.  Ground raster, per chunk of <= 64 blocks: bin count,
    tile order, 3 scan kernels, bin fill, raster.  Facade map, per chunk of blocks (<= 64, and bins of
    <= 1 GiB at 4 bytes per receiver and run plus 8 per receiver and block): triangle and
    receiver bin counts, 2 x 3 scan kernels, 3 kernels ordering the tiles by work, the two
    fills, the tile kernel and the fold."""
    chunks = (sun.n_blocks + 63) // 64
    n = chunks * 7
    if fac:
        run = min(32, max(1, B_option_run()))   # steps per light-space map
        per_block = fac.R * (4 * ((64 + run - 1) // run) + 8)
        fchunk = max(1, min(64, (1 << 30) // max(1, per_block)))
        n += 15 * ((sun.n_blocks + fchunk - 1) // fchunk)
    return n


def B_option_run():
    from paper_1907_04435_gb300 import binding as B
    return B.sa_get_option(B.SA_OPT_POINT_RUN)


# Algorithmic FP32 operations per unit of work (the method's own work, counted by the
# library's instrumented counters): in the ground raster a cell set-up (P, Q_x and Q_y of
# three edges from the triangle's affine edge constants, 4 FMAs each) 12 and a cell-step
# coverage test (three edge evaluations and compares) 9; in the light-space
# map of facades a receiver-triangle set-up (three Plücker edge moments, normal, distance)
# 55 and a step test (three dot products, distance check) 15; in the ray-traced methods a
# box test 12 and a watertight triangle test 25.
OPS_CELL, OPS_TEST = 12, 9
OPS_PAIR, OPS_PTEST = 55, 15
OPS_BOX, OPS_TRI = 12, 25

# DRAM bytes (read + write) of one launch of each hot kernel on the `district` workload,
# from one ncu capture of `dram__bytes_read.sum,dram__bytes_write.sum` (the launch list's
# profile summary gives the command).  A figure is reported only while the kernel's
# sources hash to the value they had when it was captured; otherwise traffic is null.
TRAFFIC = {
    "k_raster": {"bytes": 7002880 + 14976768, "workload": "district",
                 "sources": ("sa_raster.cu", "sa_internal.cuh"), "sha256_16": "fbe5e1cde17ff661"},
    "k_sam_tile": {"bytes": 155689216 + 26193152, "workload": "district",
                   "sources": ("sa_sam_points.cu", "sa_internal.cuh", "sa_handles.cuh"),
                   "sha256_16": "e9ff7eeb4764c3a4"},
}


def kernel_traffic(name: str, workload: str):
    import hashlib
    t = TRAFFIC.get(name)
    if t is None or t["workload"] != workload:
        return None
    m = hashlib.sha256()
    for f in t["sources"]:
        with open(os.path.join(ROOT, "paper_1907_04435_gb300", "csrc", f), "rb") as fh:
            m.update(fh.read())
    return t["bytes"] if m.hexdigest()[:16] == t["sha256_16"] else None


def roofline(B, scene, grid, fac, sun, ktimes, steps, workload):
    """ALU rooflines of the two hot kernels of a step: achieved = counted algorithmic FP32
    ops per launch / the kernel's mean launch duration, both from the timed region (CUDA
    events the library records around each launch, on its launching stream); peak = 152
    SMs x 128 FP32 lanes x the maximum SM clock (one op per lane per clock)."""
    peaks, src = load_peaks()
    clk = peaks.get("sm_max_mhz", 2070.0) * 1e6
    peak_ops = 152 * 128 * clk
    out = {}

    def entry(name, desc, ops_step, cls, work):
        t_ms, n = ktimes.get(cls, (0.0, 0))
        per_step = n / steps
        launch_ms = t_ms / n
        ops_launch = ops_step / per_step
        ach = ops_launch / (launch_ms * 1e-3)
        out[name] = {"bound": "alu", "kernel": desc, "achieved": ach / 1e12,
                     "peak": peak_ops / 1e12, "unit": "Tops/s", "frac": ach / peak_ops,
                     "traffic": kernel_traffic(name, workload), "traffic_unit": "bytes per launch",
                     "launches_per_step": per_step,
                     "mean_launch_ms": launch_ms, "kernel_ms_per_step": t_ms / steps,
                     "ops_per_launch": ops_launch, "work": work}

    c = B.sa_work_counters(scene, grid, sun, "accrual_sam")
    entry("k_raster", "k_raster (ground accrual raster)", c[2] * OPS_CELL + c[3] * OPS_TEST,
          "raster", {"cell_setups": c[2], "cell_step_tests": c[3],
                     "ops_per_setup": OPS_CELL, "ops_per_test": OPS_TEST,
                     "work_units": c[0], "cells_enumerated": c[1]})
    if fac is not None:
        c = B.sa_work_counters(scene, fac, sun, "accrual_sam")
        entry("k_sam_tile", "k_sam_tile (facade light-space accrual map)",
              c[0] * OPS_PAIR + c[1] * OPS_PTEST, "sam_points",
              {"pair_setups": c[0], "step_tests": c[1],
               "ops_per_setup": OPS_PAIR, "ops_per_test": OPS_PTEST})
    dom = max(out, key=lambda k: out[k]["kernel_ms_per_step"])
    head = dict(out[dom])
    head["peak_source"] = (f"152 SMs x 128 FP32 lanes x {clk / 1e6:.0f} MHz "
                           f"(sm_max_mhz, {src})")
    return head, out


def bench_batch(B, w, args):
    """Development variants of the district (towers added, overlapped buildings removed)
    x 4 seasonal intervals of 31 days, each variant on its own receiver region: one
    graph-captured persistent launch (sa_batch_run) against per-scenario scene builds and
    accumulations.  The first --batch-variants of the 64 variants are timed (each arm over
    the same ones); the receiver-steps of all 64 are reported beside them.  Two batched
    times separate the batch's two gains: with the tiles no changed building can shadow
    kept at the base counts (the default), and with every tile rastered."""
    import torch
    from synth import configs
    import copy
    full = configs.scenarios(n_variants=64, days=args.batch_days, base=w)
    V = min(args.batch_variants, full.V)
    sc = copy.copy(full)
    sc.tower_tris, sc.removed, sc.regions = full.tower_tris[:V], full.removed[:V], full.regions[:V]
    st0 = sc.intervals
    scene = B.Scene(w.mesh.verts, w.mesh.tris, w.mesh.tri_building, w.city.B, closed=True)
    g = w.ground
    grid = B.Receivers.ground_grid(g.x0, g.y0, g.dx, g.nx, g.ny)
    suns = [B.Sun(it.dirs, it.day_start) for it in st0]
    area = lambda regions: int((regions[:, 2] * regions[:, 3]).sum())
    units = int(sum(area(sc.regions) * it.S for it in st0))
    units_all = int(sum(area(full.regions) * it.S for it in full.intervals))

    def batched(skip):
        B.sa_set_option(B.SA_OPT_BATCH_TILE_SKIP, 1 if skip else 0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bt = B.Batch(scene, grid, sc.tower_tris, sc.removed, sc.regions, suns, with_impact=True)
        torch.cuda.synchronize()
        setup = time.perf_counter() - t0
        B.sa_set_option(B.SA_OPT_BATCH_TILE_SKIP, 1)
        tuned = bt.tune()
        counts, impact = bt.run()
        ms = _event_ms(lambda: bt.run(counts, impact), 2)
        return bt, ms, setup, tuned, counts

    bt, batch_ms, setup_s, (ctas, run), counts = batched(True)
    items, affected = bt.n_items, bt.n_affected
    del bt
    bt2, noskip_ms, _, _, counts2 = batched(False)
    if not torch.equal(counts, counts2):
        raise RuntimeError("batched counts depend on the tile skipping")
    del bt2, counts, counts2
    # per-scenario launches: each variant's mesh is built on the host first (not timed);
    # the timer covers its upload, LBVH build and one accumulation per interval on its region
    meshes = []
    for v in range(V):
        t9, tb = sc.variant_mesh(v)
        verts = np.ascontiguousarray(t9.reshape(-1, 3))
        meshes.append((verts, np.arange(verts.shape[0], dtype=np.int32).reshape(-1, 3), tb))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for v in range(V):
        verts, tris, tb = meshes[v]
        vs = B.Scene(verts, tris, tb, int(tb.max()) + 1, closed=True)
        ix0, iy0, nx, ny = (int(x) for x in sc.regions[v])
        rg = B.Receivers.ground_grid(g.x0 + ix0 * g.dx, g.y0 + iy0 * g.dx, g.dx, nx, ny)
        for s in suns:
            B.sa_accumulate(vs, rg, s, 1.0, "accrual_sam", want_minutes=False, want_continuous=False)
    torch.cuda.synchronize()
    per_ms = (time.perf_counter() - t0) * 1e3
    return {"workload": f"the first {V} of 64 variants x {len(st0)} intervals of {args.batch_days} "
                        f"days (09-17 h @ 1 min) on district regions of 256..2048 cells a side",
            "receiver_steps": units, "receiver_steps_all_64_variants": units_all,
            "items": items, "items_rastered": affected,
            "tuned": {"ctas": ctas, "run": run},
            "batched_ms": batch_ms, "batched_value": units / (batch_ms * 1e-3),
            "batch_setup_s": setup_s, "batched_with_setup_ms": batch_ms + 1e3 * setup_s,
            "batched_every_tile_ms": noskip_ms,
            "per_scenario_ms": per_ms, "per_scenario_value": units / (per_ms * 1e-3),
            "speedup": per_ms / batch_ms,
            "speedup_with_setup": per_ms / (batch_ms + 1e3 * setup_s),
            "gain_from_tile_skipping": noskip_ms / batch_ms,
            "gain_from_one_launch": per_ms / noskip_ms,
            "batched_ms_scaled_to_64_variants": batch_ms * units_all / units,
            "per_scenario_ms_scaled_to_64_variants": per_ms * units_all / units,
            "unit": UNIT}


def _event_ms(fn, reps: int) -> float:
    """Median CUDA-event time of fn() over reps runs (after one warm-up)."""
    import torch
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def bench_configs(B):
    """The other workloads of the method, each in its own terms: the small sweep case
    (16 boxes, 64^2 cells, 241 steps), the season (50,000 buildings, 4096^2 cells, 92 days)
    and the height gradient over the park (600k cells, 200 buildings, one day)."""
    import torch
    from synth import configs
    out = {}
    # 16 boxes: accrual map against both per-step sweeps (launch-bound at this size)
    w = configs.boxes16()
    g = w.ground
    scene = B.Scene(w.mesh.verts, w.mesh.tris, w.mesh.tri_building, w.city.B, closed=True)
    sun = B.Sun(w.sun.dirs, w.sun.day_start)
    grid = B.Receivers.ground_grid(g.x0, g.y0, g.dx, g.nx, g.ny)
    units = g.R * w.sun.S
    c1 = {"workload": f"16 boxes, {g.nx}x{g.ny} ground @ {g.dx} m, {w.sun.S} steps",
          "receiver_steps": units}
    for m in ("accrual_sam", "accrual_trace", "sweep_raster", "sweep_trace"):
        ms = _event_ms(lambda: B.sa_accumulate(scene, grid, sun, w.sun.step_minutes, m), 5)
        c1[m] = {"ms": ms, "value": units / (ms * 1e-3)}
    out["boxes16"] = c1
    # season: ground accrual raster over 92 days
    w = configs.season()
    g = w.ground
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    scene = B.Scene(w.mesh.verts, w.mesh.tris, w.mesh.tri_building, w.city.B, closed=True)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    sun = B.Sun(w.sun.dirs, w.sun.day_start)
    grid = B.Receivers.ground_grid(g.x0, g.y0, g.dx, g.nx, g.ny)
    units = g.R * w.sun.S
    ms = _event_ms(lambda: B.sa_accumulate(scene, grid, sun, w.sun.step_minutes, "accrual_sam"), 2)
    out["season"] = {"workload": f"{w.city.B} buildings, {w.mesh.T} triangles, {g.nx}x{g.ny} "
                                 f"ground @ {g.dx} m, {w.sun.D} days x 481 steps ({w.sun.S})",
                     "receiver_steps": units, "accrual_sam_ms": ms,
                     "value": units / (ms * 1e-3), "scene_build_s": build_s, "unit": UNIT}
    # the same season through the direction graph (5 degree bins, approximate): its time,
    # the maps it computes against the exact path's blocks, and its error
    ge, _, ce = B.sa_accumulate(scene, grid, sun, w.sun.step_minutes, "accrual_sam")
    gg, _, cg, n_edges = B.sa_accumulate_graph(scene, grid, sun, w.sun.step_minutes, "accrual_sam", 5.0)
    ge, gg = ge.double(), gg.double()
    gms = _event_ms(lambda: B.sa_accumulate_graph(scene, grid, sun, w.sun.step_minutes, "accrual_sam", 5.0), 2)
    out["season"]["direction_graph"] = {
        "bin_deg": 5.0, "maps": n_edges, "blocks": sun.n_blocks, "ms": gms,
        "speedup_over_exact": ms / gms,
        "gross_error_pct": float(100.0 * (gg - ge).abs().sum() / ge.sum()),
        "gross_area_change_pct": float(100.0 * (gg.sum() - ge.sum()) / ge.sum()),
        "continuous_mean_abs_steps": float((cg - ce).double().abs().mean())}
    del ge, gg, ce, cg
    del scene, grid
    # park: forward accrual and the height gradient (forward masks + FP64 flip refinement)
    w = configs.park()
    g = w.ground
    scene = B.Scene.from_footprints(w.city.footprints, w.city.heights, w.city.band_height)
    sun = B.Sun(w.sun.dirs, w.sun.day_start)
    grid = B.Receivers.ground_grid(g.x0, g.y0, g.dx, g.nx, g.ny)
    fwd = _event_ms(lambda: B.sa_accumulate(scene, grid, sun, w.sun.step_minutes, "accrual_sam"), 5)
    grad = _event_ms(lambda: B.sa_height_grad(scene, grid, sun, w.sun.step_minutes), 5)
    out["park_adjoint"] = {"workload": f"{g.nx}x{g.ny} park cells @ {g.dx} m, {w.city.B} buildings, "
                                       f"{w.sun.S} steps",
                           "forward_ms": fwd, "gradient_ms": grad,
                           "gradient_over_forward": grad / fwd}
    return out


def end_to_end(B, w, args, dev):
    """Same metric through the C ABI from pinned host buffers: every step copies the mesh,
    the sun table and the facade points to the device, builds the scene and its BVH, the
    sun table and the sorted receivers, accumulates, and copies the results back to pinned
    host memory.  Two worker threads, started once like the streams, build the sun table
    and sort the facade receivers on streams of their own while this thread builds the
    scene; the facades accumulate on a second stream, overlapping the ground's
    accumulation and its copy back.  Measured twice: each step alone between device
    synchronisations (`one_step`), and steps back to back with the next step's inputs
    built while the current one accumulates (the reported value)."""
    import concurrent.futures as cf

    import torch

    def pinned(a):
        return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()

    st = w.sun
    g = w.ground
    verts, tris, tb = pinned(w.mesh.verts), pinned(w.mesh.tris), pinned(w.mesh.tri_building)
    dirs, day_start = pinned(st.dirs), pinned(st.day_start)
    fpos = None if w.facade_pos is None else pinned(w.facade_pos)
    fnrm = None if w.facade_nrm is None else pinned(w.facade_nrm)
    R = g.R + (0 if fpos is None else fpos.shape[0])
    host_out = torch.empty(3 * R, dtype=torch.int32).pin_memory()
    nbytes = lambda t: 0 if t is None else t.numel() * t.element_size()
    h2d = sum(nbytes(t) for t in (verts, tris, tb, dirs, day_start, fpos, fnrm))
    d2h = 3 * R * 4

    # the scene build and the ground run on a high-priority stream: the build is a chain of
    # small kernels, and the facade sort's wide kernels on the second stream would
    # otherwise hold the SMs it waits for
    main = torch.cuda.Stream(priority=-1)
    side = torch.cuda.Stream()
    sun_stream = torch.cuda.Stream()
    Rg = g.R
    pool = cf.ThreadPoolExecutor(max_workers=2)

    def once():
        # The library's creation calls wait for their own stream before they return, and
        # ctypes lets the other threads run meanwhile: the sun table and the sorted facade
        # receivers are ready on the device once their futures resolve.  The ground
        # accumulates on the high-priority stream, the facades on the second one once the
        # scene exists; each part's results go straight to its slice of the pinned output
        # (gross | minutes | continuous, ground then facades), the ground's while the
        # facades still run.
        sun_f = pool.submit(B.Sun, dirs, day_start, args.block_len, stream=sun_stream)
        fac_f = None if fpos is None else pool.submit(B.Receivers.points, fpos, fnrm, stream=side)
        with torch.cuda.stream(main):
            scene = B.Scene(verts, tris, tb, w.city.B, closed=True, stream=main)
            grid = B.Receivers.ground_grid(g.x0, g.y0, g.dx, g.nx, g.ny)
            ready = main.record_event()
            sun = sun_f.result()
            gg, gm, gc = B.sa_accumulate(scene, grid, sun, st.step_minutes, "accrual_sam", stream=main)
            for q, t in enumerate((gg, gm.view(torch.int32), gc)):
                host_out[q * R:q * R + Rg].copy_(t, non_blocking=True)
        if fac_f is not None:
            fac = fac_f.result()
            side.wait_event(ready)
            with torch.cuda.stream(side):
                fg, fm, fc = B.sa_accumulate(scene, fac, sun, st.step_minutes, "accrual_sam", stream=side)
                for q, t in enumerate((fg, fm.view(torch.int32), fc)):
                    host_out[q * R + Rg:(q + 1) * R].copy_(t, non_blocking=True)
        torch.cuda.synchronize()

    once()
    times = []
    for _ in range(5):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        once()
        times.append(time.perf_counter() - t0)
    t_one = statistics.median(times)
    # the overlapped results equal a sequential run on one stream, bit for bit
    scene = B.Scene(verts, tris, tb, w.city.B, closed=True)
    sun = B.Sun(dirs, day_start, args.block_len)
    grid = B.Receivers.ground_grid(g.x0, g.y0, g.dx, g.nx, g.ny)
    parts = [list(B.sa_accumulate(scene, grid, sun, st.step_minutes, "accrual_sam"))]
    if fpos is not None:
        fac = B.Receivers.points(fpos, fnrm)
        parts.append(list(B.sa_accumulate(scene, fac, sun, st.step_minutes, "accrual_sam")))
    want = torch.cat([torch.cat([p[q].view(torch.int32) for p in parts]) for q in range(3)]).cpu()
    del scene, sun, grid, parts
    if not torch.equal(want, host_out):
        raise RuntimeError("end-to-end results differ from a sequential run")

    # Steps back to back, as a serving loop runs them: a builder thread uploads and builds
    # step i + 1's scene (on its own high-priority stream), sun table and sorted facade
    # receivers while step i accumulates; each step still copies its inputs from pinned
    # host memory and its results back to a pinned buffer of its own.  The handles are kept
    # until the end (destroying one synchronises the device).
    build_stream = torch.cuda.Stream(priority=-1)
    builder = cf.ThreadPoolExecutor(max_workers=1)
    n_steps = 10
    outs = [torch.empty(3 * R, dtype=torch.int32).pin_memory() for _ in range(n_steps + 1)]

    def build():
        sun_f = pool.submit(B.Sun, dirs, day_start, args.block_len, stream=sun_stream)
        fac_f = None if fpos is None else pool.submit(B.Receivers.points, fpos, fnrm, stream=side)
        with torch.cuda.stream(build_stream):
            scene = B.Scene(verts, tris, tb, w.city.B, closed=True, stream=build_stream)
        return scene, sun_f.result(), None if fac_f is None else fac_f.result()

    def accumulate(inputs, out):
        scene, sun, fac = inputs
        grid = B.Receivers.ground_grid(g.x0, g.y0, g.dx, g.nx, g.ny)
        with torch.cuda.stream(main):
            gg, gm, gc = B.sa_accumulate(scene, grid, sun, st.step_minutes, "accrual_sam", stream=main)
            for q, t in enumerate((gg, gm.view(torch.int32), gc)):
                out[q * R:q * R + Rg].copy_(t, non_blocking=True)
        if fac is not None:
            with torch.cuda.stream(acc_side):
                fg, fm, fc = B.sa_accumulate(scene, fac, sun, st.step_minutes, "accrual_sam", stream=acc_side)
                for q, t in enumerate((fg, fm.view(torch.int32), fc)):
                    out[q * R + Rg:(q + 1) * R].copy_(t, non_blocking=True)

    acc_side = torch.cuda.Stream()
    keep = []

    def pipeline(n, bufs):
        nxt = builder.submit(build)
        for i in range(n):
            cur = nxt.result()
            keep.append(cur)
            if i + 1 < n:
                nxt = builder.submit(build)
            accumulate(cur, bufs[i])
        torch.cuda.synchronize()

    pipeline(1, outs[n_steps:])                     # warm-up
    runs = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pipeline(n_steps, outs)
        runs.append((time.perf_counter() - t0) / n_steps)
        keep.clear()
    t_pipe = statistics.median(runs)
    builder.shutdown()
    pool.shutdown()
    keep.clear()
    for i, o in enumerate(outs):
        if not torch.equal(want, o):
            raise RuntimeError(f"pipelined end-to-end step {i} differs from a sequential run")
    return {"value": R * st.S / t_pipe, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "seconds_per_step": t_pipe,
            "pipelined": f"{n_steps} steps back to back, each step's inputs built while the previous one "
                         "accumulates; median of 3 such runs",
            "one_step": {"value": R * st.S / t_one, "seconds_per_step": t_one,
                         "timing": "median of 5 steps, each alone between device synchronisations"}}


# ------------------------------------------------------------------------ reference arm
def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = make_workload(args.workload)
    import oracle
    # each step is a seeded receiver sample sized so that the whole run takes about
    # 150 s of oracle work, at most cpu_seconds / 2 per step
    per_step = max(0.5, min(args.cpu_seconds / 2, 150.0 / (args.steps + 0.5 * args.warmup)))
    vals = []
    for _ in range(args.warmup):
        cpu_oracle_sample(w, per_step / 2)
    for k in range(args.steps):
        vals.append(cpu_oracle_sample(w, per_step, seed=k))
    value = statistics.median([v["value"] for v in vals])
    s = vals[0]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.median([v["seconds"] for v in vals]) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": dict(workload_config(args, w), method="FP64 oracle on a seeded receiver sample",
                           sample=s["sample"]),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.default_threads(),
                             "kind": "oracle", "sample": s["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_only_graph(args):
    """Profiling mode for the direction graph: the season's city and sun (92 days) over a
    smaller central ground grid (--graph-n cells a side), accumulated through the graph with
    5 degree bins after W warm-up runs, K timed runs; prints one JSON line."""
    import torch

    from paper_1907_04435_gb300 import binding as B
    from synth import configs
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    w = configs.season(ground_n=args.graph_n)
    g = w.ground
    scene = B.Scene(w.mesh.verts, w.mesh.tris, w.mesh.tri_building, w.city.B, closed=True)
    sun = B.Sun(w.sun.dirs, w.sun.day_start)
    grid = B.Receivers.ground_grid(g.x0, g.y0, g.dx, g.nx, g.ny)
    run = lambda: B.sa_accumulate_graph(scene, grid, sun, w.sun.step_minutes, "accrual_sam", 5.0)
    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize()
    ts, maps = [], 0
    B.sa_kernel_times()
    B.sa_set_option(B.SA_OPT_KERNEL_TIMING, 1)
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        maps = run()[3]
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    B.sa_set_option(B.SA_OPT_KERNEL_TIMING, 0)
    kt = {k: {"ms_per_run": v[0] / args.steps, "launches_per_run": v[1] / args.steps}
          for k, v in B.sa_kernel_times().items() if v[1]}
    print(json.dumps({"only_graph": True, "workload": f"season city, {g.nx}x{g.ny} ground @ {g.dx} m, "
                      f"{w.sun.D} days ({w.sun.S} steps)", "maps": maps, "blocks": sun.n_blocks,
                      "ms": statistics.median(ts), "kernel_times": kt}))


def run_only_contrib(args):
    """Profiling mode for the building contribution (Sec. 7.2): the district's scene and
    sun, a square region of --contrib-n cells a side at the grid's centre; W warm-up and K
    timed calls; prints one JSON line."""
    import torch

    from paper_1907_04435_gb300 import binding as B
    from synth import configs
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    w = configs.district(n_facade=0)
    g = w.ground
    scene = B.Scene(w.mesh.verts, w.mesh.tris, w.mesh.tri_building, w.city.B, closed=True)
    sun = B.Sun(w.sun.dirs, w.sun.day_start)
    grid = B.Receivers.ground_grid(g.x0, g.y0, g.dx, g.nx, g.ny)
    n = args.contrib_n
    xa, ya = g.x0 + (g.nx - n) // 2 * g.dx, g.y0 + (g.ny - n) // 2 * g.dx
    poly = np.array([[xa, ya], [xa + n * g.dx, ya], [xa + n * g.dx, ya + n * g.dx], [xa, ya + n * g.dx]],
                    np.float32)
    run = lambda: B.sa_building_contribution(scene, grid, sun, poly)
    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize()
    ts = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    print(json.dumps({"only_contrib": True, "region": f"{n}x{n} cells at the district grid's centre",
                      "ms": statistics.median(ts)}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="district")
    ap.add_argument("--block-len", dest="block_len", type=int, default=0)
    ap.add_argument("--skip-baselines", action="store_true")
    ap.add_argument("--only-step", action="store_true",
                    help="time one method only (for profiler runs); prints one JSON line")
    ap.add_argument("--method", default="accrual_sam",
                    choices=["accrual_sam", "accrual_trace", "sweep_trace"],
                    help="the method --only-step times (ground and facades)")
    ap.add_argument("--only-graph", action="store_true",
                    help="time the direction graph over the season's sun only (for profiler runs)")
    ap.add_argument("--graph-n", dest="graph_n", type=int, default=1024,
                    help="ground cells a side for --only-graph")
    ap.add_argument("--clocks-dir", dest="clocks_dir", default=None,
                    help="folder for the raw nvidia-smi clock samples (default: the temp folder)")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-batch", action="store_true")
    ap.add_argument("--skip-configs", action="store_true",
                    help="skip the small-sweep, season and height-gradient workloads")
    ap.add_argument("--batch-variants", type=int, default=8)
    ap.add_argument("--batch-days", type=int, default=31)
    ap.add_argument("--baseline-steps", dest="baseline_steps", type=int, default=5)
    ap.add_argument("--only-contrib", dest="only_contrib", action="store_true",
                    help="profiling mode: the building contribution over a central region")
    ap.add_argument("--contrib-n", dest="contrib_n", type=int, default=1024)
    ap.add_argument("--multi", default="problems", choices=["problems", "shard"],
                    help="under torchrun: a district per rank (weak) or one district split (strong)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.only_graph:
        run_only_graph(args)
    elif args.only_contrib:
        run_only_contrib(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
