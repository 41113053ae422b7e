#!/usr/bin/env python3
"""Benchmark of the CGA hot path (libcga) on GB300.

Default workload (--config surface; one "step" = one pass of the whole hot
path): 30M float32 points sampled on the surfaces of 200 seeded
superellipsoids in a 100 m cube, on a 12-bit-per-axis grid (24.4 mm voxels):
  build    the even- and odd-index halves (15M points each) in one batched call
  merge    the two half CGAs (Eq. 1)
  project  the merged CGA onto the xy, xz and yz planes (Eq. 3)
  nn       8,000,000 exact NN queries (4M fresh surface samples + 4M uniform
           in the box): the search structure of the merged CGA (the
           strategy cga_nn_autotune picked before timing), the Morton query
           sort, then the search (Eq. 7-8)
  decode   the merged CGA back to voxel triples
Inputs are resident in HBM before the timed region; L2 (129 MB) is flushed
between timed steps by writing a 512 MB buffer.

Other workloads: --config lidar (10 LiDAR sweeps, 1.31M points, b = 16, 1M
jittered queries), plain (100k uniform + twin), batched (512 uneven clouds
through the pre-planned pipeline replayed from a CUDA graph, against 512
sequential plain calls), served (requests over 64 resident CGAs), and the
rows after the hot path: values, perspective, search, compress.

python bench.py [--gpus N --steps K --warmup W] [--config C] [--impl reference]
prints ONE JSON line.  --impl reference times the CPU oracle on the host cores
on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
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

from paper_2110_11616_gb300 import synth  # noqa: E402

METRIC = "CGA build Mpts/s, NN queries/s, merge GB/s vs HBM peak; batched vs plain"
WORKLOAD = ("surface: 30M pts on 200 superellipsoids in a 100 m cube, b=12; batched build of the "
            "even/odd halves, merge, xy/xz/yz projections, NN search structure + Morton sort + "
            "8M exact NN (4M on-surface + 4M uniform), decode")
WORKLOAD_LIDAR = ("LiDAR frame set: 10 sweeps x 64 beams x 2048 azimuth (1,310,720 pts), b=16, "
                  "batched build (ego pose fused) + 9-merge tree (batched per level) + xy "
                  "projection + 1M jittered NN + decode")
S_POINTS, S_QUERIES, S_BITS, S_EXTENT = 30_000_000, 8_000_000, 12, 100.0
# the oracle's bounded sample of the surface step (cpu_baseline and --impl
# reference): build / merge / project / decode of the first S_SAMPLE_PTS points
# of each half; NN of the first S_SAMPLE_SURF on-surface and the first
# S_SAMPLE_UNIF uniform queries against the whole merged world
S_SAMPLE_PTS, S_SAMPLE_SURF, S_SAMPLE_UNIF = 1_000_000, 64, 32
# ncu summary of the dominant kernel of the default workload (per-launch DRAM
# bytes, and the hash of the sources the counters were taken on)
TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "k_nn_tree_surface_8M.txt")
NN_SOURCES = ("k_nn.cu", "k_tree.cu", "k_common.cuh", "cga_impl.h")
N_SWEEPS, BEAMS, STEPS_AZ, N_QUERIES = 10, 64, 2048, 1_000_000
LO, EXTENT, BITS = (-128.0, -128.0, -128.0), 256.0, 16


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["cga", "reference"], default="cga")
    ap.add_argument("--config", choices=["lidar", "plain", "surface", "batched", "served", "values",
                                         "perspective", "search", "compress"],
                    default="surface")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--flush-mb", type=int, default=512)
    ap.add_argument("--serve-seconds", type=float, default=3.0)
    return ap.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def cpu_model() -> str:
    """The host CPU's model string: /proc/cpuinfo's model name, else (Arm
    hosts list none there) lscpu's, else its implementer / part codes."""
    fields = {}
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if ":" in line:
                    k, v = line.split(":", 1)
                    fields.setdefault(k.strip().lower(), v.strip())
    except OSError:
        pass
    for k in ("model name", "cpu model", "hardware"):
        if fields.get(k):
            return fields[k]
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    if "cpu implementer" in fields:
        return (f"{os.uname().machine} implementer {fields['cpu implementer']} part "
                f"{fields.get('cpu part', '?')}")
    import platform
    return platform.processor() or platform.machine()


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def sources_hash(names) -> str:
    import hashlib
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_2110_11616_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def profiled_traffic(path, names):
    """Per-launch DRAM bytes of an ncu summary, or None when the summary is
    missing or the kernel sources changed since its counters were taken."""
    try:
        kv = {}
        with open(path) as f:
            for line in f:
                if ":" in line:
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("source_sha256") != sources_hash(names):
            return None, "kernel sources changed since the ncu capture"
        return int(kv["traffic_bytes_per_launch"]), kv.get("traffic_note", "")
    except (OSError, KeyError, ValueError):
        return None, "no ncu capture"


# ----------------------------------------------------------------- workload
def make_workload(rank: int):
    scene = synth.lidar_sweeps(N_SWEEPS, BEAMS, STEPS_AZ, seed=2 + 1000 * rank)
    q = synth.jitter_queries(scene.world, N_QUERIES, 0.2, seed=5 + 1000 * rank)
    return scene, q


def merge_tree(items, merge):
    """Pairwise merges, adjacent sweeps first: (0,1), (2,3), ... then upwards."""
    level = list(items)
    while len(level) > 1:
        nxt = [merge(level[i], level[i + 1]) for i in range(0, len(level) - 1, 2)]
        if len(level) % 2:
            nxt.append(level[-1])
        level = nxt
    return level[0]


# ------------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(prefix="cga_clocks_", suffix=".csv")
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "-i", str(gpu_index),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def start_clocks(local_rank):
    phys = os.environ.get("CUDA_VISIBLE_DEVICES", str(local_rank)).split(",")[local_rank]
    return Clocks(int(phys) if phys.strip().isdigit() else local_rank)


def timed(torch, fn, flush=None, tag=0.0):
    """Device time (ms) of fn() with CUDA events on the current stream.  The
    launches of fn() sit in an NVTX range "cga_step" (ncu --nvtx-include
    "cga_step/" selects exactly the timed steps' kernels)."""
    if flush is not None:
        flush.fill_(tag)
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    s.record()
    torch.cuda.nvtx.range_push("cga_step")
    fn()
    torch.cuda.nvtx.range_pop()
    e.record()
    e.synchronize()
    return s.elapsed_time(e)


def max_over_ranks(ms: float, world_size: int, torch, dist, device) -> float:
    """The slowest rank's time: replicas run in parallel, so the job takes as
    long as its slowest GPU (weak scaling, no data-path collective)."""
    if world_size <= 1:
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(points_per_step: int, steps: int, world_size: int, max_ms: float) -> float:
    """Whole-job Mpts/s: every rank processes its own replica of the workload."""
    return points_per_step * steps * world_size / (max_ms / 1e3) / 1e6


def base_line(args, world_size, metric, value, unit, ms_per_step, config, data):
    return {"metric": metric, "value": round(value, 4), "unit": unit, "n_gpus": world_size,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32->u16/u32/u64",
            "data": data, "config": config}


def check_e2e(torch, P):
    """The results the end-to-end steps copied back equal the device results."""
    torch.cuda.synchronize()
    if not (torch.equal(P.h_idx, P.idx.cpu()) and torch.equal(P.h_d2, P.d2.cpu())):
        raise RuntimeError("end-to-end NN results differ from the device results")


def overlapped_e2e(P, h_clouds, d_clouds):
    """One step from pinned host buffers to results in pinned host memory, as
    a user would run it: the clouds go up first (the build needs them); the
    queries go up on a side stream while the clouds are built, merged and
    projected; the NN results come down on that stream while the merged cloud
    is decoded.  The current stream waits for the side stream before the
    query sort and at the end, so every copy lies inside the caller's timed
    region, and the next step's writes wait for this step's reads."""
    torch = P.torch
    main = torch.cuda.current_stream()
    side = P.side
    for h, d in zip(h_clouds, d_clouds):
        d.copy_(h, non_blocking=True)
    side.wait_stream(main)
    with torch.cuda.stream(side):
        P.d_q.copy_(P.h_q, non_blocking=True)

    def results_down():
        side.wait_stream(main)
        with torch.cuda.stream(side):
            P.h_idx.copy_(P.idx, non_blocking=True)
            P.h_d2.copy_(P.d2, non_blocking=True)

    P.step(timed_events=False, before_sort=lambda: main.wait_stream(side), after_nn=results_down)
    main.wait_stream(side)


# --------------------------------------------------------------- GPU arm: C2
class LidarStep:
    def __init__(self, scene, queries, torch, cga):
        self.torch, self.cga = torch, cga
        self.grid = cga.grid_from_box(LO, EXTENT, BITS)
        self.h_sweeps = [torch.from_numpy(s).pin_memory() for s in scene.sweeps]
        self.h_q = torch.from_numpy(queries).pin_memory()
        self.d_sweeps = [h.cuda() for h in self.h_sweeps]
        self.d_q = self.h_q.cuda()
        self.poses = scene.poses
        m = len(queries)
        self.order = torch.empty(m, dtype=torch.int64, device="cuda")
        self.idx = torch.empty(m, dtype=torch.int32, device="cuda")
        self.d2 = torch.empty(m, dtype=torch.int64, device="cuda")
        self.h_idx = torch.empty(m, dtype=torch.int32).pin_memory()
        self.h_d2 = torch.empty(m, dtype=torch.int64).pin_memory()
        self.n_points = sum(len(s) for s in scene.sweeps)
        self.dec = torch.empty((self.n_points, 3), dtype=torch.int32, device="cuda")
        self.ev = [torch.cuda.Event(enable_timing=True) for _ in range(7)]
        self.nn_shift = ()  # NN coarse levels picked by cga_nn_autotune before timing
        self.side = torch.cuda.Stream()  # host copies overlapped with the step (e2e_step)

    def step(self, timed_events=True, batched=True, before_sort=None, after_nn=None):
        cga, ev = self.cga, self.ev
        rec = (lambda i: ev[i].record()) if timed_events else (lambda i: None)
        rec(0)
        if batched:
            sweeps = cga.cga_build_batch(self.d_sweeps, self.grid, self.poses, allocator=None)
        else:
            sweeps = [cga.cga_build(d, self.grid, xform=p, allocator=None)
                      for d, p in zip(self.d_sweeps, self.poses)]
        rec(1)
        merges = []
        level = list(sweeps)
        while len(level) > 1:
            a, b = level[0:len(level) - 1:2], level[1::2]
            if batched:
                nxt = cga.cga_merge_batch(a, b, allocator=None)
            else:
                nxt = [cga.cga_merge(x, y, allocator=None) for x, y in zip(a, b)]
            merges.extend(zip(a, b, nxt))
            if len(level) % 2:
                nxt.append(level[-1])
            level = nxt
        world = level[0]
        rec(2)
        proj = cga.cga_project(world, "xy", allocator=None)
        rec(3)
        cga.cga_nn_prepare(world, self.nn_shift)
        if before_sort is not None:
            before_sort()
        cga.cga_nn_sort_queries(world, self.d_q, self.order)
        rec(4)
        cga.cga_nn_query_ordered(world, self.d_q, self.order, self.idx, self.d2)
        rec(5)
        if after_nn is not None:
            after_nn()
        cga.cga_decode(world, out=self.dec)
        rec(6)
        self.last = (sweeps, merges, world, proj)

    def op_times(self):
        e = self.ev
        return [e[i].elapsed_time(e[i + 1]) for i in range(6)]

    def e2e_step(self):
        overlapped_e2e(self, self.h_sweeps, self.d_sweeps)

    def bytes_in(self):
        return sum(h.numel() * 4 for h in self.h_sweeps) + self.h_q.numel() * 4

    def bytes_out(self):
        return self.h_idx.numel() * 4 + self.h_d2.numel() * 8


def tune_record(shifts, times):
    """cga_nn_autotune's choice and each strategy's measured cost for the JSON
    line (its preparation plus the sample's search scaled to the step's
    queries, where the step prepares the world itself)."""
    name = lambda c: "tree" if c == (0xFFFFFFFF,) else (",".join(map(str, c)) if c else "fine")
    return {"chosen": name(tuple(shifts)),
            "sample_ms": {name(c): round(t, 4) for c, t in times.items()}}


def shape_record(shape, times):
    """A launch shape chosen by cga_autotune / cga_pipeline_autotune, with the
    candidates' times, for the JSON line."""
    return {"shape": shape,
            "sort_ms": {f"{rb}b/{th}t": round(t, 4) for (rb, th), t in times["sort"].items()},
            "merge_ms": {str(h): round(t, 4) for h, t in times["merge"].items()}}


def tune_launch_shapes(cga, clouds, grid):
    """cga_autotune on representative clouds, one per size bucket the step
    sorts or merges; returns {n: record}."""
    out = {}
    for c in clouds:
        shape, times = cga.cga_autotune(c.contiguous(), grid)
        out[str(c.numel() // 3)] = shape_record(shape, times)
    return out


def run_lidar(args, rank, world_size, local_rank, torch, dist, cga):
    scene, queries = make_workload(rank)
    P = LidarStep(scene, queries, torch, cga)
    flush = torch.empty(args.flush_mb * (1 << 20) // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if world_size > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # sort / merge launch shapes by measurement on clouds of 1, 2, 4 and 8
    # sweeps (the size buckets of the builds and of each merge level)
    shapes = tune_launch_shapes(
        cga, [torch.cat(P.d_sweeps[:k]) for k in (1, 2, 4, 8) if k <= len(P.d_sweeps)], P.grid)
    # NN strategy by measurement on this workload's 1M queries themselves (a
    # sparser sample changes how neighbouring queries share a warp's loads and
    # misjudges the window search); the world is prepared every step, so each
    # strategy is charged its preparation plus the search
    P.step(timed_events=False)
    P.nn_shift, nn_tune = cga.cga_nn_autotune(P.last[2], P.d_q, queries_per_prepare=N_QUERIES)
    for _ in range(args.warmup):
        P.step()
    torch.cuda.synchronize()
    clocks = start_clocks(local_rank)
    time.sleep(0.3)
    op_ms = np.zeros(6)
    step_ms = []
    launches0 = cga.kernel_launches()
    barrier()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        step_ms.append(timed(torch, P.step, flush, float(k)))
        op_ms += np.array(P.op_times())
    barrier()
    t_wall = time.perf_counter() - t_wall
    launches = cga.kernel_launches() - launches0
    total_ms = float(sum(step_ms))
    plain_ms = [timed(torch, lambda: P.step(timed_events=False, batched=False), flush, float(k))
                for k in range(max(3, args.steps // 2))]
    P.e2e_step()  # untimed: the first copies of the pinned buffers are slower once
    e2e_ms = []
    for k in range(max(3, args.steps // 3)):
        torch.cuda.synchronize()
        e2e_ms.append(timed(torch, P.e2e_step, flush, float(k)))
    clk = clocks.stop()
    check_e2e(torch, P)

    sweeps, merges, world, proj = P.last
    winfo = world.info()
    merge_bytes = sum(a.info()["bytes"] + b.info()["bytes"] + m.info()["bytes"]
                      for a, b, m in merges)
    op = op_ms / args.steps
    max_total = max_over_ranks(total_ms, world_size, torch, dist, "cuda")
    pts = P.n_points
    value = job_value(pts, args.steps, world_size, max_total)
    e2e_val = pts * world_size / (float(np.mean(e2e_ms)) / 1e3) / 1e6
    peak, peak_kind = measured_peaks()
    # dominant kernel: the NN search (one launch per step of k_nn_warp, or of
    # k_nn_tree when the autotuner picked the tree, timed live above between
    # events 4 and 5).  Algorithmic bytes per launch (compulsory): 12 B query
    # read, 4 B index + 8 B distance written.
    search_ms = op[4]
    algo = N_QUERIES * (12 + 4 + 8)
    achieved = algo / (search_ms / 1e3) / 1e9
    out = base_line(args, world_size, METRIC, value, "Mpts/s", max_total / args.steps,
                    {"workload": WORKLOAD_LIDAR, "points_per_step": pts, "queries_per_step": N_QUERIES,
                     "grid_bits": BITS, "l2": f"flushed between steps ({args.flush_mb} MB write)",
                     "parallelism": f"replicas x{world_size}" if world_size > 1 else "1 GPU"},
                    "synthetic (seeded LiDAR generator; stands in for the paper's LiDAR scans)")
    out.update({
        "breakdown_ms": {"build": round(op[0], 4), "merge": round(op[1], 4),
                         "project_xy": round(op[2], 4), "nn_sort": round(op[3], 4),
                         "nn_search": round(op[4], 4), "decode": round(op[5], 4)},
        "derived": {
            "build_Mpts_s": round(pts / (op[0] / 1e3) / 1e6, 2),
            "nn_queries_s": round(N_QUERIES / ((op[3] + op[4]) / 1e3), 1),
            "merge_GB_s": round(merge_bytes / (op[1] / 1e3) / 1e9, 2),
            "merge_frac_of_hbm": round(merge_bytes / (op[1] / 1e3) / 1e9 / peak, 5),
            "merge_compulsory_bytes": merge_bytes,
            "world_u": winfo["u"], "world_g": winfo["g"], "world_h": winfo["h"],
            "world_bytes": winfo["bytes"], "raw_bytes": pts * 12,
        },
        "roofline": {"kernel": ("k_nn_tree (NN search over the occupancy tree)"
                                if tuple(P.nn_shift) == (0xFFFFFFFF,) else
                                "k_nn_warp (NN window search)"), "bound": "hbm",
                     "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 6), "traffic": None,
                     "peak_source": f"{peak_kind} hbm_gbs",
                     "algorithmic_bytes_per_launch": algo,
                     "note": "compulsory bytes: 12 B query in + 12 B result out per query; "
                             "latency-bound search (dependent L1/L2 loads), not an HBM "
                             "stream; no ncu capture of this launch is on record for the "
                             "current sources, so traffic is null"},
        "e2e": {"value": round(e2e_val, 3), "unit": "Mpts/s",
                "h2d_bytes_per_step": P.bytes_in(), "d2h_bytes_per_step": P.bytes_out()},
        "plain": {"ms_per_step": round(float(np.mean(plain_ms)), 4),
                  "value": round(pts / (float(np.mean(plain_ms)) / 1e3) / 1e6, 3),
                  "note": "one call per sweep build and per merge (the step above batches "
                          "the 10 builds and each merge-tree level into one launch set)"},
        "nn_autotune": tune_record(P.nn_shift, nn_tune),
        "launch_shapes": shapes,
        "gpu_launches": int(launches),
        "clocks": clk,
        "wall_s": round(t_wall, 3),
    })
    return out, (scene, queries)


# ----------------------------------------------------- GPU arm: C3 (default)
def surface_inputs(device):
    """The surface workload's float32 inputs (seeded, drawn on `device`): the
    two 15M-point halves and the 8M queries (4M on-surface, then 4M uniform)."""
    from paper_2110_11616_gb300 import synth_gpu
    scene = synth_gpu.surface_scene(3, device=device)
    full = synth_gpu.sample_scene(scene, S_POINTS, seed=4)
    halves = [full[0::2].contiguous(), full[1::2].contiguous()]
    del full
    surf = synth_gpu.sample_scene(scene, S_QUERIES // 2, seed=5)
    uni = synth_gpu.uniform_queries(S_QUERIES // 2, 6, [0.0, 0.0, 0.0], S_EXTENT, device=device)
    import torch
    return halves, torch.cat([surf, uni]).contiguous()


def surface_config(args, world_size):
    return {"workload": WORKLOAD, "points_per_step": S_POINTS, "queries_per_step": S_QUERIES,
            "grid_bits": S_BITS, "l2": f"flushed between steps ({args.flush_mb} MB write)",
            "parallelism": f"replicas x{world_size}" if world_size > 1 else "1 GPU"}


class SurfaceStep:
    def __init__(self, torch, cga):
        self.torch, self.cga = torch, cga
        self.grid = cga.grid_from_box([0.0, 0.0, 0.0], S_EXTENT, S_BITS)
        self.d_halves, self.d_q = surface_inputs("cuda")
        self.h_halves = [h.cpu().pin_memory() for h in self.d_halves]
        self.h_q = self.d_q.cpu().pin_memory()
        m = S_QUERIES
        self.order = torch.empty(m, dtype=torch.int64, device="cuda")
        self.idx = torch.empty(m, dtype=torch.int32, device="cuda")
        self.d2 = torch.empty(m, dtype=torch.int64, device="cuda")
        self.h_idx = torch.empty(m, dtype=torch.int32).pin_memory()
        self.h_d2 = torch.empty(m, dtype=torch.int64).pin_memory()
        self.dec = torch.empty((S_POINTS, 3), dtype=torch.int32, device="cuda")
        self.ev = [torch.cuda.Event(enable_timing=True) for _ in range(7)]
        self.nn_strategy = "tree"  # replaced by cga_nn_autotune's choice before timing
        self.side = torch.cuda.Stream()  # host copies overlapped with the step (e2e_step)
        self.half_up = torch.cuda.Event()

    def step(self, timed_events=True, before_sort=None, after_nn=None, build=None):
        cga, ev = self.cga, self.ev
        rec = (lambda i: ev[i].record()) if timed_events else (lambda i: None)
        rec(0)
        if build is None:
            a, b = cga.cga_build_batch(self.d_halves, self.grid, [None, None], allocator=None)
        else:
            a, b = build()
        rec(1)
        mg = cga.cga_merge(a, b, allocator=None)
        rec(2)
        pr = cga.cga_project_batch([mg] * 3, ["xy", "xz", "yz"], allocator=None)
        rec(3)
        cga.cga_nn_prepare(mg, self.nn_strategy)
        if before_sort is not None:
            before_sort()
        cga.cga_nn_sort_queries(mg, self.d_q, self.order)
        rec(4)
        cga.cga_nn_query_ordered(mg, self.d_q, self.order, self.idx, self.d2)
        rec(5)
        if after_nn is not None:
            after_nn()
        cga.cga_decode(mg, out=self.dec)
        rec(6)
        self.last = (a, b, mg, pr)

    def op_times(self):
        e = self.ev
        return [e[i].elapsed_time(e[i + 1]) for i in range(6)]

    def e2e_step(self):
        """As overlapped_e2e, with the second half's upload overlapped too: it
        goes up on the side stream while the first half is built, and the
        halves are built by one cga_build each (the same CGAs as the batched
        build)."""
        torch, cga = self.torch, self.cga
        main = torch.cuda.current_stream()
        side = self.side
        (h0, h1), (d0, d1) = self.h_halves, self.d_halves
        d0.copy_(h0, non_blocking=True)
        side.wait_stream(main)
        with torch.cuda.stream(side):
            d1.copy_(h1, non_blocking=True)
            self.half_up.record(side)
            self.d_q.copy_(self.h_q, non_blocking=True)

        def build():
            a = cga.cga_build(d0, self.grid, allocator=None)
            main.wait_event(self.half_up)
            return a, cga.cga_build(d1, self.grid, allocator=None)

        def results_down():
            side.wait_stream(main)
            with torch.cuda.stream(side):
                self.h_idx.copy_(self.idx, non_blocking=True)
                self.h_d2.copy_(self.d2, non_blocking=True)

        self.step(timed_events=False, before_sort=lambda: main.wait_stream(side),
                  after_nn=results_down, build=build)
        main.wait_stream(side)

    def bytes_in(self):
        return sum(h.numel() * 4 for h in self.h_halves) + self.h_q.numel() * 4

    def bytes_out(self):
        return self.h_idx.numel() * 4 + self.h_d2.numel() * 8


def run_surface(args, world_size, local_rank, torch, dist, cga):
    P = SurfaceStep(torch, cga)
    flush = torch.empty(args.flush_mb * (1 << 20) // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if world_size > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # sort / merge launch shapes by measurement on a half and on the whole cloud
    reps = [P.d_halves[0], torch.cat(P.d_halves)]
    shapes = tune_launch_shapes(cga, reps, P.grid)
    del reps
    # NN strategy by measurement on a 64k sample mixing both query halves,
    # each strategy charged its preparation (done every step) plus the search
    # scaled to the step's queries
    P.step(timed_events=False)
    gen = torch.Generator("cuda").manual_seed(7)
    sample = P.d_q[torch.randperm(S_QUERIES, device="cuda", generator=gen)[:65536]].contiguous()
    shifts, nn_tune = cga.cga_nn_autotune(P.last[2], sample, queries_per_prepare=S_QUERIES)
    P.nn_strategy = shifts
    for _ in range(args.warmup):
        P.step()
    torch.cuda.synchronize()
    clocks = start_clocks(local_rank)
    time.sleep(0.3)
    op_ms = np.zeros(6)
    step_ms = []
    launches0 = cga.kernel_launches()
    barrier()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        step_ms.append(timed(torch, P.step, flush, float(k)))
        op_ms += np.array(P.op_times())
    barrier()
    t_wall = time.perf_counter() - t_wall
    launches = cga.kernel_launches() - launches0
    # end to end: one untimed pass first (the first host<->device copies of the
    # pinned buffers are slower once), then timed steps
    P.e2e_step()
    e2e_ms = []
    for k in range(max(3, args.steps // 3)):
        torch.cuda.synchronize()
        e2e_ms.append(timed(torch, P.e2e_step, flush, float(k)))
    clk = clocks.stop()
    check_e2e(torch, P)

    a, b, mg, pr = P.last
    ai, bi, mi = a.info(), b.info(), mg.info()
    merge_bytes = ai["bytes"] + bi["bytes"] + mi["bytes"]
    op = op_ms / args.steps
    total_ms = float(sum(step_ms))
    max_total = max_over_ranks(total_ms, world_size, torch, dist, "cuda")
    value = job_value(S_POINTS, args.steps, world_size, max_total)
    e2e_val = S_POINTS * world_size / (float(np.mean(e2e_ms)) / 1e3) / 1e6
    peak, peak_kind = measured_peaks()
    # dominant kernel: the NN search under the tree (k_nn_tree, two launches
    # per step: every 32nd query in Morton order, then the rest seeded by
    # them), timed live as one region between events 4 and 5.  Algorithmic
    # bytes per search (compulsory): 12 B query read + 4 B index + 8 B
    # distance written per query.
    search_ms = op[4]
    algo = S_QUERIES * (12 + 4 + 8)
    achieved = algo / (search_ms / 1e3) / 1e9
    traffic, traffic_note = profiled_traffic(TRAFFIC_PROFILE, NN_SOURCES)
    passes = math.ceil(3 * S_BITS / shapes[str(S_POINTS // 2)]["shape"]["radix_bits"])
    build_design = (S_POINTS * (12 + 8 + 16 * passes + 8) + ai["bytes"] + bi["bytes"])
    out = base_line(args, world_size, METRIC, value, "Mpts/s", max_total / args.steps,
                    surface_config(args, world_size),
                    "synthetic (seeded superellipsoid surfaces; stands in for the paper's "
                    "8iVSLF surface sequences)")
    out.update({
        "breakdown_ms": {"build": round(op[0], 4), "merge": round(op[1], 4),
                         "project_xy_xz_yz": round(op[2], 4),
                         "nn_prepare_sort": round(op[3], 4), "nn_search": round(op[4], 4),
                         "decode": round(op[5], 4)},
        "derived": {
            "build_Mpts_s": round(S_POINTS / (op[0] / 1e3) / 1e6, 2),
            "build_by_design_GB_s": round(build_design / (op[0] / 1e3) / 1e9, 1),
            "build_by_design_frac_of_hbm": round(build_design / (op[0] / 1e3) / 1e9 / peak, 4),
            "nn_queries_s": round(S_QUERIES / ((op[3] + op[4]) / 1e3), 1),
            "nn_search_queries_s": round(S_QUERIES / (op[4] / 1e3), 1),
            "merge_GB_s": round(merge_bytes / (op[1] / 1e3) / 1e9, 2),
            "merge_frac_of_hbm": round(merge_bytes / (op[1] / 1e3) / 1e9 / peak, 5),
            "merge_compulsory_bytes": merge_bytes,
            "merged_u": mi["u"], "merged_g": mi["g"], "merged_h": mi["h"],
            "merged_bytes": mi["bytes"], "raw_bytes": S_POINTS * 12,
        },
        "roofline": {"kernel": ("k_nn_tree (NN search over the occupancy tree)"
                                if tuple(P.nn_strategy) == (0xFFFFFFFF,) else
                                "k_nn_warp (NN window search)"),
                     "bound": "hbm", "achieved": round(achieved, 3), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 6), "traffic": traffic,
                     "peak_source": f"{peak_kind} hbm_gbs (burst copy)",
                     "algorithmic_bytes_per_launch": algo,
                     "note": "compulsory bytes: 12 B query in + 12 B result out per query over "
                             "the live CUDA-event time of the search (both launches of the "
                             "tree search); the search is bound by integer instruction issue "
                             "and L1/L2 latency, not HBM. traffic: ncu dram read+write of the "
                             "search's launches "
                             + (f"({traffic_note})" if traffic_note else "")},
        "e2e": {"value": round(e2e_val, 3), "unit": "Mpts/s",
                "h2d_bytes_per_step": P.bytes_in(), "d2h_bytes_per_step": P.bytes_out()},
        "nn_autotune": tune_record(tuple(shifts), nn_tune),
        "launch_shapes": shapes,
        "gpu_launches": int(launches),
        "clocks": clk,
        "wall_s": round(t_wall, 3),
    })
    return out, P


# ------------------------------------------------------------------ GPU arm: C1
def run_single(args, world_size, local_rank, torch, cga, which):
    from paper_2110_11616_gb300 import synth_gpu
    pts = torch.from_numpy(synth.uniform_cube(100_000, seed=1)).cuda()
    X = synth.rigid_xform(seed=2)
    halves = [pts, pts]
    xforms = [None, X]
    grid = cga.grid_from_box([0, 0, 0], 1.0, 10)
    q = torch.from_numpy(synth.uniform_queries(10_000, 3, [0, 0, 0], 1.0)).cuda()
    planes = ["xy"]
    workload = ("plain: 100k uniform pts + rigidly transformed twin, b=10; batched build of "
                "both, merge, xy projection, 10k uniform NN, decode")
    n_points = 200_000
    coarse_shift = ()
    m = q.shape[0]
    order = torch.empty(m, dtype=torch.int64, device="cuda")
    idx = torch.empty(m, dtype=torch.int32, device="cuda")
    d2 = torch.empty(m, dtype=torch.int64, device="cuda")
    dec = torch.empty((n_points, 3), dtype=torch.int32, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(7)]
    state = {}

    def step():
        ev[0].record()
        a, b = cga.cga_build_batch(halves, grid, xforms, allocator=None)
        ev[1].record()
        mg = cga.cga_merge(a, b, allocator=None)
        ev[2].record()
        pr = cga.cga_project_batch([mg] * len(planes), planes, allocator=None)
        ev[3].record()
        cga.cga_nn_prepare(mg, coarse_shift)
        cga.cga_nn_sort_queries(mg, q, order)
        ev[4].record()
        cga.cga_nn_query_ordered(mg, q, order, idx, d2)
        ev[5].record()
        cga.cga_decode(mg, out=dec)
        ev[6].record()
        state["last"] = (a, b, mg, pr)

    flush = torch.empty(args.flush_mb * (1 << 20) // 4, dtype=torch.float32, device="cuda")
    # sort / merge launch shapes by measurement (the cloud and the pair)
    reps = [halves[0], torch.cat(halves)]
    shapes = tune_launch_shapes(cga, reps, grid)
    del reps
    # NN strategy by measurement on a 64k sample mixing both query halves
    step()
    sample = q[torch.randperm(m, device="cuda", generator=torch.Generator("cuda").manual_seed(7))
               [:65536]].contiguous()
    coarse_shift, nn_tune = cga.cga_nn_autotune(state["last"][2], sample, queries_per_prepare=m)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = start_clocks(local_rank)
    ops = np.zeros(6)
    ms = []
    launches0 = cga.kernel_launches()
    for k in range(args.steps):
        ms.append(timed(torch, step, flush, float(k)))
        ops += np.array([ev[i].elapsed_time(ev[i + 1]) for i in range(6)])
    launches = cga.kernel_launches() - launches0
    clk = clocks.stop()
    ops /= args.steps
    a, b, mg, pr = state["last"]
    mi = mg.info()
    merge_bytes = a.info()["bytes"] + b.info()["bytes"] + mi["bytes"]
    peak, peak_kind = measured_peaks()
    total = float(sum(ms))
    out = base_line(args, world_size, METRIC, n_points * args.steps / (total / 1e3) / 1e6,
                    "Mpts/s", total / args.steps,
                    {"workload": workload, "points_per_step": n_points, "queries_per_step": m,
                     "l2": "flushed between steps"}, "synthetic (seeded generators)")
    out.update({
        "breakdown_ms": {"build": round(ops[0], 4), "merge": round(ops[1], 4),
                         "project": round(ops[2], 4), "nn_prepare_sort": round(ops[3], 4),
                         "nn_search": round(ops[4], 4), "decode": round(ops[5], 4)},
        "derived": {"build_Mpts_s": round(n_points / (ops[0] / 1e3) / 1e6, 2),
                    "nn_queries_s": round(m / ((ops[3] + ops[4]) / 1e3), 1),
                    "merge_GB_s": round(merge_bytes / (ops[1] / 1e3) / 1e9, 2),
                    "merge_frac_of_hbm": round(merge_bytes / (ops[1] / 1e3) / 1e9 / peak, 4),
                    "build_by_design_GB_s": round(
                        (n_points * (12 + 8 + 16 * math.ceil(3 * grid.bits / 8) + 8)
                         + a.info()["bytes"] + b.info()["bytes"]) / (ops[0] / 1e3) / 1e9, 1),
                    "merged_u": mi["u"], "merged_bytes": mi["bytes"], "raw_bytes": n_points * 12,
                    "peak_gbs": peak, "peak_source": peak_kind},
        "nn_autotune": tune_record(coarse_shift, nn_tune),
        "launch_shapes": shapes,
        "gpu_launches": int(launches), "clocks": clk})
    return out


# --------------------------------------------------------- GPU arm: C4 batched
def run_batched(args, world_size, local_rank, torch, cga):
    from paper_2110_11616_gb300 import synth_gpu
    S = 512
    sizes = synth.log_uniform_ints(S, 5_000, 2_000_000, seed=41)
    rng = np.random.default_rng(42)
    bits = rng.integers(10, 17, size=S)
    pts, grids, xforms, qs = [], [], [], []
    for i in range(S):
        n = int(sizes[i])
        if i % 2 == 0:
            p = synth_gpu.lidar_cloud(n, seed=1000 + i)
            grids.append(cga.grid_from_box([-128.0] * 3, 256.0, int(bits[i])))
            qs.append(synth_gpu.jitter_queries(p, 4096, 0.2, seed=3000 + i))
        else:
            p = synth_gpu.surface_cloud(n, seed=1000 + i, n_objects=max(4, min(200, n // 5000)))
            grids.append(cga.grid_from_box([0.0] * 3, 100.0, int(bits[i])))
            qs.append(synth_gpu.jitter_queries(p, 4096, 0.1, seed=3000 + i))
        pts.append(p)
        xforms.append(synth.rigid_xform(seed=2000 + i))
    total_pts = 2 * int(sizes.sum())
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        # radix digit width, threads per tile and merge-path partition of the
        # pipeline, by timing its graph replay under each candidate
        shape, tune_times = cga.pipeline_autotune(pts, grids, xforms, qs)
        pipe = cga.Pipeline(pts, grids, xforms, qs, allocator=None)
        idx_p = [t for t in pipe.idx]
        for _ in range(args.warmup):
            pipe.run_graph()
        stream.synchronize()
        clocks = start_clocks(local_rank)
        launches0 = cga.kernel_launches()
        ms = [timed(torch, pipe.run_graph) for _ in range(args.steps)]
        launches = cga.kernel_launches() - launches0
        ms_nograph = [timed(torch, pipe.run) for _ in range(max(2, args.steps // 3))]
        d2_pipe = [t.clone() for t in pipe.dist2]

        def plain():
            res = []
            for i in range(S):
                a = cga.cga_build(pts[i], grids[i], allocator=None)
                b = cga.cga_build(pts[i], grids[i], xform=xforms[i], allocator=None)
                m = cga.cga_merge(a, b, allocator=None)
                cga.cga_project(m, "xy", allocator=None)
                res.append(cga.cga_nn_query(m, qs[i]))
            return res
        # both forms on both clocks: CUDA events on the launching stream
        # (device time) and the host clock around the call + synchronize
        plain_ms, plain_dev_ms = [], []
        for _ in range(2):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0 = time.perf_counter()
            e0.record()
            res = plain()
            e1.record()
            torch.cuda.synchronize()
            plain_ms.append((time.perf_counter() - t0) * 1e3)
            plain_dev_ms.append(e0.elapsed_time(e1))
        graph_host_ms = []
        for _ in range(max(2, args.steps // 3)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pipe.run_graph()
            torch.cuda.synchronize()
            graph_host_ms.append((time.perf_counter() - t0) * 1e3)
        clk = clocks.stop()
        same = all(torch.equal(d2_pipe[i], res[i][1]) for i in range(S))
    del idx_p
    total = float(sum(ms))
    out = base_line(args, world_size, METRIC, total_pts * args.steps / (total / 1e3) / 1e6,
                    "Mpts/s", total / args.steps,
                    {"workload": "batched: 512 clouds, n log-uniform [5e3, 2e6] (LiDAR / "
                                 "superellipsoid alternating), b uniform in 10..16; build + "
                                 "transformed twin + merge + xy projection + 4096 NN each, one "
                                 "pre-planned pipeline replayed from a CUDA graph",
                     "clouds": S, "points_per_step": total_pts, "l2": "inputs > L2"},
                    "synthetic (seeded GPU generators)")
    graph_dev = total / args.steps
    out.update({"graph_ms": round(graph_dev, 3),
                "graph_host_ms": round(float(np.min(graph_host_ms)), 3),
                "pipeline_no_graph_ms": round(float(np.mean(ms_nograph)), 3),
                "plain_512_calls_ms": round(float(np.min(plain_ms)), 3),
                "plain_512_calls_device_ms": round(float(np.min(plain_dev_ms)), 3),
                "plain_timing": "512 sequential calls: host clock around the calls + "
                                "synchronize, and CUDA events around them on the same stream",
                "speedup_vs_plain": {
                    "device_clock": round(float(np.min(plain_dev_ms)) / graph_dev, 2),
                    "host_clock": round(float(np.min(plain_ms)) / float(np.min(graph_host_ms)), 2)},
                "nn_results_equal_plain": bool(same),
                "launch_shape": shape_record(shape, tune_times),
                "gpu_launches": int(launches), "clocks": clk})
    return out


# ---------------------------------------------------------- GPU arm: C5 served
def run_served(args, world_size, local_rank, torch, cga):
    from paper_2110_11616_gb300 import synth_gpu
    K = 64
    sizes = synth.log_uniform_ints(K, 100_000, 20_000_000, seed=51)
    grid = cga.grid_from_box([-128.0] * 3, 256.0, 16)
    pool, banks = [], []
    for i in range(K):
        n = int(sizes[i])
        p = (synth_gpu.lidar_cloud(n, seed=5000 + i) if i % 2 == 0 else
             synth_gpu.surface_cloud(n, seed=5000 + i, n_objects=max(4, min(200, n // 50000))))
        pool.append(cga.cga_build(p, grid, allocator=None))
        banks.append(synth_gpu.jitter_queries(p, 1_000_000, 0.2, seed=6000 + i))
        del p
    torch.cuda.synchronize()
    resident = sum(c.info()["bytes"] for c in pool)
    rng = np.random.default_rng(52)
    rate = 2000.0
    n_req = int(rate * args.serve_seconds)
    gaps = rng.exponential(1.0 / rate, size=n_req)
    arrivals = np.cumsum(gaps)
    reqs = []
    for r in range(n_req):
        if rng.random() < 0.7:
            m = int(math.exp(rng.uniform(0.0, math.log(1_000_000))))
            reqs.append(("nn", int(rng.integers(K)), m))
        else:
            reqs.append(("mp", int(rng.integers(K)), int(rng.integers(K))))
    server = cga.Server(pool, memory_budget=64 << 30, slots=4, max_batch=64)
    clocks = start_clocks(local_rank)
    t0 = time.perf_counter()
    tickets = {}
    for r, at in zip(reqs, arrivals):
        while time.perf_counter() - t0 < at:
            pass
        if r[0] == "nn":
            q = banks[r[1]][:r[2]]
            idx = torch.empty(r[2], dtype=torch.int32, device="cuda")
            d2 = torch.empty(r[2], dtype=torch.int64, device="cuda")
            tickets[server.submit_nn(r[1], q, idx, d2)] = r
        else:
            tickets[server.submit_merge_project(r[1], r[2], "xy")] = r
    server.drain()
    done = server.poll(max_n=n_req + 16)
    clk = clocks.stop()
    lat = np.array([(c["t_done_ns"] - c["t_submit_ns"]) / 1e6 for c in done])
    span = (max(c["t_done_ns"] for c in done) - min(c["t_submit_ns"] for c in done)) / 1e9
    nq = sum(r[2] for r in reqs if r[0] == "nn")
    lat_nn = np.array([(c["t_done_ns"] - c["t_submit_ns"]) / 1e6 for c in done
                       if tickets[c["ticket"]][0] == "nn"])
    lat_mp = np.array([(c["t_done_ns"] - c["t_submit_ns"]) / 1e6 for c in done
                       if tickets[c["ticket"]][0] == "mp"])
    ok = all(c["status"] == 0 for c in done)
    del done
    server.free()

    # saturation: the same request list submitted at once (admission by
    # footprint decides what runs together), against the same list run one
    # request after another through the plain calls.  Both on the host clock
    # from one common start; a request's latency is its completion time since
    # that start (every request is waiting at the start).
    def submit_all(srv):
        keep = []
        for r in reqs:
            if r[0] == "nn":
                q = banks[r[1]][:r[2]]
                idx = torch.empty(r[2], dtype=torch.int32, device="cuda")
                d2 = torch.empty(r[2], dtype=torch.int64, device="cuda")
                srv.submit_nn(r[1], q, idx, d2)
                keep.append((idx, d2))
            else:
                srv.submit_merge_project(r[1], r[2], "xy")
        return keep

    torch.cuda.synchronize()
    sat = cga.Server(pool, memory_budget=64 << 30, slots=4, max_batch=64)
    t0_ns = time.perf_counter_ns()
    t0 = time.perf_counter()
    keep = submit_all(sat)
    sat.drain()
    sat_s = time.perf_counter() - t0
    sat_done = sat.poll(max_n=n_req + 16)
    sat_ok = all(c["status"] == 0 for c in sat_done) and len(sat_done) == n_req
    # the server stamps with the steady clock; shift to perf_counter's origin
    sat_first = min(c["t_submit_ns"] for c in sat_done)
    sat_lat = np.array([(c["t_done_ns"] - sat_first) / 1e6 for c in sat_done])
    del sat_done, keep
    sat.free()
    torch.cuda.synchronize()
    start_ev = torch.cuda.Event(enable_timing=True)
    ends = [torch.cuda.Event(enable_timing=True) for _ in reqs]
    t0 = time.perf_counter()
    start_ev.record()
    for r, ev in zip(reqs, ends):
        if r[0] == "nn":
            cga.cga_nn_query(pool[r[1]], banks[r[1]][:r[2]])
        else:
            mg = cga.cga_merge(pool[r[1]], pool[r[2]], allocator=None)
            cga.cga_project(mg, "xy", allocator=None)
        ev.record()
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t0
    plain_lat = np.array([start_ev.elapsed_time(ev) for ev in ends])
    # each request alone through the plain path (a seeded sample)
    alone = []
    for r in [reqs[i] for i in rng.choice(n_req, size=min(200, n_req), replace=False)]:
        torch.cuda.synchronize()
        t = time.perf_counter()
        if r[0] == "nn":
            cga.cga_nn_query(pool[r[1]], banks[r[1]][:r[2]])
        else:
            mg = cga.cga_merge(pool[r[1]], pool[r[2]], allocator=None)
            cga.cga_project(mg, "xy", allocator=None)
        torch.cuda.synchronize()
        alone.append((time.perf_counter() - t) * 1e3)
    alone = np.array(alone)
    out = base_line(args, world_size, "served requests/s (p50/p99 latency)", n_req / span,
                    "requests/s", span * 1e3,
                    {"workload": "served: Poisson 2000 req/s over 64 resident CGAs (n log-uniform "
                                 "[1e5, 2e7], b=16); 70% NN (m log-uniform [1, 1e6]), 30% "
                                 "merge + xy projection of a random pair",
                     "requests": n_req, "resident_points": int(sizes.sum()),
                     "resident_cga_bytes": int(resident), "slots": 4, "max_batch": 64,
                     "memory_budget_bytes": 64 << 30},
                    "synthetic (seeded GPU generators)")
    out.update({"all_ok": ok, "queries_per_s": round(nq / span, 1),
                "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 3),
                               "p99": round(float(np.percentile(lat, 99)), 3),
                               "nn_p50": round(float(np.percentile(lat_nn, 50)), 3),
                               "nn_p99": round(float(np.percentile(lat_nn, 99)), 3),
                               "mp_p50": round(float(np.percentile(lat_mp, 50)), 3),
                               "mp_p99": round(float(np.percentile(lat_mp, 99)), 3)},
                "alone_latency_ms": {"p50": round(float(np.percentile(alone, 50)), 3),
                                     "p99": round(float(np.percentile(alone, 99)), 3),
                                     "sample": len(alone)},
                "saturation": {
                    "what": "the same request list submitted at once to the server, and run "
                            "one request after another through the plain calls; host clock "
                            "from one common start; latency = completion time since the start",
                    "served_s": round(sat_s, 4), "plain_s": round(plain_s, 4),
                    "served_requests_s": round(n_req / sat_s, 1),
                    "plain_requests_s": round(n_req / plain_s, 1),
                    "served_queries_s": round(nq / sat_s, 1),
                    "plain_queries_s": round(nq / plain_s, 1),
                    "served_over_plain": round(plain_s / sat_s, 3),
                    "served_latency_ms": {"p50": round(float(np.percentile(sat_lat, 50)), 3),
                                          "p99": round(float(np.percentile(sat_lat, 99)), 3)},
                    "plain_latency_ms": {"p50": round(float(np.percentile(plain_lat, 50)), 3),
                                         "p99": round(float(np.percentile(plain_lat, 99)), 3)},
                    "all_ok": bool(sat_ok)},
                "clocks": clk})
    return out


# ------------------------------------------------------ GPU arm: Value arrays
def run_values(args, world_size, local_rank, torch, cga):
    """The surface cloud with an RGB row per point: both halves built with
    per-voxel averaged colours, then merged with averaged overlaps."""
    from paper_2110_11616_gb300 import synth_gpu
    scene = synth_gpu.surface_scene(3)
    full = synth_gpu.sample_scene(scene, 30_000_000, seed=4)
    gen = torch.Generator(device="cuda").manual_seed(8)
    noise = torch.randint(-12, 13, full.shape, device="cuda", generator=gen, dtype=torch.int32)
    colour = ((full * 2.55).to(torch.int32) + noise).clamp(0, 255).to(torch.uint8).contiguous()
    halves = [full[0::2].contiguous(), full[1::2].contiguous()]
    cols = [colour[0::2].contiguous(), colour[1::2].contiguous()]
    del full, colour, noise
    grid = cga.grid_from_box([0, 0, 0], 100.0, 12)
    n_points = sum(h.shape[0] for h in halves)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    flush = torch.empty(args.flush_mb * (1 << 20) // 4, dtype=torch.float32, device="cuda")
    state = {}

    def step():
        ev[0].record()
        a = cga.cga_build_values(halves[0], cols[0], grid, policy="average", allocator=None)
        b = cga.cga_build_values(halves[1], cols[1], grid, policy="average", allocator=None)
        ev[1].record()
        m = cga.cga_merge_values(a, b, policy="average", allocator=None)
        ev[2].record()
        state["last"] = (a, b, m)

    def plain_step():
        a = cga.cga_build(halves[0], grid, allocator=None)
        b = cga.cga_build(halves[1], grid, allocator=None)
        cga.cga_merge(a, b, allocator=None)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = start_clocks(local_rank)
    launches0 = cga.kernel_launches()
    ms, ops = [], np.zeros(2)
    for k in range(args.steps):
        ms.append(timed(torch, step, flush, float(k)))
        ops += np.array([ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])])
    launches = cga.kernel_launches() - launches0
    plain = [timed(torch, plain_step, flush, float(k)) for k in range(max(3, args.steps // 2))]
    clk = clocks.stop()
    a, b, m = state["last"]
    u = m.info()["u"]
    total = float(sum(ms))
    op = ops / args.steps
    out = base_line(args, world_size, METRIC, n_points * args.steps / (total / 1e3) / 1e6,
                    "Mpts/s", total / args.steps,
                    {"workload": "values: 30M surface pts with an RGB row each, b=12; both "
                                 "halves built with per-voxel averaged colours, merged with "
                                 "averaged overlaps",
                     "points_per_step": n_points, "channels": 3, "l2": "flushed between steps"},
                    "synthetic (seeded GPU generators; colours from position plus noise)")
    out.update({"breakdown_ms": {"build_values": round(op[0], 4),
                                 "merge_values": round(op[1], 4)},
                "geometry_only_ms": round(float(np.mean(plain)), 4),
                "value_overhead_ms": round(total / args.steps - float(np.mean(plain)), 4),
                "merged_u": u, "gpu_launches": int(launches), "clocks": clk})
    return out


# ------------------------------------------- GPU arm: perspective projection
def run_perspective(args, world_size, local_rank, torch, cga):
    """The 30M-point surface world (19.2M voxels) rendered into a 1920 x 1080
    z-buffer from a camera turned 0.5 rad about y (Eq. 5-6)."""
    import math
    from paper_2110_11616_gb300 import synth_gpu
    scene = synth_gpu.surface_scene(3)
    full = synth_gpu.sample_scene(scene, 30_000_000, seed=4)
    grid = cga.grid_from_box([0, 0, 0], 100.0, 12)
    world = cga.cga_build(full, grid, allocator=None)
    del full
    u = world.info()["u"]
    W, H, theta, D = 1920, 1080, 0.5, 1400.0
    c, s = float(np.float32(math.cos(theta))), float(np.float32(math.sin(theta)))
    eye = [2048.0 - 6000.0 * s, 2048.0, 2048.0 - 6000.0 * c]
    flush = torch.empty(args.flush_mb * (1 << 20) // 4, dtype=torch.float32, device="cuda")
    out_img = {}

    def step():
        out_img["img"] = cga.cga_perspective(world, eye, c, s, D, W, H)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = start_clocks(local_rank)
    launches0 = cga.kernel_launches()
    ms = [timed(torch, step, flush, float(k)) for k in range(args.steps)]
    launches = cga.kernel_launches() - launches0
    clk = clocks.stop()
    idx, _ = out_img["img"]
    covered = int((idx != -1).sum())
    total = float(sum(ms))
    # algorithmic bytes: the CGA's arrays read once, the packed z-buffer
    # cleared, updated once per visible voxel and read, and both images written
    info = world.info()
    algo = info["bytes"] + W * H * (8 + 8 + 8) + u * 8
    peak, peak_kind = measured_peaks()
    out = base_line(args, world_size, METRIC, u * args.steps / (total / 1e3) / 1e6,
                    "Mvoxels/s", total / args.steps,
                    {"workload": "perspective: 19.2M-voxel surface world (30M pts, b=12), "
                                 "1920x1080 z-buffer, camera turned 0.5 rad about y",
                     "voxels": u, "pixels": W * H, "l2": "flushed between steps"},
                    "synthetic (seeded GPU generators)")
    out.update({"covered_pixels": covered,
                "achieved_GB_s": round(algo / (total / args.steps / 1e3) / 1e9, 2),
                "frac_of_hbm": round(algo / (total / args.steps / 1e3) / 1e9 / peak, 4),
                "peak_source": peak_kind, "gpu_launches": int(launches), "clocks": clk})
    return out


# ------------------------------------------- GPU arm: k-NN and radius search
def run_search(args, world_size, local_rank, torch, cga):
    """The LiDAR frame set's world (1.3M voxels, b = 16) and its 1M jittered
    queries: 8 nearest per query, and every voxel within 10 cm (25.6 voxels)."""
    scene, queries = make_workload(0)
    grid = cga.grid_from_box(LO, EXTENT, BITS)
    world = cga.cga_build(torch.from_numpy(scene.world.astype(np.float32)).cuda(), grid,
                          allocator=None)
    # prepared once (x directory, column table), as for the NN workload
    cga.cga_nn_prepare(world)
    q = torch.from_numpy(queries).cuda()
    m, k = q.shape[0], 8
    r2 = 655  # (25.6 voxels)^2: 10 cm at 3.9 mm voxels
    flush = torch.empty(args.flush_mb * (1 << 20) // 4, dtype=torch.float32, device="cuda")
    state = {}

    def knn_step():
        state["knn"] = cga.cga_knn(world, q, k)

    def radius_step():
        state["radius"] = cga.cga_radius(world, q, r2)

    def knn400_step():
        state["knn400"] = cga.cga_knn(world, q, 400)
        del state["knn400"]

    for _ in range(args.warmup):
        knn_step()
        radius_step()
        knn400_step()
    torch.cuda.synchronize()
    clocks = start_clocks(local_rank)
    launches0 = cga.kernel_launches()
    knn_ms = [timed(torch, knn_step, flush, float(i)) for i in range(args.steps)]
    rad_ms = [timed(torch, radius_step, flush, float(i)) for i in range(args.steps)]
    k400_ms = [timed(torch, knn400_step, flush, float(i)) for i in range(args.steps)]
    launches = cga.kernel_launches() - launches0
    clk = clocks.stop()
    total_results = int(state["radius"][0][-1].item())
    kt, rt = float(np.mean(knn_ms)), float(np.mean(rad_ms))
    out = base_line(args, world_size, METRIC, m * args.steps / (sum(knn_ms) / 1e3),
                    "queries/s", kt,
                    {"workload": "search: LiDAR world (1.3M voxels, b=16), 1M jittered queries; "
                                 "8-NN per query, and a radius search of 10 cm",
                     "queries": m, "k": k, "r2_voxels": r2, "l2": "flushed between steps",
                     "world_prepared": "cga_nn_prepare once before timing (column table)"},
                    "synthetic (seeded LiDAR generator)")
    out.update({"knn_ms": round(kt, 4), "radius_ms": round(rt, 4),
                "radius_queries_s": round(m / (rt / 1e3), 1),
                "radius_results": total_results,
                "radius_results_per_s": round(total_results / (rt / 1e3), 1),
                "knn400_ms": round(float(np.mean(k400_ms)), 4),
                "note": "radius_ms includes the wait for the total between count and fill",
                "gpu_launches": int(launches), "clocks": clk})
    return out


# ------------------------------------------- GPU arm: compression pieces
def run_compress(args, world_size, local_rank, torch, cga):
    """Temporal prediction of Sec. V-D on a pair of 30M-point surface frames
    (b = 12): the predicted frame is the reference moved by a rigid motion
    (1 degree about the scene's vertical axis through its centre, then a
    0.3 m shift).  One step clusters both frames (8 corner-seeded centres, at
    most 64 passes), takes the motion vectors, moves the predicted voxels and
    finds each one's corresponding voxel of the reference by exact NN."""
    import math
    from paper_2110_11616_gb300 import synth_gpu
    scene = synth_gpu.surface_scene(3)
    full = synth_gpu.sample_scene(scene, 30_000_000, seed=4)
    grid = cga.grid_from_box([0, 0, 0], 100.0, 12)
    th = math.radians(1.0)
    c, s_ = math.cos(th), math.sin(th)
    R = np.array([[c, -s_, 0.0], [s_, c, 0.0], [0.0, 0.0, 1.0]])
    ctr = np.array([50.0, 50.0, 50.0])
    t = ctr - R @ ctr + np.array([0.3, -0.2, 0.1])
    X = np.concatenate([R.reshape(9), t]).astype(np.float32)
    ref = cga.cga_build(full, grid, allocator=None)
    pred = cga.cga_build(full, grid, xform=X, allocator=None)
    del full
    ui, up = ref.info(), pred.info()
    u_ref, u_pred = ui["u"], up["u"]
    max_iter = 64
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    flush = torch.empty(args.flush_mb * (1 << 20) // 4, dtype=torch.float32, device="cuda")
    state = {}

    def step():
        ev[0].record()
        _, cr, nr, ir = cga.cga_kmeans(ref, max_iter, u=u_ref)
        ev[1].record()
        lp, cp, npd, ip = cga.cga_kmeans(pred, max_iter, u=u_pred)
        ev[2].record()
        mv = cga.cga_motion_vectors(cr, nr, cp, npd)
        rec = cga.cga_reconstruct(pred, lp, mv, u=u_pred)
        ev[3].record()
        idx, d2 = cga.cga_nn_query_voxels(ref, rec)
        ev[4].record()
        state["last"] = (ir, ip, mv, d2)
        state["rec"] = rec

    # The reference frame serves every predicted frame of its group, so its
    # search structures are prepared once, outside the step: the NN strategy
    # is measured on 1M reconstructed voxels (as points at voxel centres).
    step()
    rec = state.pop("rec")
    pick = torch.randperm(rec.shape[0], device="cuda",
                          generator=torch.Generator(device="cuda").manual_seed(3))[:1_000_000]
    sample = ((rec[pick].float() + 0.5) * (100.0 / 4096.0)).contiguous()
    nn_shifts, _ = cga.cga_nn_autotune(ref, sample)
    del rec, pick, sample
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = start_clocks(local_rank)
    launches0 = cga.kernel_launches()
    ms, ops = [], np.zeros(4)
    for k in range(args.steps):
        ms.append(timed(torch, step, flush, float(k)))
        ops += np.array([ev[i].elapsed_time(ev[i + 1]) for i in range(4)])
        state.pop("rec")
    launches = cga.kernel_launches() - launches0
    ir, ip, mv, d2 = state["last"]
    passes = (int(ir.item()), int(ip.item()))
    # one pass of the assign kernel alone: k-means of the reference stopped
    # after exactly its pass count, per pass
    per_pass = []
    for k in range(3):
        per_pass.append(timed(torch, lambda: cga.cga_kmeans(ref, passes[0], u=u_ref), flush,
                              float(k)) / passes[0])
    # CGA lookup (X_index searched) against the G-Arrays one (x indexes a dense
    # pointer array) on every stored voxel of the reference, shuffled
    vox = cga.cga_decode(ref)
    perm = torch.randperm(u_ref, device="cuda", generator=torch.Generator(device="cuda").manual_seed(1))
    qv = vox[perm].contiguous()
    xptr = cga.cga_garrays_x(ref)
    for _ in range(2):
        cga.cga_lookup(ref, qv)
        cga.cga_garrays_lookup(ref, xptr, qv)
    t_cga = min(timed(torch, lambda: cga.cga_lookup(ref, qv), flush, 1.0) for _ in range(3))
    t_ga = min(timed(torch, lambda: cga.cga_garrays_lookup(ref, xptr, qv), flush, 2.0)
               for _ in range(3))
    clk = clocks.stop()
    total = float(sum(ms))
    op = ops / args.steps
    d2h = d2.cpu().numpy()
    peak, peak_kind = measured_peaks()
    # algorithmic bytes of one assign pass: Z_index (2 B) and a label read and
    # write (1 B each) per voxel, Y_index + Y_pointer (6 B) per column and
    # X_index + X_pointer (6 B) per slab
    pass_bytes = 4 * u_ref + 6 * ui["g"] + 6 * ui["h"]
    pp = float(np.mean(per_pass))
    out = base_line(args, world_size, METRIC, u_pred * args.steps / (total / 1e3) / 1e6,
                    "Mvoxels/s", total / args.steps,
                    {"workload": "compress: two 30M-point surface frames (b=12, 19.2M voxels), "
                                 "the second under a 1-degree rotation and 0.3 m shift; k-means "
                                 "of both (8 corner seeds, <= 64 passes), motion vectors, "
                                 "reconstruction, NN correspondence of every predicted voxel",
                     "voxels_ref": u_ref, "voxels_pred": u_pred, "l2": "flushed between steps",
                     "reference_prepared": "once per reference: NN strategy autotuned on 1M "
                                           "reconstructed voxels, coarse shifts "
                                           + str(list(nn_shifts))},
                    "synthetic (seeded GPU generators)")
    out.update({"breakdown_ms": {"kmeans_ref": round(op[0], 4), "kmeans_pred": round(op[1], 4),
                                 "motion_reconstruct": round(op[2], 4),
                                 "nn_correspondence": round(op[3], 4)},
                "kmeans_passes": list(passes),
                "assign_pass_ms": round(pp, 4),
                "assign_pass_GB_s": round(pass_bytes / (pp / 1e3) / 1e9, 2),
                "assign_frac_of_hbm": round(pass_bytes / (pp / 1e3) / 1e9 / peak, 4),
                "peak_source": peak_kind,
                "motion_vectors_voxels": (mv.cpu().numpy() / 256.0).round(3).tolist(),
                "correspondence_mean_d2": round(float(d2h.mean()), 3),
                "correspondence_exact_frac": round(float((d2h == 0).mean()), 4),
                "lookup": {"queries": u_ref, "cga_ms": round(t_cga, 4), "garrays_ms": round(t_ga, 4),
                           "cga_x_bytes": 2 * ui["h"] + 4 * (ui["h"] + 1),
                           "garrays_x_bytes": 4 * ((1 << 12) + 1)},
                "gpu_launches": int(launches), "clocks": clk})
    return out


# ------------------------------------------------------------ oracle (CPU)
def oracle_step(orc, og, scene, queries, n_sample):
    t0 = time.perf_counter()
    sweeps = [orc.build(s, og, xform=p) for s, p in zip(scene.sweeps, scene.poses)]
    t1 = time.perf_counter()
    world = merge_tree(sweeps, orc.merge)
    t2 = time.perf_counter()
    orc.project(world, "xy")
    t3 = time.perf_counter()
    orc.nn_window(world, og, queries[:n_sample])
    t4 = time.perf_counter()
    orc.decode(world)
    t5 = time.perf_counter()
    nn_full = (t4 - t3) * (len(queries) / n_sample)
    return (t1 - t0) + (t2 - t1) + (t3 - t2) + nn_full + (t5 - t4), t5 - t0


LIDAR_NN_SAMPLE = 5_000


def cpu_baseline(scene, queries, n_sample=LIDAR_NN_SAMPLE):
    import oracle as orc
    og = orc.grid_from_box(LO, EXTENT, BITS)
    t, _ = oracle_step(orc, og, scene, queries, n_sample)
    pts = sum(len(s) for s in scene.sweeps)
    return {"value": round(pts / t / 1e6, 4), "unit": "Mpts/s", "cores": 1, "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": f"full build/merge/project/decode of the step; NN on {n_sample} of "
                      f"{len(queries)} queries, scaled to all"}


class OracleSurface:
    """The CPU oracle on the surface workload: the whole merged world is built
    once (untimed) for the NN sample; a step times build / merge / xy, xz, yz
    projections / decode of the first n_pts points of each half, and NN of
    the first n_surf on-surface and n_unif uniform queries against the world,
    then scales each part to the full step by its unit count."""

    def __init__(self, halves, queries):
        import oracle as orc
        self.orc = orc
        self.og = orc.grid_from_box([0.0, 0.0, 0.0], S_EXTENT, S_BITS)
        self.halves = [np.ascontiguousarray(h) for h in halves]
        self.q = np.ascontiguousarray(queries)
        self.world = orc.merge(orc.build(self.halves[0], self.og), orc.build(self.halves[1], self.og))

    def _pipeline(self, pts_a, pts_b):
        orc, og = self.orc, self.og
        a, b = orc.build(pts_a, og), orc.build(pts_b, og)
        m = orc.merge(a, b)
        for pl in ("xy", "xz", "yz"):
            orc.project(m, pl)
        orc.decode(m)

    def step(self, n_pts=S_SAMPLE_PTS, n_surf=S_SAMPLE_SURF, n_unif=S_SAMPLE_UNIF):
        """(scaled seconds for the full step, wall seconds of the sample)"""
        orc, og, h = self.orc, self.og, S_QUERIES // 2
        t0 = time.perf_counter()
        self._pipeline(self.halves[0][:n_pts], self.halves[1][:n_pts])
        t1 = time.perf_counter()
        orc.nn_window(self.world, og, self.q[:n_surf])
        t2 = time.perf_counter()
        orc.nn_window(self.world, og, self.q[h:h + n_unif])
        t3 = time.perf_counter()
        scaled = ((t1 - t0) * (S_POINTS // 2) / n_pts + (t2 - t1) * h / n_surf
                  + (t3 - t2) * h / n_unif)
        return scaled, t3 - t0

    def step_threads(self, cores, n_pts=S_SAMPLE_PTS, n_surf=S_SAMPLE_SURF, n_unif=S_SAMPLE_UNIF):
        """The same sample partitioned over `cores` threads (the oracle calls
        release the GIL): each half's points in `cores` chunks built in
        parallel and merged by a parallel merge tree, the three projections in
        parallel, and cores x the single-thread NN sample split over the
        threads.  Returns (scaled seconds for the full step, wall seconds)."""
        import concurrent.futures as cf
        orc, og, h = self.orc, self.og, S_QUERIES // 2
        with cf.ThreadPoolExecutor(max_workers=cores) as ex:
            t0 = time.perf_counter()
            parts = []
            for half in self.halves:
                pts = half[:n_pts]
                step = -(-len(pts) // cores)
                parts.append([pts[i:i + step] for i in range(0, len(pts), step)])
            built = [list(ex.map(lambda p: orc.build(p, og), ch)) for ch in parts]
            trees = []
            for lv in built:
                while len(lv) > 1:
                    pairs = [(lv[i], lv[i + 1]) for i in range(0, len(lv) - 1, 2)]
                    nxt = list(ex.map(lambda ab: orc.merge(*ab), pairs))
                    if len(lv) % 2:
                        nxt.append(lv[-1])
                    lv = nxt
                trees.append(lv[0])
            m = orc.merge(trees[0], trees[1])
            list(ex.map(lambda pl: orc.project(m, pl), ("xy", "xz", "yz")))
            orc.decode(m)
            t1 = time.perf_counter()
            ns, nu = n_surf * cores, n_unif * cores
            chunks = [self.q[i * n_surf:(i + 1) * n_surf] for i in range(cores)]
            chunks += [self.q[h + i * n_unif:h + (i + 1) * n_unif] for i in range(cores)]
            list(ex.map(lambda qq: orc.nn_window(self.world, og, qq), chunks[:cores]))
            t2 = time.perf_counter()
            list(ex.map(lambda qq: orc.nn_window(self.world, og, qq), chunks[cores:]))
            t3 = time.perf_counter()
        scaled = ((t1 - t0) * (S_POINTS // 2) / n_pts + (t2 - t1) * h / ns + (t3 - t2) * h / nu)
        return scaled, t3 - t0


def sample_text(n_pts=S_SAMPLE_PTS, n_surf=S_SAMPLE_SURF, n_unif=S_SAMPLE_UNIF, cores=1):
    return (f"build/merge/xy,xz,yz projections/decode of the first {n_pts} points of each half "
            f"(scaled by {S_POINTS // 2}/{n_pts}); NN (Sec. V-C window search) of "
            f"{n_surf * cores} on-surface and {n_unif * cores} uniform queries against the whole "
            f"merged world (scaled to 4M each)")


def cpu_baseline_surface(h_halves, h_q):
    o = OracleSurface(h_halves, h_q)
    t1, w1 = o.step()
    cores = host_cores()
    tc, wc = o.step_threads(cores)
    return {"value": round(S_POINTS / t1 / 1e6, 6), "unit": "Mpts/s", "cores": 1,
            "kind": "oracle", "cpu_model": cpu_model(), "sample": sample_text(),
            "wall_s": round(w1, 3),
            "all_cores": {"value": round(S_POINTS / tc / 1e6, 6), "unit": "Mpts/s",
                          "cores": cores, "kind": "oracle, thread-partitioned",
                          "sample": sample_text(cores=cores), "wall_s": round(wc, 3)}}


def run_reference(args):
    if args.config == "lidar":
        return run_reference_lidar(args)
    if args.config != "surface":
        return {"impl": "reference", "unavailable": f"the reference arm times the default "
                f"(surface) and lidar workloads only, not --config {args.config}"}
    import torch
    device = "cuda" if torch.cuda.is_available() else "cpu"
    halves, q = surface_inputs(device)
    o = OracleSurface([h.cpu().numpy() for h in halves], q.cpu().numpy())
    del halves, q
    for _ in range(args.warmup):
        o.step()
    runs = [o.step() for _ in range(args.steps)]
    scaled = sum(r[0] for r in runs)
    wall = sum(r[1] for r in runs)
    val = S_POINTS * args.steps / scaled / 1e6
    world_size = 1
    cfg = surface_config(args, world_size)
    return {"impl": "reference", "metric": METRIC, "value": round(val, 6), "unit": "Mpts/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(wall / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32->u16/u32/u64",
            "data": "synthetic (seeded superellipsoid surfaces, the GPU arm's inputs)"
                    + ("" if device == "cuda" else "; drawn on the host (no GPU)"),
            "config": cfg,
            "scaled_ms_per_full_step": round(scaled / args.steps * 1e3, 3),
            "note": "each step runs the oracle on the bounded sample below; ms_per_step is "
                    "that sample's wall time, value the full step's throughput with every "
                    "part scaled from the sample by its unit count",
            "cpu_baseline": {"value": round(val, 6), "unit": "Mpts/s", "cores": 1,
                             "kind": "oracle", "cpu_model": cpu_model(),
                             "sample": sample_text()},
            "e2e": {"value": round(val, 6), "unit": "Mpts/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def run_reference_lidar(args):
    scene, queries = make_workload(0)
    import oracle as orc
    og = orc.grid_from_box(LO, EXTENT, BITS)
    n_sample = LIDAR_NN_SAMPLE
    for _ in range(args.warmup):
        oracle_step(orc, og, scene, queries, n_sample)
    runs = [oracle_step(orc, og, scene, queries, n_sample) for _ in range(args.steps)]
    ts = [r[0] for r in runs]
    wall = [r[1] for r in runs]
    pts = sum(len(s) for s in scene.sweeps)
    val = pts * args.steps / sum(ts) / 1e6
    sample = (f"each step: full build/merge/project/decode; NN on {n_sample} of "
              f"{len(queries)} queries, time scaled to all")
    cfg = {"workload": WORKLOAD_LIDAR, "points_per_step": pts, "queries_per_step": N_QUERIES,
           "grid_bits": BITS, "l2": f"flushed between steps ({args.flush_mb} MB write)",
           "parallelism": "1 GPU"}
    return {"impl": "reference", "metric": METRIC, "value": round(val, 4), "unit": "Mpts/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(sum(wall) / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32->u16/u32/u64",
            "data": "synthetic", "config": cfg,
            "scaled_ms_per_full_step": round(sum(ts) / args.steps * 1e3, 3),
            "note": "ms_per_step is each sampled step's wall time; value scales the NN part "
                    "from the sample to all queries",
            "cpu_baseline": {"value": round(val, 4), "unit": "Mpts/s", "cores": 1,
                             "kind": "oracle", "cpu_model": cpu_model(), "sample": sample},
            "e2e": {"value": round(val, 4), "unit": "Mpts/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world_size = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)))
        return
    import torch
    import torch.distributed as dist
    from paper_2110_11616_gb300 import build_ext, cga
    build_ext.build()
    cga.load()
    torch.cuda.set_device(local_rank)
    if world_size > 1:
        dist.init_process_group("nccl")
    if args.config == "surface":
        out, P = run_surface(args, world_size, local_rank, torch, dist, cga)
        if rank == 0 and world_size == 1 and not args.no_cpu_baseline:
            h_halves = [h.numpy() for h in P.h_halves]
            h_q = P.h_q.numpy()
            del P
            out["cpu_baseline"] = cpu_baseline_surface(h_halves, h_q)
    elif args.config == "lidar":
        out, (scene, queries) = run_lidar(args, rank, world_size, local_rank, torch, dist, cga)
        if rank == 0 and world_size == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(scene, queries)
    elif args.config == "plain":
        out = run_single(args, world_size, local_rank, torch, cga, args.config)
    elif args.config == "batched":
        out = run_batched(args, world_size, local_rank, torch, cga)
    elif args.config == "values":
        out = run_values(args, world_size, local_rank, torch, cga)
    elif args.config == "perspective":
        out = run_perspective(args, world_size, local_rank, torch, cga)
    elif args.config == "compress":
        out = run_compress(args, world_size, local_rank, torch, cga)
    elif args.config == "search":
        out = run_search(args, world_size, local_rank, torch, cga)
    else:
        out = run_served(args, world_size, local_rank, torch, cga)
    if rank == 0:
        print(json.dumps(out))
    if world_size > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
