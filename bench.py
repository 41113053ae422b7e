#!/usr/bin/env python3
"""Benchmark of the CGA hot path (libcga) on GB300.

Default workload (one "step" = one pass of the whole hot path): the LiDAR-shaped
frame set -- 10 sweeps of 64 beams x 2048 azimuth steps (1,310,720 float32
points) on a 16-bit-per-axis grid over [-128, 128)^3 m.  Per step:
  build    the 10 sweep CGAs, each with its ego pose fused into quantization
  merge    a merge tree over the sweeps (sweep t with t+1, then upwards; 9
           merges) into the world CGA
  project  the world CGA onto the xy plane
  nn       1,000,000 exact NN queries (world points + N(0, 0.2 m) jitter)
  decode   the world CGA back to voxel triples
Inputs are resident in HBM before the timed region; L2 (129 MB) is flushed
between timed steps by writing a 512 MB buffer.

python bench.py [--gpus N --steps K --warmup W] [--impl reference]
prints ONE JSON line.  --impl reference times the CPU oracle on the host cores.
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

from paper_2110_11616_gb300 import synth  # noqa: E402

METRIC = "CGA build Mpts/s, NN queries/s, merge GB/s vs HBM peak; batched vs plain"
WORKLOAD = ("LiDAR frame set: 10 sweeps x 64 beams x 2048 azimuth (1,310,720 pts), b=16, "
            "batched build (ego pose fused) + 9-merge tree (batched per level) + xy projection "
            "+ 1M jittered NN + decode")
N_SWEEPS, BEAMS, STEPS_AZ, N_QUERIES = 10, 64, 2048, 1_000_000
LO, EXTENT, BITS = (-128.0, -128.0, -128.0), 256.0, 16


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["cga", "reference"], default="cga")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--flush-mb", type=int, default=512)
    return ap.parse_args()


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


# --------------------------------------------------------------- GPU arm
class GpuPipeline:
    def __init__(self, scene, queries, torch, cga):
        self.torch, self.cga = torch, cga
        self.grid = cga.grid_from_box(LO, EXTENT, BITS)
        self.h_sweeps = [torch.from_numpy(s).pin_memory() for s in scene.sweeps]
        self.h_q = torch.from_numpy(queries).pin_memory()
        self.d_sweeps = [h.cuda() for h in self.h_sweeps]
        self.d_q = self.h_q.cuda()
        self.poses = scene.poses
        m = len(queries)
        self.idx = torch.empty(m, dtype=torch.int32, device="cuda")
        self.d2 = torch.empty(m, dtype=torch.int64, device="cuda")
        self.h_idx = torch.empty(m, dtype=torch.int32).pin_memory()
        self.h_d2 = torch.empty(m, dtype=torch.int64).pin_memory()
        self.n_points = sum(len(s) for s in scene.sweeps)
        self.dec = torch.empty((self.n_points, 3), dtype=torch.int32, device="cuda")
        self.ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]

    def step(self, timed_events=True, batched=True):
        cga = self.cga
        ev = self.ev
        if timed_events:
            ev[0].record()
        if batched:
            sweeps = cga.cga_build_batch(self.d_sweeps, self.grid, self.poses, allocator=None)
        else:
            sweeps = [cga.cga_build(d, self.grid, xform=p, allocator=None)
                      for d, p in zip(self.d_sweeps, self.poses)]
        if timed_events:
            ev[1].record()
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
        if timed_events:
            ev[2].record()
        proj = cga.cga_project(world, "xy", allocator=None)
        if timed_events:
            ev[3].record()
        cga.cga_nn_query(world, self.d_q, self.idx, self.d2)
        if timed_events:
            ev[4].record()
        cga.cga_decode(world, out=self.dec)
        if timed_events:
            ev[5].record()
        self.last = (sweeps, merges, world, proj)

    def op_times(self):
        e = self.ev
        return [e[i].elapsed_time(e[i + 1]) for i in range(5)]

    def e2e_step(self):
        for h, d in zip(self.h_sweeps, self.d_sweeps):
            d.copy_(h, non_blocking=True)
        self.d_q.copy_(self.h_q, non_blocking=True)
        self.step(timed_events=False)
        self.h_idx.copy_(self.idx, non_blocking=True)
        self.h_d2.copy_(self.d2, non_blocking=True)

    def bytes_in(self):
        return sum(h.numel() * 4 for h in self.h_sweeps) + self.h_q.numel() * 4

    def bytes_out(self):
        return self.h_idx.numel() * 4 + self.h_d2.numel() * 8


def cga_bytes(info):
    return info["bytes"]


def run_gpu(args, rank, world_size, local_rank):
    import torch
    import torch.distributed as dist
    from paper_2110_11616_gb300 import build_ext, cga

    build_ext.build()
    cga.load()
    torch.cuda.set_device(local_rank)
    scene, queries = make_workload(rank)
    P = GpuPipeline(scene, queries, torch, cga)
    flush = torch.empty(args.flush_mb * (1 << 20) // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if world_size > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        P.step()
    torch.cuda.synchronize()
    phys = os.environ.get("CUDA_VISIBLE_DEVICES", str(local_rank)).split(",")[local_rank]
    clocks = Clocks(int(phys) if phys.isdigit() else local_rank)
    time.sleep(0.3)
    start_ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    end_ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    op_ms = np.zeros(5)
    launches0 = cga.kernel_launches()
    barrier()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))
        start_ev[k].record()
        P.step()
        end_ev[k].record()
        end_ev[k].synchronize()
        op_ms += np.array(P.op_times())
    barrier()
    t_wall = time.perf_counter() - t_wall
    launches = cga.kernel_launches() - launches0
    step_ms = [s.elapsed_time(e) for s, e in zip(start_ev, end_ev)]
    total_ms = float(sum(step_ms))

    # the same step as one call per cloud / per merge (the plain form)
    plain_ms = []
    for k in range(max(3, args.steps // 2)):
        flush.fill_(float(k))
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record()
        P.step(timed_events=False, batched=False)
        e.record()
        e.synchronize()
        plain_ms.append(s.elapsed_time(e))

    # end to end: host (pinned) inputs -> device -> results back to host
    e2e_ms = []
    for k in range(max(3, args.steps // 3)):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record()
        P.e2e_step()
        e.record()
        e.synchronize()
        e2e_ms.append(s.elapsed_time(e))
    clk = clocks.stop()

    # sizes of the last step for the derived numbers
    sweeps, merges, world, proj = P.last
    winfo = world.info()
    merge_bytes = 0
    for a, b, m in merges:
        merge_bytes += cga_bytes(a.info()) + cga_bytes(b.info()) + cga_bytes(m.info())
    op = op_ms / args.steps
    max_total = total_ms
    if world_size > 1:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        max_total = float(t.item())
    pts = P.n_points
    value = pts * args.steps * world_size / (max_total / 1e3) / 1e6
    e2e_val = pts * world_size / (float(np.mean(e2e_ms)) / 1e3) / 1e6
    out = {
        "metric": METRIC,
        "value": round(value, 3),
        "unit": "Mpts/s",
        "n_gpus": world_size,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(max_total / args.steps, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32->u16/u32/u64",
        "data": "synthetic (seeded LiDAR generator; stands in for the paper's LiDAR scans)",
        "config": {"workload": WORKLOAD, "points_per_step": pts, "queries_per_step": N_QUERIES,
                   "grid_bits": BITS, "l2": f"flushed between steps ({args.flush_mb} MB write)",
                   "parallelism": f"replicas x{world_size}" if world_size > 1 else "1 GPU"},
        "breakdown_ms": {"build": round(op[0], 4), "merge": round(op[1], 4),
                         "project_xy": round(op[2], 4), "nn": round(op[3], 4),
                         "decode": round(op[4], 4)},
        "derived": {
            "build_Mpts_s": round(pts / (op[0] / 1e3) / 1e6, 2),
            "nn_queries_s": round(N_QUERIES / (op[3] / 1e3), 1),
            "merge_GB_s": round(merge_bytes / (op[1] / 1e3) / 1e9, 2),
            "merge_compulsory_bytes": merge_bytes,
            "world_u": winfo["u"], "world_g": winfo["g"], "world_h": winfo["h"],
            "world_bytes": winfo["bytes"], "raw_bytes": pts * 12,
        },
        "e2e": {"value": round(e2e_val, 3), "unit": "Mpts/s",
                "h2d_bytes_per_step": P.bytes_in(), "d2h_bytes_per_step": P.bytes_out()},
        "plain": {"ms_per_step": round(float(np.mean(plain_ms)), 4),
                  "value": round(pts / (float(np.mean(plain_ms)) / 1e3) / 1e6, 3),
                  "note": "one call per sweep build and per merge (the step above batches "
                          "the 10 builds and each merge-tree level into one launch set)"},
        "gpu_launches": int(launches),
        "clocks": clk,
        "wall_s": round(t_wall, 3),
    }
    return out, P


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
    return (t1 - t0) + (t2 - t1) + (t3 - t2) + nn_full + (t5 - t4)


def cpu_baseline(scene, queries, n_sample=20_000):
    import oracle as orc
    og = orc.grid_from_box(LO, EXTENT, BITS)
    t = oracle_step(orc, og, scene, queries, n_sample)
    pts = sum(len(s) for s in scene.sweeps)
    return {"value": round(pts / t / 1e6, 4), "unit": "Mpts/s", "cores": 1, "kind": "oracle",
            "sample": f"full build/merge/project/decode of the step; NN on {n_sample} of "
                      f"{len(queries)} queries, scaled to all"}


def run_reference(args, rank):
    scene, queries = make_workload(0)
    import oracle as orc
    og = orc.grid_from_box(LO, EXTENT, BITS)
    n_sample = 5_000
    for _ in range(args.warmup):
        oracle_step(orc, og, scene, queries, n_sample)
    ts = [oracle_step(orc, og, scene, queries, n_sample) for _ in range(args.steps)]
    pts = sum(len(s) for s in scene.sweeps)
    val = pts * args.steps / sum(ts) / 1e6
    sample = (f"each step: full build/merge/project/decode; NN on {n_sample} of "
              f"{len(queries)} queries, time scaled to all")
    return {"impl": "reference", "metric": METRIC, "value": round(val, 4), "unit": "Mpts/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(sum(ts) / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32->u16/u32/u64",
            "data": "synthetic", "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": round(val, 4), "unit": "Mpts/s", "cores": 1,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(val, 4), "unit": "Mpts/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world_size = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, rank)))
        return
    if world_size > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    out, P = run_gpu(args, rank, world_size, local_rank)
    if rank == 0 and world_size == 1 and not args.no_cpu_baseline:
        scene, queries = make_workload(0)
        out["cpu_baseline"] = cpu_baseline(scene, queries)
    if rank == 0:
        print(json.dumps(out))
    if world_size > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
