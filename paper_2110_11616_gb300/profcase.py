"""Profiling case for ncu: one operation of the surface workload, repeated.

The ncu summaries under profiles/ are taken on this case (a capture of one
kernel on a bounded problem, with few launches before it), not on the
benchmark loop: the surface world (seeded superellipsoid surfaces in a 100 m
cube, 12-bit grid) is built from --points points, then --op runs --repeat
times back to back:

  nn     NN queries (half on-surface, half uniform in the box; --queries in
         all) against the merged world after cga_nn_prepare_levels with the
         given strategy, in Morton order (sort once, search --repeat times;
         --presorted stores the queries in that order first).  With --world
         lidar the world is the LiDAR frame set instead (10 sweeps of 64 x
         2048 returns built with their poses and merged, 16-bit grid) and the
         queries are world points jittered by 0.2 m
  merge  the merge of the two half-cloud CGAs
  build  the batched build of the two halves

Example (ncu skips the first, warm-up launch and captures the next):

    python -m paper_2110_11616_gb300.profcase --op nn --points 30000000 \
        --queries 1000000 --repeat 2
"""
from __future__ import annotations

import argparse
import sys


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", choices=["nn", "merge", "build"], required=True)
    ap.add_argument("--world", choices=["surface", "lidar"], default="surface")
    ap.add_argument("--points", type=int, default=30_000_000)
    ap.add_argument("--queries", type=int, default=1_000_000)
    ap.add_argument("--strategy", default="tree", help='"tree", "fine" or coarse shifts "2,5"')
    ap.add_argument("--repeat", type=int, default=2)
    ap.add_argument("--radix-bits", type=int, default=9, help="launch shape of the sort passes")
    ap.add_argument("--merge-half", type=int, default=1024, help="merge partition (columns)")
    ap.add_argument("--presorted", action="store_true",
                    help="nn: store the queries in their Morton order first, so that the search "
                         "reads queries and writes results in slot order")
    args = ap.parse_args(argv)

    import torch

    from paper_2110_11616_gb300 import build_ext, cga, synth, synth_gpu
    build_ext.build()
    cga.load()
    if args.world == "lidar":
        if args.op != "nn":
            ap.error("--world lidar takes --op nn")
        sc = synth.lidar_sweeps(10, 64, 2048, seed=2)
        g = cga.grid_from_box([-128.0] * 3, 256.0, 16)
        level = cga.cga_build_batch([torch.from_numpy(x).cuda() for x in sc.sweeps], g, sc.poses,
                                    allocator=None)
        while len(level) > 1:
            nxt = cga.cga_merge_batch(level[0:len(level) - 1:2], level[1::2], allocator=None)
            if len(level) % 2:
                nxt.append(level[-1])
            level = nxt
        world = level[0]
        q = torch.from_numpy(synth.jitter_queries(sc.world, args.queries, 0.2, seed=5)).cuda()
        return _search(cga, torch, world, q, args)
    scene = synth_gpu.surface_scene(3)
    full = synth_gpu.sample_scene(scene, args.points, seed=4)
    halves = [full[0::2].contiguous(), full[1::2].contiguous()]
    del full
    grid = cga.grid_from_box([0.0, 0.0, 0.0], 100.0, 12)
    # the launch shape the benchmark's autotuner picks for this workload
    shape = {"radix_bits": args.radix_bits, "sort_threads": 512, "merge_half": args.merge_half}
    for n in (args.points // 2, args.points):
        cga.tuning_set(12, n, shape)
    if args.op == "build":
        for _ in range(args.repeat):
            cga.cga_build_batch(halves, grid, [None, None], allocator=None)
        torch.cuda.synchronize()
        return 0
    a, b = cga.cga_build_batch(halves, grid, [None, None], allocator=None)
    if args.op == "merge":
        for _ in range(args.repeat):
            cga.cga_merge(a, b, allocator=None)
        torch.cuda.synchronize()
        return 0
    mg = cga.cga_merge(a, b, allocator=None)
    del a, b, halves
    h = args.queries // 2
    q = torch.cat([synth_gpu.sample_scene(scene, h, seed=5),
                   synth_gpu.uniform_queries(args.queries - h, 6, [0.0, 0.0, 0.0], 100.0)])
    return _search(cga, torch, mg, q.contiguous(), args)


def _search(cga, torch, mg, q, args) -> int:
    if args.strategy == "fine":
        strategy = ()
    elif args.strategy == "tree":
        strategy = "tree"
    else:
        strategy = tuple(int(v) for v in args.strategy.split(","))
    cga.cga_nn_prepare(mg, strategy)
    m = q.shape[0]
    order = torch.empty(m, dtype=torch.int64, device="cuda")
    idx = torch.empty(m, dtype=torch.int32, device="cuda")
    d2 = torch.empty(m, dtype=torch.int64, device="cuda")
    cga.cga_nn_sort_queries(mg, q, order)
    if args.presorted:
        q = q[(order & 0xFFFFFFFF).long()].contiguous()
        order = None
    for _ in range(args.repeat):
        cga.cga_nn_query_ordered(mg, q, order, idx, d2)
    torch.cuda.synchronize()
    return 0


if __name__ == "__main__":
    sys.exit(main())
