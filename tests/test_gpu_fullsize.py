"""Full-size parity on the surface and batched benchmark workloads, built by
the same GPU generators and calls bench.py times.

Surface (30M points, b = 12): every CGA array of both halves, the merge, the
three projections and the decode is compared whole with the CPU oracle; NN
runs over all 8M queries with the strategy cga_nn_autotune picks (as
bench.py does), a seeded sample of 4000 on-surface and 20000 uniform queries
is compared with the oracle's window search one by one (threads over query
chunks), and every answer is checked for consistency with the decoded
voxels.

Batched (512 clouds): the pipeline is replayed from its CUDA graph; a seeded
sample of clouds (with the smallest and the largest) is compared whole with
the oracle: cloud, twin, merge, xy projection and all 4096 NN answers.
"""
import numpy as np
import oracle_threads
import pytest

from paper_2110_11616_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
LEVELS = ("X_index", "X_pointer", "Y_index", "Y_pointer", "Z_index")


@pytest.fixture(scope="module")
def cg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_11616_gb300 import build_ext, cga
    build_ext.build()
    cga.load()
    return cga


def host(t):
    return t.detach().cpu().numpy()


def assert_cga(gpu, o, what=""):
    d = gpu.download()
    for lv in LEVELS:
        np.testing.assert_array_equal(d[lv], getattr(o, lv), err_msg=f"{what} {lv}")


def assert_2d(gpu, o, what=""):
    d = gpu.download()
    for lv in ("U_index", "U_pointer", "V_index"):
        np.testing.assert_array_equal(d[lv], getattr(o, lv), err_msg=f"{what} {lv}")


def test_config_surface_30M(cg, orc):
    from paper_2110_11616_gb300 import synth_gpu
    scene = synth_gpu.surface_scene(3)
    full = synth_gpu.sample_scene(scene, 30_000_000, seed=4)
    halves = [full[0::2].contiguous(), full[1::2].contiguous()]
    del full
    grid = cg.grid_from_box([0, 0, 0], 100.0, 12)
    og = orc.grid_from_box([0, 0, 0], 100.0, 12)
    surf = synth_gpu.sample_scene(scene, 4_000_000, seed=5)
    uni = synth_gpu.uniform_queries(4_000_000, 6, [0.0, 0.0, 0.0], 100.0)
    q = torch.cat([surf, uni]).contiguous()
    m = q.shape[0]

    a, b = cg.cga_build_batch(halves, grid, [None, None], allocator=None)
    mg = cg.cga_merge(a, b, allocator=None)
    planes = ["xy", "xz", "yz"]
    pr = cg.cga_project_batch([mg] * 3, planes, allocator=None)
    # the NN strategy bench.py times: cga_nn_autotune on the same 64k sample
    gen = torch.Generator("cuda").manual_seed(7)
    sample = q[torch.randperm(m, device="cuda", generator=gen)[:65536]].contiguous()
    chosen, _ = cg.cga_nn_autotune(mg, sample, queries_per_prepare=m)
    order = torch.empty(m, dtype=torch.int64, device="cuda")
    idx = torch.empty(m, dtype=torch.int32, device="cuda")
    d2 = torch.empty(m, dtype=torch.int64, device="cuda")
    cg.cga_nn_sort_queries(mg, q, order)
    cg.cga_nn_query_ordered(mg, q, order, idx, d2)
    u = mg.info()["u"]
    dec = cg.cga_decode(mg)
    torch.cuda.synchronize()

    oa, ob = orc.build(host(halves[0]), og), orc.build(host(halves[1]), og)
    assert_cga(a, oa, "half 0")
    assert_cga(b, ob, "half 1")
    om = orc.merge(oa, ob)
    assert om.u == u
    assert_cga(mg, om, "merge")
    for p, plane in zip(pr, planes):
        assert_2d(p, orc.project(om, plane), f"project {plane}")
    ovox = orc.decode(om)
    np.testing.assert_array_equal(host(dec).astype(np.uint32), ovox)

    qh = host(q)
    gi = host(idx).view(np.uint32)
    gd = host(d2).view(np.uint64)
    # 4000 on-surface and 20000 uniform (far) queries against the oracle's
    # window search, on every host core
    rng = np.random.default_rng(9)
    pick = np.concatenate([rng.choice(m // 2, 4_000, replace=False),
                           m // 2 + rng.choice(m // 2, 20_000, replace=False)])
    oi, od = oracle_threads.nn_window(orc, om, og, qh[pick])
    np.testing.assert_array_equal(gd[pick], od, err_msg=f"sampled dist2 ({chosen})")
    np.testing.assert_array_equal(gi[pick], oi, err_msg=f"sampled idx ({chosen})")
    # every answer: a stored voxel at exactly the reported squared distance
    assert np.all(gi < u)
    qv, ok = orc.query_voxels(og, qh)
    assert ok.all()
    rd = ((qv - ovox[gi].astype(np.int64)) ** 2).sum(1).astype(np.uint64)
    np.testing.assert_array_equal(rd, gd, err_msg="dist2 inconsistent with idx")


def check_nn_sample(orc, o_cga, og, q, gi, gd, n_sample, seed, what):
    rng = np.random.default_rng(seed)
    pick = rng.choice(len(q), size=min(n_sample, len(q)), replace=False)
    oi, od = orc.nn_window(o_cga, og, q[pick])
    np.testing.assert_array_equal(gd[pick], od, err_msg=f"{what} sampled dist2")
    np.testing.assert_array_equal(gi[pick], oi, err_msg=f"{what} sampled idx")
    vox = orc.decode(o_cga).astype(np.int64)
    qv, ok = orc.query_voxels(og, q)
    assert ok.all() and np.all(gi < o_cga.u), what
    rd = ((qv - vox[gi]) ** 2).sum(1).astype(np.uint64)
    np.testing.assert_array_equal(rd, gd, err_msg=f"{what} dist2 inconsistent with idx")


def test_config_batched_512(cg, orc):
    from paper_2110_11616_gb300 import synth_gpu
    S = 512
    sizes = synth.log_uniform_ints(S, 5_000, 2_000_000, seed=41)
    bits = np.random.default_rng(42).integers(10, 17, size=S)
    pts, grids, ogrids, xforms, qs = [], [], [], [], []
    for i in range(S):
        n = int(sizes[i])
        if i % 2 == 0:
            p = synth_gpu.lidar_cloud(n, seed=1000 + i)
            box = ([-128.0] * 3, 256.0)
            qs.append(synth_gpu.jitter_queries(p, 4096, 0.2, seed=3000 + i))
        else:
            p = synth_gpu.surface_cloud(n, seed=1000 + i, n_objects=max(4, min(200, n // 5000)))
            box = ([0.0] * 3, 100.0)
            qs.append(synth_gpu.jitter_queries(p, 4096, 0.1, seed=3000 + i))
        grids.append(cg.grid_from_box(box[0], box[1], int(bits[i])))
        ogrids.append(orc.grid_from_box(box[0], box[1], int(bits[i])))
        pts.append(p)
        xforms.append(synth.rigid_xform(seed=2000 + i))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        cg.pipeline_autotune(pts, grids, xforms, qs)
        pipe = cg.Pipeline(pts, grids, xforms, qs, allocator=None)
        pipe.run_graph()
        pipe.run_graph()
    stream.synchronize()
    rng = np.random.default_rng(43)
    sample = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)),
                     *rng.choice(S, 4, replace=False).tolist()})
    for i in sample:
        ph, og = host(pts[i]), ogrids[i]
        oa, ob = orc.build(ph, og), orc.build(ph, og, xform=xforms[i])
        om = orc.merge(oa, ob)
        assert_cga(pipe.view(i, "cloud"), oa, f"cloud {i}")
        assert_cga(pipe.view(i, "twin"), ob, f"twin {i}")
        assert_cga(pipe.view(i, "merged"), om, f"merged {i}")
        assert_2d(pipe.view_xy(i), orc.project(om, "xy"), f"xy {i}")
        gi = host(pipe.idx[i]).view(np.uint32)
        gd = host(pipe.dist2[i]).view(np.uint64)
        check_nn_sample(orc, om, og, host(qs[i]), gi, gd, 300, 44 + i, f"cloud {i}")
    pipe.free()
