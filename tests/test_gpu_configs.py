"""Full-size parity on the benchmark workloads, in the launch configuration
bench.py times.

Every CGA array (builds, merges, projections, decode) is compared whole with
the CPU oracle.  NN: the plain configuration's 10k queries and all 1M LiDAR
queries are compared with the oracle's window search one by one (the LiDAR
check under the fine search, the occupancy tree and the autotuned strategy);
elsewhere a seeded sample is compared and every query's (idx, dist2) pair is
checked for consistency (dist2 is the squared distance from the query voxel
to the voxel at idx) on the whole set.
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32).reshape(-1, 3)).cuda()


def assert_cga(gpu, o, what=""):
    d = gpu.download()
    for lv in LEVELS:
        np.testing.assert_array_equal(d[lv], getattr(o, lv), err_msg=f"{what} {lv}")


def assert_2d(gpu, o, what=""):
    d = gpu.download()
    for lv in ("U_index", "U_pointer", "V_index"):
        np.testing.assert_array_equal(d[lv], getattr(o, lv), err_msg=f"{what} {lv}")


def check_nn(cg, orc, gpu_cga, o_cga, og, q, n_sample, seed):
    idx, d2 = cg.cga_nn_query(gpu_cga, dev(q))
    gi = idx.cpu().numpy().view(np.uint32)
    gd = d2.cpu().numpy().view(np.uint64)
    rng = np.random.default_rng(seed)
    pick = rng.choice(len(q), size=min(n_sample, len(q)), replace=False)
    oi, od = orc.nn_window(o_cga, og, q[pick])
    np.testing.assert_array_equal(gd[pick], od, err_msg="sampled dist2")
    np.testing.assert_array_equal(gi[pick], oi, err_msg="sampled idx")
    # whole set: idx in range and dist2 equal to the squared distance from the
    # query voxel (oracle quantization) to the voxel the GPU returned
    dec = orc.decode(o_cga).astype(np.int64)
    qv, ok = orc.query_voxels(og, q)
    assert ok.all()
    assert np.all(gi < o_cga.u)
    rd = ((qv - dec[gi]) ** 2).sum(1).astype(np.uint64)
    np.testing.assert_array_equal(rd, gd, err_msg="dist2 inconsistent with idx")
    return gi, gd


def merge_tree(items, merge):
    level = list(items)
    while len(level) > 1:
        nxt = [merge(level[i], level[i + 1]) for i in range(0, len(level) - 1, 2)]
        if len(level) % 2:
            nxt.append(level[-1])
        level = nxt
    return level[0]


def test_config_plain_100k(cg, orc):
    """100k uniform points, 10-bit grid; twin under a seeded rigid transform;
    build, merge, xy projection, 10k uniform NN queries."""
    pts = synth.uniform_cube(100_000, seed=1)
    X = synth.rigid_xform(seed=2, max_deg=10.0, max_t=0.05)
    g, og = cg.grid_from_box([0, 0, 0], 1.0, 10), orc.grid_from_box([0, 0, 0], 1.0, 10)
    a, b = cg.cga_build(dev(pts), g), cg.cga_build(dev(pts), g, xform=X)
    oa, ob = orc.build(pts, og), orc.build(pts, og, xform=X)
    assert_cga(a, oa, "A")
    assert_cga(b, ob, "B")
    m = cg.cga_merge(a, b)
    om = orc.merge(oa, ob)
    assert_cga(m, om, "merge")
    assert_2d(cg.cga_project(m, "xy"), orc.project(om, "xy"), "xy")
    q = synth.uniform_queries(10_000, 3, [0, 0, 0], 1.0)
    idx, d2 = cg.cga_nn_query(m, dev(q))
    oi, od = orc.nn_window(om, og, q)
    np.testing.assert_array_equal(d2.cpu().numpy().view(np.uint64), od)
    np.testing.assert_array_equal(idx.cpu().numpy().view(np.uint32), oi)
    bi, bd = orc.nn_brute(om, og, q[:300])
    np.testing.assert_array_equal(od[:300], bd)
    dec = cg.cga_decode(m).cpu().numpy().astype(np.uint32)
    np.testing.assert_array_equal(dec, orc.decode(om))


def test_config_lidar_frames(cg, orc):
    """10 sweeps x 64 x 2048, 16-bit grid over [-128, 128)^3 m, ego pose fused
    into each build; merge tree; xy projection; 1M jittered NN; decode."""
    scene = synth.lidar_sweeps(10, 64, 2048, seed=2)
    q = synth.jitter_queries(scene.world, 1_000_000, 0.2, seed=5)
    lo, ext = [-128.0] * 3, 256.0
    g, og = cg.grid_from_box(lo, ext, 16), orc.grid_from_box(lo, ext, 16)
    gs = [cg.cga_build(dev(s), g, xform=p) for s, p in zip(scene.sweeps, scene.poses)]
    os_ = [orc.build(s, og, xform=p) for s, p in zip(scene.sweeps, scene.poses)]
    for i, (x, y) in enumerate(zip(gs, os_)):
        assert_cga(x, y, f"sweep {i}")
    gw = merge_tree(gs, cg.cga_merge)
    ow = merge_tree(os_, orc.merge)
    assert_cga(gw, ow, "world")
    assert_2d(cg.cga_project(gw, "xy"), orc.project(ow, "xy"), "xy")
    # all 1M answers against the oracle (threads over query chunks), for the
    # fine search, the occupancy tree and the strategy cga_nn_autotune picks
    # on all the queries with the preparation charged per step (the launch
    # configuration bench.py times)
    oi, od = oracle_threads.nn_window(orc, ow, og, q)
    for prep in [(), "tree", "autotune"]:
        if prep == "autotune":
            cg.cga_nn_autotune(gw, dev(q), queries_per_prepare=len(q))
        else:
            cg.cga_nn_prepare(gw, prep)
        idx, d2 = cg.cga_nn_query(gw, dev(q))
        np.testing.assert_array_equal(d2.cpu().numpy().view(np.uint64), od, err_msg=f"{prep} dist2")
        np.testing.assert_array_equal(idx.cpu().numpy().view(np.uint32), oi, err_msg=f"{prep} idx")
    dec = cg.cga_decode(gw).cpu().numpy().astype(np.uint32)
    np.testing.assert_array_equal(dec, orc.decode(ow))
