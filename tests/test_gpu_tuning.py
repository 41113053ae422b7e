"""GPU parity under every launch shape the autotuner can pick: the digit width
(8 or 9 bits, so 30-, 36- and 48-bit keys take different pass counts), the
threads per tile and the merge-path partition change only the speed, never a
bit of any result.  Each case sets the shape for every table entry, runs the
operations and compares them with the CPU oracle, then restores the
defaults."""
import itertools

import numpy as np
import pytest

from paper_2110_11616_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
LEVELS = ("X_index", "X_pointer", "Y_index", "Y_pointer", "Z_index")
TILE = 4096
SORTS = [(8, 256), (8, 512), (9, 512)]
HALVES = [512, 1024, 2048]


@pytest.fixture(scope="module")
def cg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_11616_gb300 import build_ext, cga
    build_ext.build()
    cga.load()
    return cga


def set_all(cg, shape):
    for bits in range(1, 17):
        for nb in range(0, 32):
            cg.tuning_set(bits, (1 << (nb - 1)) if nb else 0, shape)


@pytest.fixture()
def shaped(cg):
    yield lambda shape: set_all(cg, shape)
    set_all(cg, None)


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


@pytest.mark.parametrize("sort,half", list(itertools.product(SORTS, HALVES)))
@pytest.mark.parametrize("bits", [10, 12, 16])
def test_shape_build_merge_project(cg, orc, shaped, sort, half, bits):
    shaped({"radix_bits": sort[0], "sort_threads": sort[1], "merge_half": half})
    n = 5 * TILE + 123
    pts = synth.uniform_cube(n, seed=bits * 7 + half, lo=-0.02, extent=1.04)
    X = synth.rigid_xform(seed=bits + half)
    g, og = cg.grid_from_box([0, 0, 0], 1.0, bits), orc.grid_from_box([0, 0, 0], 1.0, bits)
    a, b = cg.cga_build(dev(pts), g), cg.cga_build(dev(pts[: n // 3]), g, xform=X)
    oa, ob = orc.build(pts, og), orc.build(pts[: n // 3], og, xform=X)
    assert_cga(a, oa, "build")
    assert_cga(b, ob, "build twin")
    m = cg.cga_merge(a, b)
    om = orc.merge(oa, ob)
    assert_cga(m, om, "merge")
    for plane in ("xy", "xz", "yz"):
        assert_2d(cg.cga_project(m, plane), orc.project(om, plane), plane)
    # NN over a coarse level, which is built by the same sort kernels
    cg.cga_nn_prepare(m, (2,))
    q = synth.uniform_queries(3000, bits, [-0.1] * 3, 1.2)
    idx, d2 = cg.cga_nn_query(m, dev(q))
    oi, od = orc.nn_window(om, og, q)
    np.testing.assert_array_equal(d2.cpu().numpy().view(np.uint64), od)
    np.testing.assert_array_equal(idx.cpu().numpy().view(np.uint32), oi)


@pytest.mark.parametrize("half", HALVES)
def test_merge_dense_and_sparse_tiles(cg, orc, shaped, half):
    """One merge whose tiles take both tile paths: voxel by voxel where the
    columns hold few voxels, column by column across blocks of full columns
    (more voxels per tile than the voxel-level stage holds), with columns of
    both blocks overlapping so that their z lists are united."""
    shaped({"radix_bits": 8, "sort_threads": 256, "merge_half": half})
    bits = 10
    g, og = cg.make_grid(bits, 1.0, (0.0, 0.0, 0.0)), orc.Grid(bits, 1.0, (0.0, 0.0, 0.0))
    rng = np.random.default_rng(half)
    sparse = rng.integers(0, 1 << bits, (80_000, 3)).astype(np.float32) + 0.5
    v = np.stack(np.meshgrid(np.arange(300, 348), np.arange(500, 540), np.arange(100, 148),
                             indexing="ij"), -1).reshape(-1, 3).astype(np.float32) + 0.5
    pa = np.concatenate([sparse[:40_000], v])
    pb = np.concatenate([sparse[40_000:], v[::2] + np.float32([0, 10, 20])])
    oa, ob = orc.build(pa, og), orc.build(pb, og)
    m = cg.cga_merge(cg.cga_build(dev(pa), g), cg.cga_build(dev(pb), g))
    om = orc.merge(oa, ob)
    assert_cga(m, om, "merge")
    assert_cga(cg.cga_merge(cg.cga_build(dev(pb), g), cg.cga_build(dev(pa), g)), om, "merge B, A")


@pytest.mark.parametrize("shape", [(8, 256, 512), (9, 512, 1024), (9, 512, 2048)])
def test_shape_batches_and_graph_pipeline(cg, orc, shaped, shape):
    shaped(dict(zip(("radix_bits", "sort_threads", "merge_half"), shape)))
    specs = [(0, 10), (1, 16), (3 * TILE + 1, 12), (60_000, 16), (TILE, 11), (20_000, 14)]
    items = []
    for i, (n, bits) in enumerate(specs):
        items.append((synth.uniform_cube(n, seed=300 + i, lo=-0.03, extent=1.06),
                      synth.rigid_xform(seed=310 + i), cg.grid_from_box([0, 0, 0], 1.0, bits),
                      orc.grid_from_box([0, 0, 0], 1.0, bits)))
    pts = [dev(p) for p, _, _, _ in items]
    grids = [g for _, _, g, _ in items]
    A = cg.cga_build_batch(pts, grids)
    B = cg.cga_build_batch(pts, grids, [X for _, X, _, _ in items])
    M = cg.cga_merge_batch(A, B)
    oms = []
    for i, (p, X, _, og) in enumerate(items):
        om = orc.merge(orc.build(p, og), orc.build(p, og, xform=X))
        assert_cga(M[i], om, f"merge {i}")
        oms.append(om)
    planes = ["xz", "yz", "xy", "xz", "yz", "xy"]
    P = cg.cga_project_batch(M, planes)
    for i, (om, pl) in enumerate(zip(oms, planes)):
        assert_2d(P[i], orc.project(om, pl), f"project {i} {pl}")
    pipe = cg.Pipeline(pts, grids, [X for _, X, _, _ in items], [None] * len(items))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        pipe.run_graph()
    stream.synchronize()
    for i, om in enumerate(oms):
        assert_cga(pipe.view(i, "merged"), om, f"pipeline merged {i}")
    pipe.free()


def test_autotune_picks_a_candidate_and_keeps_results(cg, orc, shaped):
    shaped(None)
    pts = synth.uniform_cube(200_000, seed=77)
    g, og = cg.grid_from_box([0, 0, 0], 1.0, 12), orc.grid_from_box([0, 0, 0], 1.0, 12)
    shape, times = cg.cga_autotune(dev(pts), g)
    assert (shape["radix_bits"], shape["sort_threads"]) in times["sort"]
    assert shape["merge_half"] in times["merge"]
    assert min(times["sort"], key=times["sort"].get) == (shape["radix_bits"], shape["sort_threads"])
    assert min(times["merge"], key=times["merge"].get) == shape["merge_half"]
    assert all(t > 0 for t in list(times["sort"].values()) + list(times["merge"].values()))
    assert cg.tuning_get(12, 200_000) == shape
    a = cg.cga_build(dev(pts), g)
    assert_cga(a, orc.build(pts, og))
    h = len(pts) // 2
    assert_cga(cg.cga_merge(cg.cga_build(dev(pts[:h]), g), cg.cga_build(dev(pts[h:]), g)),
               orc.build(pts, og))


def test_pipeline_autotune_keeps_results(cg, orc, shaped):
    shaped(None)
    specs = [(30_000, 12), (3 * TILE + 5, 16), (0, 10), (9_000, 14)]
    items = []
    for i, (n, bits) in enumerate(specs):
        items.append((synth.uniform_cube(n, seed=400 + i, lo=-0.03, extent=1.06),
                      synth.rigid_xform(seed=410 + i), cg.grid_from_box([0, 0, 0], 1.0, bits),
                      orc.grid_from_box([0, 0, 0], 1.0, bits)))
    pts = [dev(p) for p, _, _, _ in items]
    grids = [g for _, _, g, _ in items]
    xs = [X for _, X, _, _ in items]
    qs = [dev(synth.uniform_queries(700, 420 + i, [-0.1] * 3, 1.2)) for i in range(len(items))]
    shape, times = cg.pipeline_autotune(pts, grids, xs, qs)
    assert min(times["sort"], key=times["sort"].get) == (shape["radix_bits"], shape["sort_threads"])
    assert min(times["merge"], key=times["merge"].get) == shape["merge_half"]
    assert cg.tuning_get(16, 30_000) == shape
    pipe = cg.Pipeline(pts, grids, xs, qs)
    pipe.run_graph()
    torch.cuda.synchronize()
    for i, (p, X, _, og) in enumerate(items):
        om = orc.merge(orc.build(p, og), orc.build(p, og, xform=X))
        assert_cga(pipe.view(i, "merged"), om, f"merged {i}")
        oi, od = orc.nn_window(om, og, qs[i].cpu().numpy())
        np.testing.assert_array_equal(pipe.dist2[i].cpu().numpy().view(np.uint64), od)
        np.testing.assert_array_equal(pipe.idx[i].cpu().numpy().view(np.uint32), oi)
    pipe.free()
