"""GPU parity: every libcga result equals the CPU oracle's, element by element.

All outputs are integers, so the bar is bit-exact equality.  Sizes span
several 4096-key tiles with ragged tails, the empty and one-point clouds, all
duplicates, grids of 1..16 bits (both the 32-bit and the 64-bit key paths),
points outside the box, non-finite input, ties in NN, and queries far outside
the box.
"""
import numpy as np
import pytest

from paper_2110_11616_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
LEVELS = ("X_index", "X_pointer", "Y_index", "Y_pointer", "Z_index")
TILE = 4096


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


def grids(cg, orc, lo, ext, bits):
    return cg.grid_from_box(lo, ext, bits), orc.grid_from_box(lo, ext, bits)


def assert_cga(gpu, o, what=""):
    d = gpu.download()
    for lv in LEVELS:
        np.testing.assert_array_equal(d[lv], getattr(o, lv), err_msg=f"{what} {lv}")


def assert_2d(gpu, o, what=""):
    d = gpu.download()
    for lv in ("U_index", "U_pointer", "V_index"):
        np.testing.assert_array_equal(d[lv], getattr(o, lv), err_msg=f"{what} {lv}")


def nn_check(cg, orc, gpu_cga, o_cga, og, q, brute=True):
    idx, d2 = cg.cga_nn_query(gpu_cga, dev(q))
    gi = idx.cpu().numpy().view(np.uint32)
    gd = d2.cpu().numpy().view(np.uint64)
    oi, od = (orc.nn_brute if brute else orc.nn_window)(o_cga, og, q)
    np.testing.assert_array_equal(gd, od, err_msg="dist2")
    np.testing.assert_array_equal(gi, oi, err_msg="idx")


# ------------------------------------------------------------------- build
@pytest.mark.parametrize("n", [0, 1, 2, 100, TILE - 1, TILE, TILE + 1, 3 * TILE + 17, 100_000])
@pytest.mark.parametrize("bits", [10, 16])
def test_build_sizes(cg, orc, n, bits):
    pts = synth.uniform_cube(n, seed=100 + n, lo=-0.02, extent=1.04)
    g, og = grids(cg, orc, [0, 0, 0], 1.0, bits)
    a = cg.cga_build(dev(pts), g)
    assert_cga(a, orc.build(pts, og), f"n={n} b={bits}")
    assert a.info()["u"] == orc.build(pts, og).u


@pytest.mark.parametrize("bits", [1, 2, 3, 5, 7, 8, 9, 11, 12, 13, 14, 15])
def test_build_bits(cg, orc, bits):
    pts = synth.uniform_cube(50_000, seed=bits, lo=-0.1, extent=1.2)
    g, og = grids(cg, orc, [0, 0, 0], 1.0, bits)
    assert_cga(cg.cga_build(dev(pts), g), orc.build(pts, og), f"b={bits}")


@pytest.mark.parametrize("bits", [10, 16])
def test_build_transform(cg, orc, bits):
    pts = synth.uniform_cube(70_000, seed=5)
    X = synth.rigid_xform(seed=6)
    g, og = grids(cg, orc, [0, 0, 0], 1.0, bits)
    assert_cga(cg.cga_build(dev(pts), g, xform=X), orc.build(pts, og, xform=X))


def test_build_all_duplicates(cg, orc):
    pts = np.tile(np.array([[0.25, 0.5, 0.75]], np.float32), (3 * TILE + 5, 1))
    g, og = grids(cg, orc, [0, 0, 0], 1.0, 12)
    a = cg.cga_build(dev(pts), g)
    assert_cga(a, orc.build(pts, og))
    assert a.info()["u"] == 1


def test_build_fmaf_boundary_case(cg, orc):
    # exact p*s + o is just below 14; a separate multiply and add gives 14.
    p, s, o = 2.043496608734131, 1274.286376953125, -2590.0
    g = cg.make_grid(10, s, (o, o, o))
    og = orc.Grid(10, float(np.float32(s)), (float(np.float32(o)),) * 3)
    pts = np.array([[p, p, p]], np.float32)
    a = cg.cga_build(dev(pts), g)
    assert_cga(a, orc.build(pts, og))
    assert list(a.download()["X_index"]) == [13]


def test_build_lidar_sweep_with_pose(cg, orc):
    scene = synth.lidar_sweeps(n_sweeps=2, beams=64, steps=512, seed=7, with_world=False)
    g, og = grids(cg, orc, [-128, -128, -128], 256.0, 16)
    for pts, pose in zip(scene.sweeps, scene.poses):
        assert_cga(cg.cga_build(dev(pts), g, xform=pose), orc.build(pts, og, xform=pose))


def test_build_nonfinite_is_reported(cg, orc):
    pts = synth.uniform_cube(10_000, seed=9)
    pts[7777, 1] = np.nan
    g, _ = grids(cg, orc, [0, 0, 0], 1.0, 10)
    a = cg.cga_build(dev(pts), g)
    assert a.status() == cg.ERR_NONFINITE
    pts[7777, 1] = 0.5
    X = np.array([3e38, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0], np.float32)
    pts[5, 0] = 10.0
    b = cg.cga_build(dev(pts), g, xform=X)
    assert b.status() == cg.ERR_NONFINITE
    assert cg.cga_merge(b, b).status() == cg.ERR_NONFINITE


def test_full_lattice_closed_form(cg):
    k = 40
    ax = np.arange(k, dtype=np.float32)
    vox = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1).reshape(-1, 3)
    vox = vox[np.random.default_rng(0).permutation(len(vox))]
    a = cg.cga_build(dev(vox), cg.make_grid(6, 1.0, (0.0, 0.0, 0.0)))
    d = a.download()
    assert np.array_equal(d["X_index"], np.arange(k))
    assert np.array_equal(d["X_pointer"], np.arange(k + 1) * k)
    assert np.array_equal(d["Y_index"], np.tile(np.arange(k), k))
    assert np.array_equal(d["Y_pointer"], np.arange(k * k + 1) * k)
    assert np.array_equal(d["Z_index"], np.tile(np.arange(k), k * k))


# ------------------------------------------------------------------- merge
@pytest.mark.parametrize("na,nb", [(0, 0), (0, 5000), (5000, 0), (1, 1), (20_000, 3),
                                   (40_000, 60_000), (3 * TILE + 1, 2 * TILE - 1)])
@pytest.mark.parametrize("bits", [10, 16])
def test_merge_parity(cg, orc, na, nb, bits):
    pa = synth.uniform_cube(na, seed=11)
    pb = synth.uniform_cube(nb, seed=12)
    X = synth.rigid_xform(seed=13)
    g, og = grids(cg, orc, [0, 0, 0], 1.0, bits)
    a, b = cg.cga_build(dev(pa), g), cg.cga_build(dev(pb), g, xform=X)
    m = cg.cga_merge(a, b)
    om = orc.merge(orc.build(pa, og), orc.build(pb, og, xform=X))
    assert_cga(m, om, f"merge {na}+{nb}")


def test_merge_identities(cg, orc):
    pa = synth.uniform_cube(30_000, seed=21)
    g, og = grids(cg, orc, [0, 0, 0], 1.0, 8)   # 256^3: many shared voxels
    a = cg.cga_build(dev(pa), g)
    oa = orc.build(pa, og)
    assert_cga(cg.cga_merge(a, a), oa, "A u A")
    pb = synth.uniform_cube(30_000, seed=22)
    b = cg.cga_build(dev(pb), g)
    ob = orc.build(pb, og)
    assert_cga(cg.cga_merge(b, a), orc.merge(oa, ob), "B u A")
    mm = cg.cga_merge(cg.cga_merge(a, b), cg.cga_merge(b, a))
    assert_cga(mm, orc.merge(oa, ob), "(A u B) u (B u A)")


def test_merge_disjoint_and_interleaved(cg, orc):
    g, og = grids(cg, orc, [0, 0, 0], 1.0, 12)
    lo = synth.uniform_cube(25_000, seed=31, lo=0.0, extent=0.5)
    hi = synth.uniform_cube(25_000, seed=32, lo=0.5, extent=0.5)
    for pa, pb in ((lo, hi), (hi, lo)):
        m = cg.cga_merge(cg.cga_build(dev(pa), g), cg.cga_build(dev(pb), g))
        assert_cga(m, orc.merge(orc.build(pa, og), orc.build(pb, og)))
    # interleaved slabs: even x voxels in A, odd in B
    v = np.stack(np.meshgrid(np.arange(64), np.arange(16), np.arange(16), indexing="ij"),
                 -1).reshape(-1, 3).astype(np.float32)
    ev, od = v[v[:, 0] % 2 == 0], v[v[:, 0] % 2 == 1]
    ug = cg.make_grid(7, 1.0, (0.0, 0.0, 0.0))
    oug = orc.Grid(7, 1.0, (0.0, 0.0, 0.0))
    m = cg.cga_merge(cg.cga_build(dev(ev), ug), cg.cga_build(dev(od), ug))
    assert_cga(m, orc.merge(orc.build(ev, oug), orc.build(od, oug)))


def test_merge_grid_mismatch(cg):
    pa = synth.uniform_cube(100, seed=41)
    a = cg.cga_build(dev(pa), cg.grid_from_box([0, 0, 0], 1.0, 10))
    b = cg.cga_build(dev(pa), cg.grid_from_box([0, 0, 0], 1.0, 11))
    c = cg.cga_build(dev(pa), cg.grid_from_box([0, 0, 0.001], 1.0, 10))
    for other in (b, c):
        with pytest.raises(cg.CgaError) as e:
            cg.cga_merge(a, other)
        assert e.value.code == cg.ERR_GRID_MISMATCH


# -------------------------------------------------------------- projection
@pytest.mark.parametrize("plane", ["xy", "xz", "yz"])
@pytest.mark.parametrize("bits,n", [(4, 3000), (5, 3000), (10, 100_000), (12, 50_000),
                                    (13, 40_000), (14, 20_000), (16, 20_000), (16, 0), (10, 1),
                                    (12, 0)])
def test_project_parity(cg, orc, plane, bits, n):
    """xy copies the top two levels; xz and yz go through a bitmap of the 2D
    voxels on grids of 5 to 13 bits and through the sort pipeline otherwise
    (both edges of that range, empty and single-point clouds included)."""
    pts = synth.uniform_cube(n, seed=50 + bits)
    g, og = grids(cg, orc, [0, 0, 0], 1.0, bits)
    a = cg.cga_build(dev(pts), g)
    assert_2d(cg.cga_project(a, plane), orc.project(orc.build(pts, og), plane), plane)


# ---------------------------------------------------------------------- NN
@pytest.mark.parametrize("bits,n", [(4, 50), (6, 2000), (10, 20_000), (16, 5000)])
def test_nn_parity_small(cg, orc, bits, n):
    pts = synth.uniform_cube(n, seed=60 + bits)
    g, og = grids(cg, orc, [0, 0, 0], 1.0, bits)
    a = cg.cga_build(dev(pts), g)
    oa = orc.build(pts, og)
    q = np.concatenate([synth.uniform_queries(2000, 61, [0, 0, 0], 1.0),
                        synth.uniform_queries(300, 62, [-2, -2, -2], 5.0),
                        pts[:300]])
    nn_check(cg, orc, a, oa, og, q, brute=n * len(q) < 3e7)


def test_nn_ties_and_sentinels(cg, orc):
    ug = cg.make_grid(4, 1.0, (0.0, 0.0, 0.0))
    oug = orc.Grid(4, 1.0, (0.0, 0.0, 0.0))
    vox = np.array([[6, 5, 5], [5, 6, 5], [5, 5, 6], [4, 5, 5], [5, 4, 5], [0, 0, 0], [2, 0, 0],
                    [0, 2, 9], [0, 0, 11]], np.float32)
    a = cg.cga_build(dev(vox), ug)
    oa = orc.build(vox, oug)
    q = np.array([[5, 5, 5], [1, 0, 0], [0, 1, 10], [np.nan, 1, 1], [1, np.inf, 1],
                  [-100, -100, -100], [3.5, 3.5, 3.5]], np.float32)
    nn_check(cg, orc, a, oa, oug, q)
    empty = cg.cga_build(dev(np.zeros((0, 3), np.float32)), ug)
    idx, d2 = cg.cga_nn_query(empty, dev(q))
    assert np.all(idx.cpu().numpy().view(np.uint32) == 0xFFFFFFFF)
    assert np.all(d2.cpu().numpy().view(np.uint64) == np.uint64(0xFFFFFFFFFFFFFFFF))


def test_nn_full_lattice(cg, orc):
    k = 20
    ax = np.arange(k, dtype=np.float32)
    vox = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1).reshape(-1, 3)
    a = cg.cga_build(dev(vox), cg.make_grid(5, 1.0, (0.0, 0.0, 0.0)))
    q = np.random.default_rng(3).uniform(-40, 60, size=(5000, 3)).astype(np.float32)
    idx, d2 = cg.cga_nn_query(a, dev(q))
    qi = np.floor(q.astype(np.float64)).astype(np.int64)
    c = np.clip(qi, 0, k - 1)
    assert np.array_equal(d2.cpu().numpy(), ((qi - c) ** 2).sum(1))
    assert np.array_equal(idx.cpu().numpy().astype(np.int64), c[:, 0] * k * k + c[:, 1] * k + c[:, 2])


# ------------------------------------------------------------------ decode
@pytest.mark.parametrize("bits,n", [(10, 100_000), (16, 3 * TILE + 3), (3, 500), (10, 0)])
def test_decode_parity(cg, orc, bits, n):
    pts = synth.uniform_cube(n, seed=70 + n)
    g, og = grids(cg, orc, [0, 0, 0], 1.0, bits)
    a = cg.cga_build(dev(pts), g)
    got = cg.cga_decode(a).cpu().numpy().astype(np.uint32).reshape(-1, 3)
    np.testing.assert_array_equal(got, orc.decode(orc.build(pts, og)))


def test_nn_two_step_equals_one_call(cg, orc):
    pts = synth.uniform_cube(60_000, seed=91)
    g, og = grids(cg, orc, [0, 0, 0], 1.0, 11)
    a = cg.cga_build(dev(pts), g)
    q = dev(synth.uniform_queries(50_000, 92, [-0.1] * 3, 1.2))
    order = cg.cga_nn_sort_queries(a, q)
    keys = order.cpu().numpy().view(np.uint64)
    assert np.all(np.diff(keys.astype(np.float64)) >= 0) or np.all(keys[1:] >= keys[:-1])
    assert np.array_equal(np.sort(keys & np.uint64(0xFFFFFFFF)), np.arange(len(keys), dtype=np.uint64))
    idx = torch.empty(50_000, dtype=torch.int32, device="cuda")
    d2 = torch.empty(50_000, dtype=torch.int64, device="cuda")
    cg.cga_nn_query_ordered(a, q, order, idx, d2)
    ri, rd = cg.cga_nn_query(a, q)
    assert torch.equal(idx, ri) and torch.equal(d2, rd)
    idx2 = torch.empty_like(idx)
    d22 = torch.empty_like(d2)
    cg.cga_nn_query_ordered(a, q, None, idx2, d22)   # query order
    assert torch.equal(idx2, ri) and torch.equal(d22, rd)


@pytest.mark.parametrize("shift", [1, 2, 3, 5, (1, 2), (2, 5), (3, 7), (4, 9)])
@pytest.mark.parametrize("kind", ["uniform", "surface", "lidar"])
def test_nn_two_level_parity(cg, orc, shift, kind):
    """NN after cga_nn_prepare (one or two coarse levels, cells of 2^shift
    voxels) equals the oracle, for queries near the points, uniform in the box
    and far outside it."""
    if kind == "uniform":
        pts = synth.uniform_cube(30_000, seed=95)
        lo, ext, bits = [0.0] * 3, 1.0, 10
    elif kind == "surface":
        scene = synth.superellipsoid_scene(n_objects=12, seed=96, extent=100.0)
        pts = synth.sample_surfaces(scene, 60_000, seed=97)
        lo, ext, bits = [0.0] * 3, 100.0, 12
    else:
        sc = synth.lidar_sweeps(2, 64, 512, seed=98)
        pts = sc.world.astype(np.float32)
        lo, ext, bits = [-128.0] * 3, 256.0, 16
    g, og = grids(cg, orc, lo, ext, bits)
    a = cg.cga_build(dev(pts), g)
    cg.cga_nn_prepare(a, shift)
    oa = orc.build(pts, og)
    lo_a = np.asarray(lo, np.float64)
    q = np.concatenate([
        (pts[:1500].astype(np.float64) + np.random.default_rng(1).normal(0, ext / 200, (1500, 3))),
        synth.uniform_queries(1500, 99, lo, ext),
        synth.uniform_queries(200, 100, lo_a - ext, 3 * ext),
    ]).astype(np.float32)
    nn_check(cg, orc, a, oa, og, q, brute=False)
    # the same with the queries sorted (large batch path)
    idx, d2 = cg.cga_nn_query(a, dev(np.tile(q, (4, 1))))
    oi, od = orc.nn_window(oa, og, q)
    assert np.array_equal(d2.cpu().numpy().view(np.uint64), np.tile(od, 4))
    assert np.array_equal(idx.cpu().numpy().view(np.uint32), np.tile(oi, 4))


def test_nn_autotune_keeps_results(cg, orc):
    scene = synth.superellipsoid_scene(n_objects=10, seed=120, extent=100.0)
    pts = synth.sample_surfaces(scene, 80_000, seed=121)
    g, og = grids(cg, orc, [0.0] * 3, 100.0, 12)
    a = cg.cga_build(dev(pts), g)
    q = np.concatenate([synth.sample_surfaces(scene, 2000, seed=122),
                        synth.uniform_queries(2000, 123, [0.0] * 3, 100.0)])
    shifts, times = cg.cga_nn_autotune(a, dev(q))
    assert shifts in times and min(times, key=times.get) == shifts
    assert set(times) == set(cg.NN_AUTOTUNE_CANDIDATES)
    nn_check(cg, orc, a, orc.build(pts, og), og, q, brute=False)
    # a small grid cannot take the deepest candidates: they report no time
    g6, og6 = grids(cg, orc, [0.0] * 3, 100.0, 6)
    a6 = cg.cga_build(dev(pts), g6)
    shifts6, times6 = cg.cga_nn_autotune(a6, dev(q))
    assert (3, 6) not in times6 and (4, 8) not in times6 and (2, 5) in times6
    assert min(times6, key=times6.get) == shifts6
    nn_check(cg, orc, a6, orc.build(pts, og6), og6, q, brute=False)


def test_nn_prepare_levels_args(cg):
    """Coarse shifts must be strictly increasing, in 1..bits-1, at most two."""
    pts = synth.uniform_cube(5000, seed=124)
    a = cg.cga_build(dev(pts), cg.grid_from_box([0.0] * 3, 1.0, 8))
    for bad in [(3, 3), (4, 2), (8,), (1, 2, 3)]:
        with pytest.raises(cg.CgaError):
            cg.cga_nn_prepare(a, bad)
    cg.cga_nn_prepare(a, (1, 7))
    idx, d2 = cg.cga_nn_query(a, dev(pts[:100]))
    assert int(d2.max()) == 0
