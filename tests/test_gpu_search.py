"""GPU parity of radius search and k-NN: every voxel within a squared radius
(ascending CGA index) and the k least (distance^2, key) equal the oracle's
exhaustive results element by element."""
import numpy as np
import pytest

from paper_2110_11616_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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


def world(cg, orc, kind, bits):
    if kind == "uniform":
        pts = synth.uniform_cube(20_000, seed=bits, lo=-0.02, extent=1.04)
        lo, ext = [0.0] * 3, 1.0
    elif kind == "surface":
        sc = synth.superellipsoid_scene(n_objects=8, seed=bits, extent=100.0)
        pts = synth.sample_surfaces(sc, 40_000, seed=bits + 1)
        lo, ext = [0.0] * 3, 100.0
    else:
        sc = synth.lidar_sweeps(2, 64, 256, seed=bits, with_world=True)
        pts = sc.world.astype(np.float32)
        lo, ext = [-128.0] * 3, 256.0
    g, og = cg.grid_from_box(lo, ext, bits), orc.grid_from_box(lo, ext, bits)
    return pts, lo, ext, g, og, cg.cga_build(dev(pts), g), orc.build(pts, og)


def queries(pts, lo, ext, n, seed):
    rng = np.random.default_rng(seed)
    near = pts[rng.integers(0, len(pts), n)] + rng.normal(0, ext / 300, (n, 3))
    return np.concatenate([near, synth.uniform_queries(n // 4, seed, np.asarray(lo) - 0.2 * ext,
                                                       1.4 * ext),
                           [[np.nan, 0, 0]]]).astype(np.float32)


@pytest.mark.parametrize("kind,bits", [("uniform", 7), ("uniform", 10), ("surface", 10),
                                       ("lidar", 16)])
@pytest.mark.parametrize("r2", [0, 3, 40, 700])
def test_radius_parity(cg, orc, kind, bits, r2):
    pts, lo, ext, g, og, a, oa = world(cg, orc, kind, bits)
    q = queries(pts, lo, ext, 400, bits + r2)
    off, idx, d2 = cg.cga_radius(a, dev(q), r2)
    ooff, oidx, od2 = orc.radius(oa, og, q, r2)
    np.testing.assert_array_equal(off.cpu().numpy().view(np.uint64), ooff)
    np.testing.assert_array_equal(idx.cpu().numpy().view(np.uint32), oidx)
    np.testing.assert_array_equal(d2.cpu().numpy().view(np.uint64), od2)


@pytest.mark.parametrize("kind,bits", [("uniform", 7), ("uniform", 10), ("surface", 10),
                                       ("lidar", 16)])
@pytest.mark.parametrize("k", [1, 2, 7, 16, 32])
def test_knn_parity(cg, orc, kind, bits, k):
    pts, lo, ext, g, og, a, oa = world(cg, orc, kind, bits)
    q = queries(pts, lo, ext, 400, bits * k)
    idx, d2 = cg.cga_knn(a, dev(q), k)
    oi, od = orc.knn(oa, og, q, k)
    np.testing.assert_array_equal(d2.cpu().numpy().view(np.uint64), od)
    np.testing.assert_array_equal(idx.cpu().numpy().view(np.uint32), oi)


@pytest.mark.parametrize("kind,bits", [("uniform", 7), ("surface", 10), ("lidar", 16)])
@pytest.mark.parametrize("k", [33, 100, 400, 1024])
def test_knn_large_k_parity(cg, orc, kind, bits, k):
    """k above 32 collects candidates in a shared-memory buffer that is sorted
    and cut to k whenever it fills (the paper's Fig. 3 shows 400-NN)."""
    pts, lo, ext, g, og, a, oa = world(cg, orc, kind, bits)
    q = queries(pts, lo, ext, 120, bits * k)
    idx, d2 = cg.cga_knn(a, dev(q), k)
    oi, od = orc.knn(oa, og, q, k)
    np.testing.assert_array_equal(d2.cpu().numpy().view(np.uint64), od)
    np.testing.assert_array_equal(idx.cpu().numpy().view(np.uint32), oi)


def test_knn_large_k_few_voxels(cg, orc):
    """Fewer stored voxels than k: the tail holds the sentinels."""
    ax = np.arange(4, dtype=np.float32)
    vox = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1).reshape(-1, 3) + 0.5
    og, g = orc.Grid(4, 1.0, (0.0, 0.0, 0.0)), cg.make_grid(4, 1.0, (0.0, 0.0, 0.0))
    a, oa = cg.cga_build(dev(vox), g), orc.build(vox, og)
    q = np.array([[1.5, 1.5, 1.5], [9, 9, 9], [np.inf, 0, 0]], np.float32)
    for k in (40, 64, 65, 200):
        idx, d2 = cg.cga_knn(a, dev(q), k)
        oi, od = orc.knn(oa, og, q, k)
        np.testing.assert_array_equal(idx.cpu().numpy().view(np.uint32), oi)
        np.testing.assert_array_equal(d2.cpu().numpy().view(np.uint64), od)


@pytest.mark.parametrize("kind,bits", [("uniform", 10), ("surface", 10), ("lidar", 16)])
def test_prepared_world_parity(cg, orc, kind, bits):
    """After cga_nn_prepare the walks read each column's voxel and z range from
    the column table and skip the z searches it makes unnecessary."""
    pts, lo, ext, g, og, a, oa = world(cg, orc, kind, bits)
    cg.cga_nn_prepare(a)
    q = queries(pts, lo, ext, 9000, bits + 11)
    for r2 in (40, 700):
        off, idx, d2 = cg.cga_radius(a, dev(q), r2)
        ooff, oidx, od2 = orc.radius(oa, og, q, r2)
        np.testing.assert_array_equal(off.cpu().numpy().view(np.uint64), ooff)
        np.testing.assert_array_equal(idx.cpu().numpy().view(np.uint32), oidx)
        np.testing.assert_array_equal(d2.cpu().numpy().view(np.uint64), od2)
    for k in (8, 100):
        ki, kd = cg.cga_knn(a, dev(q[:3000]), k)
        oi, od = orc.knn(oa, og, q[:3000], k)
        np.testing.assert_array_equal(kd.cpu().numpy().view(np.uint64), od)
        np.testing.assert_array_equal(ki.cpu().numpy().view(np.uint32), oi)


def test_knn_one_equals_nn(cg):
    pts = synth.uniform_cube(30_000, seed=3)
    g = cg.grid_from_box([0, 0, 0], 1.0, 12)
    a = cg.cga_build(dev(pts), g)
    q = dev(synth.uniform_queries(12_000, 4, [-0.1] * 3, 1.2))   # Morton-ordered batch
    ki, kd = cg.cga_knn(a, q, 1)
    ni, nd = cg.cga_nn_query(a, q)
    assert torch.equal(ki[:, 0], ni) and torch.equal(kd[:, 0], nd)


@pytest.mark.parametrize("kind,bits", [("uniform", 10), ("surface", 10)])
def test_ordered_batch_parity(cg, orc, kind, bits):
    """Batches of 8192 queries and more are searched in Morton order; every
    result still lands in its own query's row."""
    pts, lo, ext, g, og, a, oa = world(cg, orc, kind, bits)
    q = queries(pts, lo, ext, 9000, bits + 5)
    assert len(q) >= 8192
    off, idx, d2 = cg.cga_radius(a, dev(q), 40)
    ooff, oidx, od2 = orc.radius(oa, og, q, 40)
    np.testing.assert_array_equal(off.cpu().numpy().view(np.uint64), ooff)
    np.testing.assert_array_equal(idx.cpu().numpy().view(np.uint32), oidx)
    np.testing.assert_array_equal(d2.cpu().numpy().view(np.uint64), od2)
    ki, kd = cg.cga_knn(a, dev(q), 8)
    oi, od = orc.knn(oa, og, q, 8)
    np.testing.assert_array_equal(kd.cpu().numpy().view(np.uint64), od)
    np.testing.assert_array_equal(ki.cpu().numpy().view(np.uint32), oi)


def test_lattice_ties_and_few_voxels(cg, orc):
    ax = np.arange(6, dtype=np.float32)
    vox = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1).reshape(-1, 3) + 0.5
    og = orc.Grid(4, 1.0, (0.0, 0.0, 0.0))
    g = cg.make_grid(4, 1.0, (0.0, 0.0, 0.0))
    a, oa = cg.cga_build(dev(vox), g), orc.build(vox, og)
    q = np.array([[2.5, 2.5, 2.5], [0.5, 0.5, 0.5], [3.0, 3.0, 3.0], [-9, 20, 3]], np.float32)
    for k in (7, 19, 32):
        idx, d2 = cg.cga_knn(a, dev(q), k)
        oi, od = orc.knn(oa, og, q, k)
        np.testing.assert_array_equal(idx.cpu().numpy().view(np.uint32), oi)
    few = cg.cga_build(dev(vox[:5]), g)
    idx, d2 = cg.cga_knn(few, dev(q), 8)
    oi, od = orc.knn(orc.build(vox[:5], og), og, q, 8)
    np.testing.assert_array_equal(idx.cpu().numpy().view(np.uint32), oi)
    np.testing.assert_array_equal(d2.cpu().numpy().view(np.uint64), od)


def test_search_arguments(cg):
    a = cg.cga_build(dev(np.zeros((1, 3))), cg.grid_from_box([0, 0, 0], 1.0, 8))
    with pytest.raises(cg.CgaError):
        cg.cga_knn(a, dev(np.zeros((2, 3))), 1025)
    with pytest.raises(cg.CgaError):
        cg.cga_knn(a, dev(np.zeros((2, 3))), 0)
