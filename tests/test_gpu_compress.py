"""GPU parity of the compression pieces (Sec. V-D) and the G-Arrays lookup:
k-means labels, centres, counts and pass counts, motion vectors, the
reconstructed frame, its NN correspondence in the reference, point lookups
and the dense X pointer equal the oracle's element by element."""
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


def devi(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32).reshape(-1, 3)).cuda()


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def frames(kind, bits, seed):
    """(reference points, predicted points, box lo, extent): the predicted frame
    is the reference under a small rigid motion plus some points of its own."""
    if kind == "uniform":
        ref = synth.uniform_cube(30_000, seed, lo=0.05, extent=0.9)
        lo, ext = [0.0] * 3, 1.0
    elif kind == "surface":
        sc = synth.superellipsoid_scene(n_objects=10, seed=seed, extent=100.0)
        ref = synth.sample_surfaces(sc, 60_000, seed=seed + 1)
        lo, ext = [0.0] * 3, 100.0
    else:
        sc = synth.lidar_sweeps(2, 64, 256, seed=seed, with_world=True)
        ref = sc.world.astype(np.float32)
        lo, ext = [-128.0] * 3, 256.0
    X = synth.rigid_xform(seed + 7, max_deg=3.0, max_t=0.02 * ext)
    pred = synth.apply_xform64(X, ref).astype(np.float32)
    extra = synth.uniform_cube(len(ref) // 20, seed + 9, lo=lo[0] + 0.2 * ext, extent=0.6 * ext)
    return ref, np.concatenate([pred, extra]).astype(np.float32), lo, ext


def build_both(cg, orc, pts, lo, ext, bits):
    g, og = cg.grid_from_box(lo, ext, bits), orc.grid_from_box(lo, ext, bits)
    return cg.cga_build(dev(pts), g), orc.build(pts, og)


def check_kmeans(cg, orc, a, oa, max_iter):
    lab, cen, cnt, it = cg.cga_kmeans(a, max_iter)
    ol, oc, on, oi = orc.kmeans(oa, max_iter)
    assert int(it.item()) == oi
    np.testing.assert_array_equal(lab.cpu().numpy(), ol)
    np.testing.assert_array_equal(cen.cpu().numpy(), oc)
    np.testing.assert_array_equal(cnt.cpu().numpy().astype(np.uint64), on)
    return lab, cen, cnt, (ol, oc, on, oi)


@pytest.mark.parametrize("kind,bits", [("uniform", 8), ("surface", 10), ("lidar", 16)])
@pytest.mark.parametrize("max_iter", [1, 2, 5, 300])
def test_kmeans_parity(cg, orc, kind, bits, max_iter):
    ref, _, lo, ext = frames(kind, bits, 3)
    a, oa = build_both(cg, orc, ref, lo, ext, bits)
    assert oa.u > 3 * 4096  # several tiles and a ragged tail
    check_kmeans(cg, orc, a, oa, max_iter)


def test_kmeans_golden_and_degenerate(cg, orc):
    from test_oracle_compress import load_cases  # the hand-worked fixtures
    for case in load_cases():
        vox = case["voxels"].astype(np.float32) + 0.5
        g = cg.make_grid(case["bits"], 1.0, (0.0, 0.0, 0.0))
        a = cg.cga_build(dev(vox), g)
        lab, cen, cnt, it = cg.cga_kmeans(a, case["max_iter"])
        np.testing.assert_array_equal(lab.cpu().numpy(), case["labels"])
        np.testing.assert_array_equal(cen.cpu().numpy(), case["centres"])
        np.testing.assert_array_equal(cnt.cpu().numpy(), case["counts"])
        assert int(it.item()) == case["iters"]
    g = cg.make_grid(4, 1.0, (0.0, 0.0, 0.0))
    empty = cg.cga_build(dev(np.zeros((0, 3))), g)
    lab, cen, cnt, it = cg.cga_kmeans(empty, 10)
    assert lab.numel() == 0 and int(it.item()) == 0
    assert not cen.any().item() and not cnt.any().item()
    one = cg.cga_build(dev(np.array([[3.5, 4.5, 5.5]])), g)
    lab, cen, cnt, it = cg.cga_kmeans(one, 10)
    assert lab.tolist() == [0] and int(it.item()) == 2 and cnt.tolist() == [1] + [0] * 7


@pytest.mark.parametrize("kind,bits", [("uniform", 8), ("surface", 10), ("lidar", 16)])
def test_prediction_chain_parity(cg, orc, kind, bits):
    """Cluster both frames, motion vectors, reconstruction, and the NN
    correspondence of every reconstructed voxel in the reference."""
    ref, pred, lo, ext = frames(kind, bits, 11)
    a_ref, o_ref = build_both(cg, orc, ref, lo, ext, bits)
    a_pred, o_pred = build_both(cg, orc, pred, lo, ext, bits)
    _, cr, nr, (_, ocr, onr, _) = check_kmeans(cg, orc, a_ref, o_ref, 64)
    lp, cp, npd, (olp, ocp, onp, _) = check_kmeans(cg, orc, a_pred, o_pred, 64)
    mv = cg.cga_motion_vectors(cr, nr, cp, npd)
    omv = orc.motion_vectors(ocr, onr, ocp, onp)
    np.testing.assert_array_equal(mv.cpu().numpy(), omv)
    rec = cg.cga_reconstruct(a_pred, lp, mv)
    orec = orc.reconstruct(o_pred, olp, omv)
    np.testing.assert_array_equal(rec.cpu().numpy(), orec)
    take = np.random.default_rng(1).choice(len(orec), size=min(len(orec), 12_000), replace=False)
    idx, d2 = cg.cga_nn_query_voxels(a_ref, devi(orec[take]))
    oi, od = orc.nn_voxels(o_ref, orec[take])
    np.testing.assert_array_equal(u32(idx), oi)
    np.testing.assert_array_equal(d2.cpu().numpy().view(np.uint64), od)


def test_residual_frame_parity(cg, orc):
    """The residual of the reconstructed frame against its NN correspondence in
    the reference, with the frames' averaged colours (Value arrays)."""
    ref, pred, lo, ext = frames("surface", 10, 21)
    g, og = cg.grid_from_box(lo, ext, 10), orc.grid_from_box(lo, ext, 10)
    col = lambda p: (np.abs(p) * 2.55 % 256).astype(np.uint8)
    a_ref = cg.cga_build_values(dev(ref), torch.from_numpy(col(ref)).cuda(), g)
    a_pred = cg.cga_build_values(dev(pred), torch.from_numpy(col(pred)).cuda(), g)
    o_ref, ov_ref = orc.build_values(ref, col(ref), og)
    o_pred, ov_pred = orc.build_values(pred, col(pred), og)
    _, cr, nr, _ = cg.cga_kmeans(a_ref, 64)
    lp, cp, npd, _ = cg.cga_kmeans(a_pred, 64)
    rec = cg.cga_reconstruct(a_pred, lp, cg.cga_motion_vectors(cr, nr, cp, npd))
    idx, _ = cg.cga_nn_query_voxels(a_ref, rec)
    idx[::97] = -1  # some points without a corresponding point
    res = cg.cga_residual(cg.cga_values(a_pred), cg.cga_values(a_ref), idx)
    want = orc.residual(ov_pred, ov_ref, u32(idx))
    np.testing.assert_array_equal(res.cpu().numpy(), want)


def test_nn_query_voxels_extremes(cg, orc):
    pts = synth.uniform_cube(20_000, 5)
    g, og = cg.grid_from_box([0, 0, 0], 1.0, 9), orc.grid_from_box([0, 0, 0], 1.0, 9)
    a, oa = cg.cga_build(dev(pts), g), orc.build(pts, og)
    rng = np.random.default_rng(2)
    qv = rng.integers(-600, 1200, (9000, 3))
    qv[:6] = [[2**31 - 1, 0, 0], [-(2**31), 5, 5], [0, 2**31 - 1, -(2**31)],
              [511, 511, 511], [0, 0, 0], [2**30 + 5, -(2**30) - 5, 7]]
    idx, d2 = cg.cga_nn_query_voxels(a, devi(qv))
    oi, od = orc.nn_voxels(oa, qv)
    np.testing.assert_array_equal(u32(idx), oi)
    np.testing.assert_array_equal(d2.cpu().numpy().view(np.uint64), od)


@pytest.mark.parametrize("kind,bits", [("uniform", 8), ("surface", 10), ("lidar", 16)])
def test_lookup_and_garrays_parity(cg, orc, kind, bits):
    ref, pred, lo, ext = frames(kind, bits, 17)
    a, oa = build_both(cg, orc, ref, lo, ext, bits)
    stored = orc.decode(oa).astype(np.int64)
    rng = np.random.default_rng(bits)
    side = 1 << bits
    q = np.concatenate([stored[rng.integers(0, len(stored), 20_000)],
                        stored[rng.integers(0, len(stored), 20_000)] + rng.integers(-1, 2, (20_000, 3)),
                        rng.integers(-2, side + 2, (10_000, 3))])
    want = orc.lookup_voxels(oa, q)
    np.testing.assert_array_equal(u32(cg.cga_lookup(a, devi(q))), want)
    xp = cg.cga_garrays_x(a)
    np.testing.assert_array_equal(u32(xp), orc.garrays_x(oa))
    np.testing.assert_array_equal(u32(cg.cga_garrays_lookup(a, xp, devi(q))), want)


def test_compress_arguments(cg):
    g = cg.make_grid(4, 1.0, (0.0, 0.0, 0.0))
    a = cg.cga_build(dev(np.array([[1.5, 1.5, 1.5]])), g)
    for bad in (0, 1025):
        with pytest.raises(cg.CgaError):
            cg.cga_kmeans(a, bad)
