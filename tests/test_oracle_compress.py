"""Pins of the oracle's compression pieces (Sec. V-D) and the G-Arrays form
(Sec. V): hand-worked k-means fixtures, the fixed-point property of a
converged k-means, exact translation equivariance (motion vectors that undo a
shift, reconstruction onto the reference), and lookups and dense X pointers
checked against numpy set routines."""
import os

import numpy as np
import pytest

import oracle as orc
from paper_2110_11616_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "kmeans_fixtures.txt")
U32_MAX = np.iinfo(np.uint32).max


def _rows(text):
    return [[int(t) for t in r.split()] for r in text.split(";")]


def load_cases():
    cases, cur = [], None
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, _, val = line.partition(" ")
        if key == "case":
            cur = {"name": val}
            cases.append(cur)
        elif key in ("voxels", "centres"):
            cur[key] = np.array(_rows(val), np.int64)
        elif key in ("labels", "counts"):
            cur[key] = np.array([int(t) for t in val.split()], np.int64)
        else:
            cur[key] = int(val)
    return cases


def cga_of_voxels(vox, bits):
    g = orc.Grid(bits, 1.0, (0.0, 0.0, 0.0))
    return orc.build(np.asarray(vox, np.float32) + 0.5, g), g


@pytest.mark.parametrize("case", load_cases(), ids=lambda c: c["name"])
def test_kmeans_hand_fixtures(case):
    a, _ = cga_of_voxels(case["voxels"], case["bits"])
    np.testing.assert_array_equal(orc.decode(a), case["voxels"])  # listed in CGA order
    lab, cen, cnt, it = orc.kmeans(a, case["max_iter"])
    np.testing.assert_array_equal(lab, case["labels"])
    np.testing.assert_array_equal(cen, case["centres"])
    np.testing.assert_array_equal(cnt, case["counts"])
    assert it == case["iters"]


def random_cga(seed, n=3000, bits=8):
    pts = synth.uniform_cube(n, seed)
    pts = np.concatenate([pts, synth.uniform_cube(n // 3, seed + 1, lo=0.1, extent=0.2)])
    return cga_of_voxels(np.floor(pts * (1 << bits)).astype(np.int64), bits)


def sq_dist_to_centres(v, cen):
    d = 256 * v[:, None, :].astype(np.int64) - cen[None, :, :]
    return (d * d).sum(axis=2)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_kmeans_converged_is_a_fixed_point(seed):
    """At convergence every label is the argmin over the final centres (lower
    index on ties) and every non-empty centre is its members' rounded mean."""
    a, _ = random_cga(seed)
    lab, cen, cnt, it = orc.kmeans(a, 500)
    assert 1 < it < 500
    v = orc.decode(a).astype(np.int64)
    np.testing.assert_array_equal(np.argmin(sq_dist_to_centres(v, cen), axis=1), lab)
    np.testing.assert_array_equal(np.bincount(lab, minlength=8), cnt)
    for c in range(8):
        if cnt[c]:
            s = v[lab == c].sum(axis=0)
            n = int(cnt[c])
            np.testing.assert_array_equal(cen[c], (256 * s + n // 2) // n)


def test_kmeans_first_pass_from_corners():
    a, _ = random_cga(7)
    v = orc.decode(a).astype(np.int64)
    lo, hi = v.min(axis=0), v.max(axis=0)
    corners = np.array([[hi[ax] if (c >> ax) & 1 else lo[ax] for ax in range(3)]
                        for c in range(8)], np.int64) * 256
    lab, _, _, it = orc.kmeans(a, 1)
    assert it == 1
    np.testing.assert_array_equal(lab, np.argmin(sq_dist_to_centres(v, corners), axis=1))


def test_kmeans_degenerate():
    a, _ = cga_of_voxels([[3, 4, 5]], 4)
    lab, cen, cnt, it = orc.kmeans(a, 10)
    assert list(lab) == [0] and it == 2 and cnt[0] == 1 and cnt[1:].sum() == 0
    np.testing.assert_array_equal(cen, np.tile([768, 1024, 1280], (8, 1)))
    e, _ = cga_of_voxels(np.zeros((0, 3)), 4)
    lab, cen, cnt, it = orc.kmeans(e, 10)
    assert len(lab) == 0 and it == 0 and not cen.any() and not cnt.any()
    with pytest.raises(Exception):
        orc.kmeans(a, 0)


@pytest.mark.parametrize("shift", [(3, -2, 5), (0, 0, 0), (-7, 11, 1)])
def test_translation_motion_and_reconstruction(shift):
    """A frame shifted by whole voxels: its clusters shift with it, the motion
    vectors are exactly -256 * shift, and the reconstruction lands on the
    reference voxel by voxel (NN distance 0, same CGA index)."""
    rng = np.random.default_rng(5)
    ref_v = np.unique(rng.integers(20, 230, (2500, 3)), axis=0)
    pred_v = ref_v + np.array(shift)
    ref, _ = cga_of_voxels(ref_v, 8)
    pred, _ = cga_of_voxels(pred_v, 8)
    lr, cr, nr, ir = orc.kmeans(ref, 300)
    lp, cp, np_, ip = orc.kmeans(pred, 300)
    np.testing.assert_array_equal(lr, lp)
    np.testing.assert_array_equal(cp, cr + 256 * np.array(shift))
    mv = orc.motion_vectors(cr, nr, cp, np_)
    want = np.where((nr > 0)[:, None], -256 * np.array(shift)[None, :], 0)
    np.testing.assert_array_equal(mv, want)
    rec = orc.reconstruct(pred, lp, mv)
    np.testing.assert_array_equal(rec, orc.decode(ref).astype(np.int32))
    idx, d2 = orc.nn_voxels(ref, rec)
    np.testing.assert_array_equal(idx, np.arange(ref.u))
    assert not d2.any()


def test_motion_vectors_empty_clusters():
    cr = np.arange(24).reshape(8, 3) * 10
    cp = np.arange(24).reshape(8, 3)
    nr = np.array([1, 0, 2, 3, 0, 1, 1, 1], np.uint64)
    npred = np.array([1, 1, 0, 3, 0, 1, 0, 1], np.uint64)
    mv = orc.motion_vectors(cr, nr, cp, npred)
    both = (nr > 0) & (npred > 0)
    np.testing.assert_array_equal(mv[both], (cr - cp)[both])
    assert not mv[~both].any()


def test_reconstruct_rounds_half_up():
    a, _ = cga_of_voxels([[10, 10, 10]], 5)
    for m, step in [(128, 1), (127, 0), (-128, 0), (-129, -1), (383, 1), (384, 2), (-384, -1),
                    (-385, -2), (2560, 10), (-2560, -10)]:
        mv = np.zeros((8, 3), np.int64)
        mv[0] = [m, -m, 0]
        out = orc.reconstruct(a, [0], mv)
        want_y = 10 + (-m + 128) // 256
        assert out[0].tolist() == [10 + step, want_y, 10], (m, out)


def test_lookup_and_garrays():
    a, _ = random_cga(11, n=4000, bits=7)
    v = orc.decode(a).astype(np.int64)
    np.testing.assert_array_equal(orc.lookup_voxels(a, v), np.arange(a.u))
    rng = np.random.default_rng(3)
    q = rng.integers(-3, 131, (5000, 3))
    stored = {tuple(r) for r in v.tolist()}
    want = np.array([U32_MAX if tuple(r) not in stored else 0 for r in q.tolist()], np.uint32)
    got = orc.lookup_voxels(a, q)
    absent = want == U32_MAX
    np.testing.assert_array_equal(got[absent], want[absent])
    np.testing.assert_array_equal(v[got[~absent]], q[~absent])
    xp = orc.garrays_x(a)
    assert len(xp) == 129 and xp[0] == 0 and xp[-1] == a.g
    cols = np.unique(v[:, :2], axis=0)
    np.testing.assert_array_equal(np.diff(xp.astype(np.int64)),
                                  np.bincount(cols[:, 0], minlength=128))
    np.testing.assert_array_equal(orc.garrays_lookup(a, xp, q), got)
    np.testing.assert_array_equal(orc.garrays_lookup(a, xp, v), np.arange(a.u))


def test_nn_voxels_matches_float_queries():
    a, g = random_cga(13, n=2000, bits=6)
    rng = np.random.default_rng(4)
    qv = rng.integers(-20, 90, (400, 3))
    i1, d1 = orc.nn_voxels(a, qv)
    i2, d2 = orc.nn_brute(a, g, qv.astype(np.float32) + 0.5)
    np.testing.assert_array_equal(i1, i2)
    np.testing.assert_array_equal(d1, d2)
    big = np.array([[2**31 - 1, 0, 0], [-(2**31), 5, 5]])
    i3, d3 = orc.nn_voxels(a, big)
    i4, d4 = orc.nn_brute(a, g, np.array([[2.0**30, 0.5, 0.5], [-(2.0**30), 5.5, 5.5]],
                                         np.float32))
    np.testing.assert_array_equal(i3, i4)
    np.testing.assert_array_equal(d3, d4)


def test_residual_hand_example():
    """Sec. V-D residual: pred - ref[idx] per channel; no correspondence keeps pred."""
    pred = np.array([[10, 20, 30], [5, 5, 5], [0, 255, 128]], np.uint8)
    ref = np.array([[1, 2, 3], [200, 0, 255]], np.uint8)
    idx = np.array([1, U32_MAX, 0], np.uint32)
    np.testing.assert_array_equal(orc.residual(pred, ref, idx),
                                  [[-190, 20, -225], [5, 5, 5], [-1, 253, 125]])


def test_residual_reconstructs_prediction():
    rng = np.random.default_rng(8)
    ref = rng.integers(0, 256, (500, 3)).astype(np.uint8)
    pred = rng.integers(0, 256, (700, 3)).astype(np.uint8)
    idx = rng.integers(0, 500, 700).astype(np.uint32)
    idx[::50] = U32_MAX
    res = orc.residual(pred, ref, idx).astype(np.int64)
    have = idx != U32_MAX
    np.testing.assert_array_equal(ref[idx[have]].astype(np.int64) + res[have], pred[have])
    np.testing.assert_array_equal(res[~have], pred[~have])


def test_prediction_chain_residual_is_zero_under_translation():
    """Values that move with their voxels: clustering, motion vectors,
    reconstruction and NN correspondence bring every predicted voxel onto its
    reference voxel, so the residual frame is all zeros."""
    rng = np.random.default_rng(12)
    ref_v = np.unique(rng.integers(20, 230, (2000, 3)), axis=0)
    shift = np.array([4, -3, 2])
    colour = lambda v: np.stack([(v[:, 0] * 7 + v[:, 1]) % 256, (v[:, 1] * 5) % 256,
                                 (v[:, 2] * 3 + 1) % 256], 1).astype(np.uint8)
    g = orc.Grid(8, 1.0, (0.0, 0.0, 0.0))
    ref, ref_vals = orc.build_values((ref_v + 0.5).astype(np.float32), colour(ref_v), g)
    pred, pred_vals = orc.build_values((ref_v + shift + 0.5).astype(np.float32), colour(ref_v), g)
    lr, cr, nr, _ = orc.kmeans(ref, 300)
    lp, cp, npd, _ = orc.kmeans(pred, 300)
    mv = orc.motion_vectors(cr, nr, cp, npd)
    rec = orc.reconstruct(pred, lp, mv)
    idx, d2 = orc.nn_voxels(ref, rec)
    assert not d2.any()
    assert not orc.residual(pred_vals, ref_vals, idx).any()
