"""Pins of the oracle's perspective projection (Eq. 5-6): closed forms worked
by hand (a voxel on the optical axis, the Eq. 5 divide, a 90-degree turn),
occlusion and tie rules, voxels behind the eye, and invariance under moving
the voxels and the eye together."""
import numpy as np
import pytest

from paper_2110_11616_gb300 import synth

EMPTY = np.uint32(0xFFFFFFFF)


def lattice_cga(orc, vox, bits=8):
    """A CGA holding exactly the given integer voxels (grid scale 1, offset 0)."""
    g = orc.Grid(bits, 1.0, (0.0, 0.0, 0.0))
    return orc.build(np.asarray(vox, np.float32).reshape(-1, 3), g)


def test_single_voxel_closed_form(orc):
    # voxel (10, 20, 50), eye at the origin, D = 100: px = 100*10/50 = 20,
    # py = 100*20/50 = 40; pixel (20 + 32, 40 + 64) in a 64 x 128 image.
    a = lattice_cga(orc, [[10, 20, 50]])
    idx, dep = orc.perspective(a, [0, 0, 0], 1.0, 0.0, 100.0, 64, 128)
    assert idx[104, 52] == 0 and dep[104, 52] == 50.0
    assert (idx != EMPTY).sum() == 1 and np.isinf(dep[idx == EMPTY]).all()


def test_nearer_voxel_occludes(orc):
    # (10, 20, 50) and (20, 40, 100) lie on one ray from the origin
    a = lattice_cga(orc, [[20, 40, 100], [10, 20, 50]])
    idx, dep = orc.perspective(a, [0, 0, 0], 1.0, 0.0, 100.0, 64, 128)
    keys = orc.decode(a).tolist()
    assert keys[idx[104, 52]] == [10, 20, 50] and dep[104, 52] == 50.0
    assert (idx != EMPTY).sum() == 1


def test_equal_depth_tie_keeps_smaller_index(orc):
    # D = 1: (10, 20, 50) -> px 0.2, (11, 20, 50) -> px 0.22: the same pixel
    a = lattice_cga(orc, [[11, 20, 50], [10, 20, 50]])
    idx, dep = orc.perspective(a, [0, 0, 0], 1.0, 0.0, 1.0, 8, 8)
    assert (idx != EMPTY).sum() == 1
    assert orc.decode(a)[idx[idx != EMPTY][0]].tolist() == [10, 20, 50]


def test_quarter_turn_about_y(orc):
    # cos = 0, sin = 1: x' = -sz, z' = sx.  Voxel (50, 0, 10) from the origin:
    # z' = 50, x' = -10, px = 100 * -10 / 50 = -20 -> u = -20 + 32 = 12, v = 0 + 32
    a = lattice_cga(orc, [[50, 0, 10]])
    idx, dep = orc.perspective(a, [0, 0, 0], 0.0, 1.0, 100.0, 64, 64)
    assert idx[32, 12] == 0 and dep[32, 12] == 50.0


def test_behind_the_eye_is_dropped(orc):
    a = lattice_cga(orc, [[10, 10, 5], [10, 10, 20]])
    idx, _ = orc.perspective(a, [10, 10, 20], 1.0, 0.0, 10.0, 16, 16)  # z' = -15 and 0
    assert (idx == EMPTY).all()


def test_translation_invariance(orc):
    pts = synth.uniform_cube(3000, seed=5)
    g = orc.grid_from_box([0, 0, 0], 1.0, 7)
    a = orc.build(pts, g)
    vox = orc.decode(a).astype(np.int64)
    b = lattice_cga(orc, vox + np.array([13, 7, 21]), bits=8)
    i1, d1 = orc.perspective(a, [64, 64, -90], 0.8, 0.6, 120.0, 96, 80)
    i2, d2 = orc.perspective(b, [77, 71, -69], 0.8, 0.6, 120.0, 96, 80)
    np.testing.assert_array_equal(i1, i2)
    np.testing.assert_array_equal(d1, d2)


def test_each_pixel_keeps_its_nearest_voxel(orc):
    pts = synth.uniform_cube(5000, seed=6)
    g = orc.grid_from_box([0, 0, 0], 1.0, 6)
    a = orc.build(pts, g)
    idx, dep = orc.perspective(a, [32, 32, -40], 1.0, 0.0, 50.0, 40, 40)
    hit = idx != EMPTY
    # every kept voxel is at least as near as any voxel of a pixel-sized
    # neighbourhood that lands in the same pixel: checked by re-projecting all
    # voxels with float64 and comparing depths where pixels agree
    vox = orc.decode(a).astype(np.float64)
    z = vox[:, 2] + 40
    u = np.floor(50 * (vox[:, 0] - 32) / z + 20)
    v = np.floor(50 * (vox[:, 1] - 32) / z + 20)
    for p in np.flatnonzero(hit.ravel())[:200]:
        pv, pu = divmod(p, 40)
        same = (u == pu) & (v == pv)
        if same.any():
            assert dep.ravel()[p] <= z[same].min() + 1e-3


def test_invalid(orc):
    a = lattice_cga(orc, [[1, 2, 3]])
    with pytest.raises(orc.OracleError):
        orc.perspective(a, [0, 0, 0], 1.0, 0.0, 0.0, 4, 4)
