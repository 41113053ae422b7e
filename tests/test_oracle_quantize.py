"""Pins for the oracle's grid and quantize/encode step (a1).

The paper gives no quantization formula (Sec. II-E-2-a asks for a bounding box
that holds every point; Sec. VI-C sets QP = bits per axis).  The reading pinned
here: q = floorf(fmaf(p, scale, offset)) clamped to [0, 2^b - 1], key =
x << 2b | y << b | z, with the rigid transform evaluated as a fixed fmaf chain.
Expected values come from exact rational arithmetic (tests/exact_f32.py) or
are worked by hand.
"""
import math

import numpy as np
import pytest

import exact_f32 as ex
from paper_2110_11616_gb300 import synth


def test_grid_from_box_unit_cube(orc):
    g = orc.grid_from_box([0, 0, 0], 1.0, 10)
    assert g.scale == 1024.0 and g.offset == (0.0, 0.0, 0.0)


def test_grid_from_box_lidar_box(orc):
    g = orc.grid_from_box([-128, -128, -128], 256.0, 16)
    assert g.scale == 256.0 and g.offset == (32768.0, 32768.0, 32768.0)


def test_grid_rejects_bad_bits(orc):
    for bits in (0, 17):
        with pytest.raises(orc.OracleError):
            orc.grid_from_box([0, 0, 0], 1.0, bits)


def _key(x, y, z, b):
    return (x << (2 * b)) | (y << b) | z


def test_voxel_boundaries_and_clamp(orc):
    g = orc.grid_from_box([0, 0, 0], 1.0, 10)
    k = 517
    on = np.float32(k / 1024.0)              # exact in float: lands on voxel k
    below = np.nextafter(on, np.float32(-1))  # just under the boundary: k - 1
    pts = np.array([[on, below, 0.0],
                    [1.0, 0.999999, -0.001],      # upper face -> clamp 1023; negative -> 0
                    [5.0, -7.0, 0.5]], np.float32)
    keys = orc.quantize(pts, g)
    assert int(keys[0]) == _key(k, k - 1, 0, 10)
    assert int(keys[1]) == _key(1023, 1023, 0, 10)
    assert int(keys[2]) == _key(1023, 0, 512, 10)


def test_fma_not_mul_then_add(orc):
    # exact p*s + o = 13.99989..., but rounding p*s first gives 14.0 exactly
    p, s, o = 2.043496608734131, 1274.286376953125, -2590.0
    p32, s32, o32 = np.float32(p), np.float32(s), np.float32(o)
    assert math.floor(float(np.float32(np.float32(p32 * s32) + o32))) == 14
    assert ex.quantize_axis(p32, s32, o32, 10) == 13
    g = orc.Grid(10, float(s32), (float(o32), float(o32), float(o32)))
    keys = orc.quantize(np.array([[p32, p32, p32]], np.float32), g)
    assert int(keys[0]) == _key(13, 13, 13, 10)


@pytest.mark.parametrize("bits", [1, 5, 10, 12, 16])
def test_quantize_matches_exact_arithmetic(orc, bits):
    pts = synth.uniform_cube(300, seed=11, lo=-0.1, extent=1.2)
    g = orc.grid_from_box([0, 0, 0], 1.0, bits)
    keys = orc.quantize(pts, g)
    for i in range(len(pts)):
        q = [ex.quantize_axis(pts[i, a], g.scale, g.offset[a], bits) for a in range(3)]
        assert int(keys[i]) == _key(*q, bits)


def test_transform_matches_exact_fma_chain(orc):
    pts = synth.uniform_cube(200, seed=12)
    X = synth.rigid_xform(seed=13, max_deg=10.0, max_t=0.05)
    g = orc.grid_from_box([0, 0, 0], 1.0, 16)
    keys = orc.quantize(pts, g, xform=X)
    for i in range(len(pts)):
        p2 = ex.transform(X, pts[i])
        q = [ex.quantize_axis(p2[a], g.scale, g.offset[a], 16) for a in range(3)]
        assert int(keys[i]) == _key(*q, 16)


def test_identity_transform_is_no_transform(orc):
    pts = synth.uniform_cube(1000, seed=14)
    ident = np.array([1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0], np.float32)
    g = orc.grid_from_box([0, 0, 0], 1.0, 12)
    assert np.array_equal(orc.quantize(pts, g), orc.quantize(pts, g, xform=ident))


def test_nonfinite_is_an_error(orc):
    g = orc.grid_from_box([0, 0, 0], 1.0, 10)
    for bad in (np.nan, np.inf, -np.inf):
        pts = np.array([[0.1, 0.2, 0.3], [0.1, bad, 0.3]], np.float32)
        with pytest.raises(orc.OracleError) as e:
            orc.quantize(pts, g)
        assert e.value.code == orc.ERR_NONFINITE


def test_transform_overflow_is_nonfinite(orc):
    g = orc.grid_from_box([0, 0, 0], 1.0, 10)
    X = np.array([3e38, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0], np.float32)
    with pytest.raises(orc.OracleError) as e:
        orc.quantize(np.array([[10.0, 0.5, 0.5]], np.float32), g, xform=X)
    assert e.value.code == orc.ERR_NONFINITE


def test_query_voxels_match_exact_arithmetic(orc):
    q = synth.uniform_queries(300, 15, [-3, -3, -3], 7.0)
    q[5] = [np.nan, 0, 0]
    g = orc.grid_from_box([0, 0, 0], 1.0, 10)
    v, ok = orc.query_voxels(g, q)
    assert not ok[5] and ok.sum() == len(q) - 1
    for i in range(len(q)):
        if ok[i]:
            assert [int(x) for x in v[i]] == [ex.quantize_query_axis(q[i, a], g.scale, g.offset[a])
                                              for a in range(3)]
    big = orc.Grid(4, 1.0e9, (0.0, 0.0, 0.0))
    v, ok = orc.query_voxels(big, np.array([[10.0, -10.0, 0.0]], np.float32))
    assert list(v[0]) == [1 << 30, -(1 << 30), 0]
