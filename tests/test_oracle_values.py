"""Pins of the oracle's Value array (Sec. V) for builds and merges.

Expected values: the hand-derived fixtures of tests/golden/value_fixtures.txt,
closed forms (identical attributes average to themselves; the average of a
row with itself is the row), invariants (input permutation for averages, the
geometry equals the plain build / merge), and independent numpy computations
of the per-voxel mean and first row on random clouds.
"""
import os

import numpy as np
import pytest

from paper_2110_11616_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_value_cases():
    cases, cur = {}, None
    with open(os.path.join(GOLDEN, "value_fixtures.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            head, _, rest = line.partition(" ")
            if head == "case":
                cur = {"name": rest.strip()}
            elif head == "end":
                cases[cur["name"]] = cur
            elif head in ("bits",):
                cur[head] = int(rest)
            elif head == "policy":
                cur[head] = rest.strip()
            else:
                rows = [[int(v) for v in r.split()] for r in rest.split(";") if r.strip()]
                cur[head] = np.array(rows, np.int64)
    return cases


CASES = load_value_cases()


def unit_grid(orc, bits):
    return orc.Grid(bits, 1.0, (0.0, 0.0, 0.0))


def as_points(vox):
    return np.asarray(vox, np.float64).astype(np.float32).reshape(-1, 3)


@pytest.mark.parametrize("name", [n for n in CASES if n.startswith("build")])
def test_build_fixture(orc, name):
    c = CASES[name]
    g = unit_grid(orc, c["bits"])
    cga, vals = orc.build_values(as_points(c["points"]), c["attrs"].astype(np.uint8), g,
                                 policy=c["policy"])
    np.testing.assert_array_equal(orc.decode(cga), c["voxels"])
    np.testing.assert_array_equal(vals, c["values"])


@pytest.mark.parametrize("name", [n for n in CASES if n.startswith("merge")])
def test_merge_fixture(orc, name):
    c = CASES[name]
    g = unit_grid(orc, c["bits"])
    a, va = orc.build_values(as_points(c["a"]), c["a_values"].astype(np.uint8), g, policy="first")
    b, vb = orc.build_values(as_points(c["b"]), c["b_values"].astype(np.uint8), g, policy="first")
    m, vm = orc.merge_values(a, va, b, vb, policy=c["policy"])
    np.testing.assert_array_equal(orc.decode(m), c["voxels"])
    np.testing.assert_array_equal(vm, c["values"])


def random_cloud(n, seed, channels):
    rng = np.random.default_rng(seed)
    pts = synth.uniform_cube(n, seed=seed)
    attr = rng.integers(0, 256, size=(n, channels), dtype=np.uint8)
    return pts, attr


@pytest.mark.parametrize("channels", [1, 2, 3, 4])
def test_geometry_equals_plain_build(orc, channels):
    pts, attr = random_cloud(5000, 11 + channels, channels)
    g = orc.grid_from_box([0, 0, 0], 1.0, 5)
    ref = orc.build(pts, g)
    for policy in ("average", "first"):
        c, v = orc.build_values(pts, attr, g, policy=policy)
        for lv in ("X_index", "X_pointer", "Y_index", "Y_pointer", "Z_index"):
            np.testing.assert_array_equal(getattr(c, lv), getattr(ref, lv))
        assert v.shape == (ref.u, channels)


def numpy_voxel_values(orc, pts, attr, g):
    """Per-voxel round-half-up mean and first row by numpy (np.unique inverse
    map, np.add.at sums, the minimum index per voxel)."""
    keys = orc.quantize(pts, g)
    uk, inv = np.unique(keys, return_inverse=True)
    sums = np.zeros((len(uk), attr.shape[1]), np.int64)
    np.add.at(sums, inv, attr.astype(np.int64))
    cnt = np.bincount(inv, minlength=len(uk)).astype(np.int64)[:, None]
    mean = (sums + cnt // 2) // cnt
    first_idx = np.full(len(uk), len(pts), np.int64)
    np.minimum.at(first_idx, inv, np.arange(len(pts)))
    return mean.astype(np.uint8), attr[first_idx]


def test_average_and_first_match_numpy(orc):
    pts, attr = random_cloud(20000, 21, 3)
    g = orc.grid_from_box([0, 0, 0], 1.0, 4)  # 4096 voxels: many duplicates
    mean, first = numpy_voxel_values(orc, pts, attr, g)
    _, va = orc.build_values(pts, attr, g, policy="average")
    _, vf = orc.build_values(pts, attr, g, policy="first")
    np.testing.assert_array_equal(va, mean)
    np.testing.assert_array_equal(vf, first)


def test_identical_attributes_average_to_themselves(orc):
    pts = synth.uniform_cube(8000, seed=31)
    g = orc.grid_from_box([0, 0, 0], 1.0, 3)
    keys = orc.quantize(pts, g)
    attr = np.stack([(keys * 37 + c) % 256 for c in range(3)], 1).astype(np.uint8)
    c, va = orc.build_values(pts, attr, g, policy="average")
    expect = np.stack([(orc.decode_keys(c) * 37 + ch) % 256 for ch in range(3)], 1)
    np.testing.assert_array_equal(va, expect.astype(np.uint8))
    _, vf = orc.build_values(pts, attr, g, policy="first")
    np.testing.assert_array_equal(vf, va)


def test_average_is_permutation_invariant_and_first_follows_the_point(orc):
    pts, attr = random_cloud(6000, 41, 2)
    g = orc.grid_from_box([0, 0, 0], 1.0, 4)
    perm = np.random.default_rng(42).permutation(len(pts))
    _, v1 = orc.build_values(pts, attr, g, policy="average")
    _, v2 = orc.build_values(pts[perm], attr[perm], g, policy="average")
    np.testing.assert_array_equal(v1, v2)
    # first under a permutation = the row of the point that comes first in it
    _, vf = orc.build_values(pts[perm], attr[perm], g, policy="first")
    _, expect = numpy_voxel_values(orc, pts[perm], attr[perm], g)
    np.testing.assert_array_equal(vf, expect)


def test_rounding_half_up_cases(orc):
    g = unit_grid(orc, 2)
    for vals, expect in (([1, 2], 2), ([0, 255], 128), ([0, 0, 1], 0), ([0, 1, 1], 1),
                         ([255] * 7, 255), ([254, 255], 255), ([3, 4, 4, 4], 4)):
        pts = np.zeros((len(vals), 3), np.float32)
        _, v = orc.build_values(pts, np.array(vals, np.uint8), g, policy="average")
        assert v.tolist() == [[expect]], (vals, v)


@pytest.mark.parametrize("policy", ["base", "average"])
def test_merge_closed_forms(orc, policy):
    pts, attr = random_cloud(4000, 51, 3)
    pts2, attr2 = random_cloud(3000, 52, 3)
    g = orc.grid_from_box([0, 0, 0], 1.0, 5)
    a, va = orc.build_values(pts, attr, g)
    b, vb = orc.build_values(pts2, attr2, g)
    # with itself: the same rows under both policies
    m, vm = orc.merge_values(a, va, a, va, policy=policy)
    np.testing.assert_array_equal(vm, va)
    # with an empty cloud: the other side's rows
    e, ve = orc.build_values(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.uint8), g)
    np.testing.assert_array_equal(orc.merge_values(a, va, e, ve, policy=policy)[1], va)
    np.testing.assert_array_equal(orc.merge_values(e, ve, b, vb, policy=policy)[1], vb)
    # geometry is the plain merge; rows follow the rule voxel by voxel
    m, vm = orc.merge_values(a, va, b, vb, policy=policy)
    ref = orc.merge(a, b)
    np.testing.assert_array_equal(orc.decode_keys(m), orc.decode_keys(ref))
    ka, kb, km = orc.decode_keys(a), orc.decode_keys(b), orc.decode_keys(m)
    ia = {int(k): i for i, k in enumerate(ka)}
    ib = {int(k): i for i, k in enumerate(kb)}
    for p, k in enumerate(km):
        k = int(k)
        if k in ia and k in ib:
            want = va[ia[k]] if policy == "base" else (va[ia[k]].astype(int) + vb[ib[k]] + 1) // 2
        else:
            want = va[ia[k]] if k in ia else vb[ib[k]]
        np.testing.assert_array_equal(vm[p], want)


def test_average_merge_is_commutative(orc):
    pts, attr = random_cloud(4000, 61, 2)
    pts2, attr2 = random_cloud(4000, 62, 2)
    g = orc.grid_from_box([0, 0, 0], 1.0, 4)
    a, va = orc.build_values(pts, attr, g)
    b, vb = orc.build_values(pts2, attr2, g)
    np.testing.assert_array_equal(orc.merge_values(a, va, b, vb, "average")[1],
                                  orc.merge_values(b, vb, a, va, "average")[1])


def test_invalid_arguments(orc):
    g = unit_grid(orc, 3)
    pts = np.zeros((2, 3), np.float32)
    with pytest.raises(orc.OracleError):
        orc.build_values(pts, np.zeros((2, 5), np.uint8), g)
