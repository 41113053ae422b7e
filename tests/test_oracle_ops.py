"""Pins for the oracle's merge (a5), projection (a6) and NN search (a7).

Merge: Eq. 1 (set union) -- checked against numpy.union1d, the hand fixture,
and the algebra of a union (idempotent, identity, commutative, associative).
Projection: Eq. 3 with m = 1 -- checked against numpy.unique of the 2D voxels,
the hand fixtures, the xy identity with the CGA's own top two levels, and the
closed form of a lattice.  NN: Eq. 7-8 -- the exhaustive oracle against a
vectorised numpy search, the Sec. V-C window oracle against the exhaustive
one, hand-built ties, a stored voxel, and the closed form of a full lattice.
"""
import numpy as np
import pytest

import exact_f32 as ex
from golden_io import load_cases, voxels_to_float
from paper_2110_11616_gb300 import synth

CASES = load_cases()
LEVELS = ("X_index", "X_pointer", "Y_index", "Y_pointer", "Z_index")


def unit_grid(orc, bits):
    return orc.Grid(bits, 1.0, (0.0, 0.0, 0.0))


def same(a, b):
    return all(np.array_equal(getattr(a, lv), getattr(b, lv)) for lv in LEVELS)


def cloud(orc, n, seed, bits, xform=None):
    g = orc.grid_from_box([0, 0, 0], 1.0, bits)
    return orc.build(synth.uniform_cube(n, seed=seed), g, xform=xform), g


# ---------------------------------------------------------------- merge (Eq. 1)
def test_merge_fixture(orc):
    c = CASES["merge_six_points"]
    g = unit_grid(orc, c["bits"])
    m = orc.merge(orc.build(voxels_to_float(c["a"]), g), orc.build(voxels_to_float(c["b"]), g))
    for lv in LEVELS:
        assert np.array_equal(getattr(m, lv), c[lv]), lv


@pytest.mark.parametrize("bits", [3, 8, 10, 16])
def test_merge_is_union1d(orc, bits):
    a, g = cloud(orc, 3000, 21, bits)
    b, _ = cloud(orc, 2000, 22, bits, xform=synth.rigid_xform(23))
    m = orc.merge(a, b)
    assert np.array_equal(orc.decode_keys(m),
                          np.union1d(orc.decode_keys(a), orc.decode_keys(b)))


def test_merge_algebra(orc):
    a, _ = cloud(orc, 1500, 31, 6)
    b, _ = cloud(orc, 1500, 32, 6)
    c, _ = cloud(orc, 1500, 33, 6)
    empty = orc.build(np.zeros((0, 3), np.float32), orc.grid_from_box([0, 0, 0], 1.0, 6))
    assert same(orc.merge(a, a), a)
    assert same(orc.merge(a, empty), a) and same(orc.merge(empty, a), a)
    assert same(orc.merge(a, b), orc.merge(b, a))
    assert same(orc.merge(orc.merge(a, b), c), orc.merge(a, orc.merge(b, c)))


# ------------------------------------------------------------ projection (Eq. 3)
@pytest.mark.parametrize("name", ["six_points", "one_column", "one_x_many_y",
                                  "single_point", "empty"])
@pytest.mark.parametrize("plane", ["xy", "xz", "yz"])
def test_project_fixture(orc, name, plane):
    c = CASES[name]
    p = orc.project(orc.build(voxels_to_float(c["points"]), unit_grid(orc, c["bits"])), plane)
    for lv in ("U_index", "U_pointer", "V_index"):
        assert np.array_equal(getattr(p, lv), c[f"{plane}.{lv}"]), (name, plane, lv)


@pytest.mark.parametrize("bits", [4, 10, 16])
def test_project_equals_numpy_unique(orc, bits):
    a, _ = cloud(orc, 5000, 41, bits)
    xyz = orc.decode(a).astype(np.int64)
    for plane, (i, j) in {"xy": (0, 1), "xz": (0, 2), "yz": (1, 2)}.items():
        p = orc.project(a, plane)
        uv = np.unique(xyz[:, [i, j]], axis=0)
        ui, counts = np.unique(uv[:, 0], return_counts=True)
        assert np.array_equal(p.U_index, ui)
        assert np.array_equal(p.U_pointer, np.concatenate([[0], np.cumsum(counts)]))
        assert np.array_equal(p.V_index, uv[:, 1])


def test_project_xy_is_top_two_levels(orc):
    a, _ = cloud(orc, 8000, 42, 9)
    p = orc.project(a, "xy")
    assert np.array_equal(p.U_index, a.X_index)
    assert np.array_equal(p.U_pointer, a.X_pointer)
    assert np.array_equal(p.V_index, a.Y_index)


@pytest.mark.parametrize("plane", ["xy", "xz", "yz"])
def test_project_lattice_is_square(orc, plane):
    k = 6
    ax = np.arange(k)
    vox = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1).reshape(-1, 3)
    p = orc.project(orc.build(voxels_to_float(vox), unit_grid(orc, 3)), plane)
    assert np.array_equal(p.U_index, ax)
    assert np.array_equal(p.U_pointer, np.arange(k + 1) * k)
    assert np.array_equal(p.V_index, np.tile(ax, k))


# ------------------------------------------------------------------ NN (Eq. 7-8)
def numpy_nn(orc, a, grid, q):
    """Vectorised exhaustive search: int64 squared distances, lexsort on
    (distance, key) -- a different technique from the oracle's scan."""
    keys = orc.decode_keys(a).astype(np.uint64)
    xyz = orc.decode(a).astype(np.int64)
    qi = np.array([[ex.quantize_query_axis(p[k], grid.scale, grid.offset[k]) for k in range(3)]
                   for p in q], np.int64)
    d2 = ((qi[:, None, :] - xyz[None, :, :]) ** 2).sum(-1)
    idx = np.empty(len(q), np.uint32)
    best = np.empty(len(q), np.uint64)
    for j in range(len(q)):
        order = np.lexsort((keys, d2[j]))
        idx[j] = order[0]
        best[j] = d2[j, order[0]]
    return idx, best


@pytest.mark.parametrize("bits,n,seed", [(3, 40, 51), (5, 300, 52), (8, 800, 53)])
def test_nn_brute_matches_numpy(orc, bits, n, seed):
    a, g = cloud(orc, n, seed, bits)
    q = synth.uniform_queries(150, seed + 100, [-0.2, -0.2, -0.2], 1.4)
    i1, d1 = orc.nn_brute(a, g, q)
    i2, d2 = numpy_nn(orc, a, g, q)
    assert np.array_equal(i1, i2) and np.array_equal(d1, d2)


@pytest.mark.parametrize("bits,n,seed", [(2, 10, 61), (4, 200, 62), (7, 3000, 63),
                                         (10, 5000, 64), (16, 2000, 65)])
def test_nn_window_matches_brute(orc, bits, n, seed):
    a, g = cloud(orc, n, seed, bits)
    q = np.concatenate([
        synth.uniform_queries(400, seed + 1, [0, 0, 0], 1.0),
        synth.uniform_queries(100, seed + 2, [-3, -3, -3], 7.0),   # far outside the box
        synth.uniform_cube(n, seed=seed)[:100],                    # on stored voxels
    ])
    iw, dw = orc.nn_window(a, g, q)
    ib, db = orc.nn_brute(a, g, q)
    assert np.array_equal(iw, ib) and np.array_equal(dw, db)


def test_nn_on_stored_voxel(orc):
    a, g = cloud(orc, 2000, 71, 10)
    pts = synth.uniform_cube(2000, seed=71)
    for fn in (orc.nn_brute, orc.nn_window):
        idx, d2 = fn(a, g, pts[:200])
        keys = orc.decode_keys(a)
        qk = orc.quantize(pts[:200], g)
        assert np.all(d2 == 0) and np.array_equal(keys[idx], qk)


def test_nn_ties_take_smaller_key(orc):
    g = unit_grid(orc, 4)
    # (0,0,0) and (2,0,0) are both at distance 1 from (1,0,0).
    a = orc.build(voxels_to_float([[2, 0, 0], [0, 0, 0]]), g)
    # (0,0,2) and (0,2,0) are both at squared distance 2 from (0,1,1); key(0,0,2) = 2 is smaller.
    b = orc.build(voxels_to_float([[0, 2, 0], [0, 0, 2]]), g)
    # four voxels tied around (5,5,5) at squared distance 1; (4,5,5) has the smallest key.
    c = orc.build(voxels_to_float([[6, 5, 5], [5, 6, 5], [5, 5, 6], [4, 5, 5], [5, 4, 5]]), g)
    for fn in (orc.nn_brute, orc.nn_window):
        i, d = fn(a, g, np.array([[1.0, 0.0, 0.0]], np.float32))
        assert (int(i[0]), int(d[0])) == (0, 1)
        i, d = fn(b, g, np.array([[0.0, 1.0, 1.0]], np.float32))
        assert (int(i[0]), int(d[0])) == (0, 2)
        i, d = fn(c, g, np.array([[5.0, 5.0, 5.0]], np.float32))
        assert (int(i[0]), int(d[0])) == (0, 1)


def test_nn_full_lattice_is_clamp(orc):
    k = 7
    ax = np.arange(k)
    vox = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1).reshape(-1, 3)
    g = unit_grid(orc, 3)
    a = orc.build(voxels_to_float(vox), g)
    rng = np.random.default_rng(3)
    q = rng.uniform(-20, 30, size=(300, 3)).astype(np.float32)
    qi = np.floor(q.astype(np.float64)).astype(np.int64)
    c = np.clip(qi, 0, k - 1)
    expect_d2 = ((qi - c) ** 2).sum(1)
    expect_idx = c[:, 0] * k * k + c[:, 1] * k + c[:, 2]
    for fn in (orc.nn_brute, orc.nn_window):
        idx, d2 = fn(a, g, q)
        assert np.array_equal(d2.astype(np.int64), expect_d2)
        assert np.array_equal(idx.astype(np.int64), expect_idx)


def test_nn_empty_and_nonfinite(orc):
    g = orc.grid_from_box([0, 0, 0], 1.0, 8)
    empty = orc.build(np.zeros((0, 3), np.float32), g)
    a, _ = cloud(orc, 100, 81, 8)
    q = np.array([[0.5, 0.5, 0.5], [np.nan, 0.1, 0.1], [0.2, np.inf, 0.3]], np.float32)
    for fn in (orc.nn_brute, orc.nn_window):
        idx, d2 = fn(empty, g, q)
        assert np.all(idx == orc.U32_MAX) and np.all(d2 == orc.U64_MAX)
        idx, d2 = fn(a, g, q)
        assert idx[0] != orc.U32_MAX
        assert np.all(idx[1:] == orc.U32_MAX) and np.all(d2[1:] == orc.U64_MAX)


def test_nn_far_query_clamped_to_2_pow_30(orc):
    g = orc.Grid(4, 1.0e9, (0.0, 0.0, 0.0))
    a = orc.build(np.zeros((1, 3), np.float32), g)
    idx, d2 = orc.nn_brute(a, g, np.array([[10.0, -10.0, 0.0]], np.float32))
    assert int(d2[0]) == 2 * (1 << 60)
