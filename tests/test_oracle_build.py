"""Pins for the oracle's build (a1-a3) and decode (a4).

Expected values: the hand-derived fixtures of tests/golden/cga_fixtures.txt
(Sec. V recurrences worked by hand), the closed form of a full lattice,
the structural invariants of the Sec. V arrays, and numpy's own
sort/unique routines (independent of the oracle's std::sort/std::unique).
"""
import numpy as np
import pytest

from golden_io import load_cases, voxels_to_float
from paper_2110_11616_gb300 import synth

CASES = load_cases()
LEVELS = ("X_index", "X_pointer", "Y_index", "Y_pointer", "Z_index")


def unit_grid(orc, bits):
    return orc.Grid(bits, 1.0, (0.0, 0.0, 0.0))


@pytest.mark.parametrize("name", [n for n in CASES if "points" in CASES[n]])
def test_fixture_arrays(orc, name):
    c = CASES[name]
    a = orc.build(voxels_to_float(c["points"]), unit_grid(orc, c["bits"]))
    for lv in LEVELS:
        assert np.array_equal(getattr(a, lv), c[lv]), (name, lv)


def check_invariants(a, n=None):
    """Structural facts of the Sec. V arrays."""
    h, g, u = a.h, a.g, a.u
    assert h <= g <= u and (n is None or u <= n)
    assert len(a.X_pointer) == h + 1 and len(a.Y_pointer) == g + 1
    assert a.X_pointer[0] == 0 and a.X_pointer[-1] == g
    assert a.Y_pointer[0] == 0 and a.Y_pointer[-1] == u
    assert np.all(np.diff(a.X_index.astype(np.int64)) > 0)
    assert np.all(np.diff(a.X_pointer.astype(np.int64)) > 0)
    assert np.all(np.diff(a.Y_pointer.astype(np.int64)) > 0)
    for i in range(h):
        ys = a.Y_index[a.X_pointer[i]:a.X_pointer[i + 1]].astype(np.int64)
        assert np.all(np.diff(ys) > 0)
    zs = a.Z_index.astype(np.int64)
    for j in range(g):
        assert np.all(np.diff(zs[a.Y_pointer[j]:a.Y_pointer[j + 1]]) > 0)


def split_keys(keys, b):
    k = keys.astype(np.uint64)
    m = np.uint64((1 << b) - 1)
    return np.stack([k >> np.uint64(2 * b), (k >> np.uint64(b)) & m, k & m], axis=1)


@pytest.mark.parametrize("bits,n,seed", [(4, 500, 1), (6, 3000, 2), (10, 20000, 3),
                                         (16, 5000, 4), (1, 50, 5)])
def test_decode_equals_numpy_unique(orc, bits, n, seed):
    pts = synth.uniform_cube(n, seed=seed, lo=-0.05, extent=1.1)
    g = orc.grid_from_box([0, 0, 0], 1.0, bits)
    a = orc.build(pts, g)
    check_invariants(a, n)
    q = split_keys(orc.quantize(pts, g), bits).astype(np.int64)
    expect = np.unique(q, axis=0)          # lexicographic (x, y, z), duplicates dropped
    got = orc.decode(a).astype(np.int64)
    assert np.array_equal(got, expect)
    assert np.array_equal(orc.decode_keys(a), np.unique(orc.quantize(pts, g)))


@pytest.mark.parametrize("k", [1, 2, 5, 9])
def test_full_lattice_closed_form(orc, k):
    ax = np.arange(k)
    vox = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1).reshape(-1, 3)
    rng = np.random.default_rng(k)
    vox = vox[rng.permutation(len(vox))]
    a = orc.build(voxels_to_float(vox), unit_grid(orc, 4))
    assert np.array_equal(a.X_index, ax)
    assert np.array_equal(a.X_pointer, np.arange(k + 1) * k)
    assert np.array_equal(a.Y_index, np.tile(ax, k))
    assert np.array_equal(a.Y_pointer, np.arange(k * k + 1) * k)
    assert np.array_equal(a.Z_index, np.tile(ax, k * k))


def test_permutation_and_duplication_invariance(orc):
    pts = synth.uniform_cube(4000, seed=7)
    g = orc.grid_from_box([0, 0, 0], 1.0, 7)
    a = orc.build(pts, g)
    rng = np.random.default_rng(0)
    shuffled = pts[rng.permutation(len(pts))]
    doubled = np.concatenate([pts, pts[rng.integers(0, len(pts), 2000)]])
    for other in (orc.build(shuffled, g), orc.build(doubled, g)):
        for lv in LEVELS:
            assert np.array_equal(getattr(a, lv), getattr(other, lv))


def test_from_sorted_keys_roundtrip(orc):
    pts = synth.uniform_cube(5000, seed=8)
    g = orc.grid_from_box([0, 0, 0], 1.0, 8)
    keys = np.unique(orc.quantize(pts, g))
    a = orc.from_sorted_keys(keys, 8)
    assert np.array_equal(orc.decode_keys(a), keys)


def test_all_duplicates(orc):
    pts = np.tile(np.array([[0.3, 0.6, 0.9]], np.float32), (1000, 1))
    a = orc.build(pts, orc.grid_from_box([0, 0, 0], 1.0, 10))
    assert (a.h, a.g, a.u) == (1, 1, 1)
    assert list(a.X_pointer) == [0, 1] and list(a.Y_pointer) == [0, 1]


def test_bytes_formula(orc):
    pts = synth.uniform_cube(3000, seed=9)
    a = orc.build(pts, orc.grid_from_box([0, 0, 0], 1.0, 6))
    total = sum(getattr(a, lv).nbytes for lv in LEVELS)
    assert total == a.nbytes() == 2 * a.h + 4 * (a.h + 1) + 2 * a.g + 4 * (a.g + 1) + 2 * a.u


def test_lookup_finds_every_point_and_nothing_else(orc):
    c = CASES["six_points"]
    a = orc.build(voxels_to_float(c["points"]), unit_grid(orc, 3))
    dec = orc.decode(a)
    for i, (x, y, z) in enumerate(dec):
        assert orc.lookup(a, int(x), int(y), int(z)) == i
    present = {tuple(map(int, r)) for r in dec}
    for x in range(8):
        for y in range(8):
            for z in range(8):
                if (x, y, z) not in present:
                    assert orc.lookup(a, x, y, z) == -1
