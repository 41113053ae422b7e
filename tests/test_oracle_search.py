"""Pins of the oracle's radius search and k-NN (the Eq. 8 set generalised
to a radius and to the k nearest): closed forms on a full lattice (the
voxels within r^2 = 1, 2, 3 of an interior voxel are 7, 19 and 27; its 7
nearest are itself and the 6 face neighbours), agreement of k = 1 with the
exhaustive NN, vectorised numpy distances over the decoded voxels,
consistency between the two searches, and the sentinel rules."""
import numpy as np
import pytest

from paper_2110_11616_gb300 import synth

EMPTY32, EMPTY64 = np.uint32(0xFFFFFFFF), np.uint64(0xFFFFFFFFFFFFFFFF)


def lattice(orc, k=9, bits=5):
    ax = np.arange(k, dtype=np.float32)
    vox = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1).reshape(-1, 3)
    g = orc.Grid(bits, 1.0, (0.0, 0.0, 0.0))
    return orc.build(vox, g), g


@pytest.mark.parametrize("r2,count", [(0, 1), (1, 7), (2, 19), (3, 27), (4, 33)])
def test_lattice_radius_closed_form(orc, r2, count):
    a, g = lattice(orc)
    q = np.array([[4.5, 4.5, 4.5]], np.float32)  # voxel (4, 4, 4)
    off, idx, d2 = orc.radius(a, g, q, r2)
    assert int(off[-1]) == count
    assert (np.diff(idx.astype(np.int64)) > 0).all()  # ascending CGA index


def test_lattice_knn_closed_form(orc):
    a, g = lattice(orc)
    idx, d2 = orc.knn(a, g, np.array([[4.5, 4.5, 4.5]], np.float32), 7)
    assert d2[0].tolist() == [0, 1, 1, 1, 1, 1, 1]
    vox = orc.decode(a)[idx[0]].tolist()
    # ties broken by the smaller key: x-major, then y, then z
    assert vox == [[4, 4, 4], [3, 4, 4], [4, 3, 4], [4, 4, 3], [4, 4, 5], [4, 5, 4], [5, 4, 4]]


def test_knn_one_is_the_nn(orc):
    g = orc.grid_from_box([0, 0, 0], 1.0, 7)
    a = orc.build(synth.uniform_cube(4000, seed=3), g)
    q = synth.uniform_queries(300, 4, [-0.2] * 3, 1.4)
    ki, kd = orc.knn(a, g, q, 1)
    ni, nd = orc.nn_brute(a, g, q)
    np.testing.assert_array_equal(ki[:, 0], ni)
    np.testing.assert_array_equal(kd[:, 0], nd)


def numpy_distances(orc, a, g, q):
    vox = orc.decode(a).astype(np.int64)
    qv, ok = orc.query_voxels(g, q)
    d = ((vox[None, :, :] - qv[:, None, :]) ** 2).sum(-1)
    return d, ok


def test_against_numpy(orc):
    g = orc.grid_from_box([0, 0, 0], 1.0, 6)
    a = orc.build(synth.uniform_cube(2500, seed=5), g)
    q = synth.uniform_queries(120, 6, [-0.1] * 3, 1.2)
    d, ok = numpy_distances(orc, a, g, q)
    off, idx, d2 = orc.radius(a, g, q, 30)
    for j in range(len(q)):
        sel = np.flatnonzero(d[j] <= 30) if ok[j] else np.zeros(0, np.int64)
        np.testing.assert_array_equal(idx[off[j]:off[j + 1]], sel)
        np.testing.assert_array_equal(d2[off[j]:off[j + 1]], d[j][sel])
    ki, kd = orc.knn(a, g, q, 12)
    for j in range(len(q)):
        order = np.lexsort((np.arange(a.u), d[j]))[:12]
        np.testing.assert_array_equal(ki[j], order)
        np.testing.assert_array_equal(kd[j], d[j][order])


def test_radius_and_knn_agree(orc):
    g = orc.grid_from_box([0, 0, 0], 1.0, 6)
    a = orc.build(synth.uniform_cube(3000, seed=7), g)
    q = synth.uniform_queries(80, 8, [0.0] * 3, 1.0)
    ki, kd = orc.knn(a, g, q, 64)
    for r2 in (4, 20, 60):
        off, idx, _ = orc.radius(a, g, q, r2)
        counts = np.diff(off.astype(np.int64))
        inside = (kd <= r2).sum(1)
        # whenever fewer than k voxels are inside, the k-NN list holds all of them
        full = inside < 64
        np.testing.assert_array_equal(counts[full], inside[full])


def test_sentinels(orc):
    g = orc.grid_from_box([0, 0, 0], 1.0, 4)
    a = orc.build(synth.uniform_cube(5, seed=9), g)
    q = np.array([[0.5, 0.5, 0.5], [np.nan, 0, 0]], np.float32)
    ki, kd = orc.knn(a, g, q, 8)
    assert (ki[0, a.u:] == EMPTY32).all() and (kd[0, a.u:] == EMPTY64).all()
    assert (ki[1] == EMPTY32).all()
    off, idx, d2 = orc.radius(a, g, q, 10 ** 6)
    assert int(off[1] - off[0]) == a.u and int(off[2] - off[1]) == 0
