"""Batched forms: every item of a batched call (and of the pre-planned,
graph-replayed pipeline) equals the CPU oracle's result for that item alone.
Items mix sizes (empty, one point, ragged tiles), grids (1..16 bits, both key
widths) and transforms in one launch set."""
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


def assert_cga(gpu, o, what=""):
    d = gpu.download()
    for lv in LEVELS:
        np.testing.assert_array_equal(d[lv], getattr(o, lv), err_msg=f"{what} {lv}")


def assert_2d(gpu, o, what=""):
    d = gpu.download()
    for lv in ("U_index", "U_pointer", "V_index"):
        np.testing.assert_array_equal(d[lv], getattr(o, lv), err_msg=f"{what} {lv}")


SPECS = [(0, 10), (1, 16), (5000, 1), (100_000, 10), (3 * TILE + 1, 12), (70_000, 16),
         (TILE, 11), (2, 3), (20_000, 8)]


def make_items(cg, orc, seed=0):
    items = []
    for i, (n, bits) in enumerate(SPECS):
        pts = synth.uniform_cube(n, seed=seed + 10 * i, lo=-0.03, extent=1.06)
        X = synth.rigid_xform(seed=seed + 10 * i + 1)
        items.append((pts, X, cg.grid_from_box([0, 0, 0], 1.0, bits),
                      orc.grid_from_box([0, 0, 0], 1.0, bits)))
    return items


def test_build_batch(cg, orc):
    items = make_items(cg, orc)
    pts = [dev(p) for p, _, _, _ in items]
    xs = [X if i % 2 else None for i, (_, X, _, _) in enumerate(items)]
    out = cg.cga_build_batch(pts, [g for _, _, g, _ in items], xs)
    for i, ((p, _, _, og), x) in enumerate(zip(items, xs)):
        assert_cga(out[i], orc.build(p, og, xform=x), f"item {i}")


def test_merge_project_nn_batch(cg, orc):
    items = make_items(cg, orc, seed=100)
    pts = [dev(p) for p, _, _, _ in items]
    grids = [g for _, _, g, _ in items]
    A = cg.cga_build_batch(pts, grids)
    B = cg.cga_build_batch(pts, grids, [X for _, X, _, _ in items])
    M = cg.cga_merge_batch(A, B)
    oms = []
    for i, (p, X, _, og) in enumerate(items):
        om = orc.merge(orc.build(p, og), orc.build(p, og, xform=X))
        assert_cga(M[i], om, f"merge {i}")
        oms.append(om)
    planes = ["xy", "xz", "yz"] * 3
    P = cg.cga_project_batch(M, planes)
    for i, (om, pl) in enumerate(zip(oms, planes)):
        assert_2d(P[i], orc.project(om, pl), f"project {i} {pl}")
    qs = [synth.uniform_queries(500 + 3000 * (i % 4), 7 + i, [-0.1] * 3, 1.2)
          for i in range(len(items))]
    res = cg.cga_nn_query_batch(M, [dev(q) for q in qs])
    for i, ((idx, d2), om, q, (_, _, _, og)) in enumerate(zip(res, oms, qs, items)):
        oi, od = orc.nn_window(om, og, q)
        np.testing.assert_array_equal(d2.cpu().numpy().view(np.uint64), od, err_msg=f"nn {i}")
        np.testing.assert_array_equal(idx.cpu().numpy().view(np.uint32), oi, err_msg=f"nn {i}")


def test_pipeline_and_graph_replay(cg, orc):
    items = make_items(cg, orc, seed=200)
    pts = [dev(p) for p, _, _, _ in items]
    qs = [synth.uniform_queries(0 if i == 2 else 1000 + 2500 * i, 30 + i, [-0.1] * 3, 1.2)
          for i in range(len(items))]
    dq = [dev(q) if len(q) else None for q in qs]
    pipe = cg.Pipeline(pts, [g for _, _, g, _ in items], [X for _, X, _, _ in items], dq)
    expect = []
    for i, (p, X, _, og) in enumerate(items):
        oa, ob = orc.build(p, og), orc.build(p, og, xform=X)
        om = orc.merge(oa, ob)
        oi, od = orc.nn_window(om, og, qs[i]) if len(qs[i]) else (None, None)
        expect.append((oa, ob, om, orc.project(om, "xy"), oi, od))

    def check(tag):
        torch.cuda.synchronize()
        for i, (oa, ob, om, oxy, oi, od) in enumerate(expect):
            assert_cga(pipe.view(i, "cloud"), oa, f"{tag} cloud {i}")
            assert_cga(pipe.view(i, "twin"), ob, f"{tag} twin {i}")
            assert_cga(pipe.view(i, "merged"), om, f"{tag} merged {i}")
            assert_2d(pipe.view_xy(i), oxy, f"{tag} xy {i}")
            if oi is not None:
                np.testing.assert_array_equal(pipe.dist2[i].cpu().numpy().view(np.uint64), od)
                np.testing.assert_array_equal(pipe.idx[i].cpu().numpy().view(np.uint32), oi)

    pipe.run()
    check("run")
    for t in pipe.dist2:
        t.fill_(0)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        pipe.run_graph()
        pipe.run_graph()
    stream.synchronize()
    check("graph")
    pipe.free()
