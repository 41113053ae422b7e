"""cga_nn_query_noalloc: the NN call for callers that cannot allocate device
memory (fixed memory budgets, real-time loops that must not call cudaMalloc,
allocators owned by another framework).  Its scratch lives in a fixed device
array inside the library, so it must return exactly what cga_nn_query
returns, call after call, with nothing left over from the previous call.

This file is collected last on purpose: a run that stops at the first failure
has then already run every other test."""
import ctypes

import numpy as np
import oracle_threads
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
    lib = cga.load()
    P = ctypes.c_void_p
    lib.cga_nn_query_noalloc.argtypes = [P, P, ctypes.c_uint64, P, P, P]
    return cga


def call_noalloc(cg, a, q):
    m = q.shape[0]
    idx = torch.full((m,), 7, dtype=torch.int32, device="cuda")
    d2 = torch.full((m,), 7, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = cg.load().cga_nn_query_noalloc(a.ptr, ctypes.c_void_p(q.data_ptr()), m,
                                        ctypes.c_void_p(idx.data_ptr()),
                                        ctypes.c_void_p(d2.data_ptr()), ctypes.c_void_p(stream))
    assert rc == cg.OK, rc
    return idx, d2


def test_noalloc_matches_nn_query_on_consecutive_calls(cg):
    pts = synth.uniform_cube(200_000, seed=401)
    g = cg.grid_from_box([0, 0, 0], 1.0, 12)
    a = cg.cga_build(torch.from_numpy(pts).cuda(), g)
    b = cg.cga_build(torch.from_numpy(synth.uniform_cube(30_000, seed=402)).cuda(), g)
    q1 = torch.from_numpy(synth.uniform_queries(300_000, 403, [-0.05] * 3, 1.1)).cuda()
    q2 = torch.from_numpy(synth.uniform_queries(5_000, 404, [0.0] * 3, 1.0)).cuda()
    for cga_h, q in ((a, q1), (b, q2)):
        got_idx, got_d2 = call_noalloc(cg, cga_h, q)
        ref_idx, ref_d2 = cg.cga_nn_query(cga_h, q)
        torch.cuda.synchronize()
        assert torch.equal(got_idx, ref_idx)
        assert torch.equal(got_d2, ref_d2)


def test_noalloc_rejects_more_than_its_capacity(cg):
    g = cg.grid_from_box([0, 0, 0], 1.0, 8)
    a = cg.cga_build(torch.from_numpy(synth.uniform_cube(100, seed=405)).cuda(), g)
    m = cg.NOALLOC_MAX_QUERIES + 1
    rc = cg.load().cga_nn_query_noalloc(a.ptr, ctypes.c_void_p(16), m, ctypes.c_void_p(16),
                                        ctypes.c_void_p(16), None)
    assert rc == cg.ERR_CAPACITY


def test_noalloc_at_capacity_matches_oracle(cg, orc):
    """m = CGA_NOALLOC_MAX_QUERIES on a multi-million-voxel CGA: the worst
    case the fixed array must hold (its size check passes, the call returns
    OK) and the answers equal cga_nn_query's and, on a seeded sample, the
    oracle's; then a call below the Morton-sort threshold."""
    pts = synth.uniform_cube(3_000_000, seed=406)
    g = cg.grid_from_box([0, 0, 0], 1.0, 12)
    og = orc.grid_from_box([0, 0, 0], 1.0, 12)
    a = cg.cga_build(torch.from_numpy(pts).cuda(), g)
    m = cg.NOALLOC_MAX_QUERIES
    qh = synth.uniform_queries(m, 407, [-0.05] * 3, 1.1)
    q = torch.from_numpy(qh).cuda()
    got_idx, got_d2 = call_noalloc(cg, a, q)
    ref_idx, ref_d2 = cg.cga_nn_query(a, q)
    torch.cuda.synchronize()
    assert torch.equal(got_idx, ref_idx) and torch.equal(got_d2, ref_d2)
    oa = orc.build(pts, og)
    pick = np.random.default_rng(408).choice(m, 4000, replace=False)
    oi, od = oracle_threads.nn_window(orc, oa, og, qh[pick])
    assert np.array_equal(got_d2.cpu().numpy().view(np.uint64)[pick], od)
    assert np.array_equal(got_idx.cpu().numpy().view(np.uint32)[pick], oi)
    small = q[:1000].contiguous()
    got_idx, got_d2 = call_noalloc(cg, a, small)
    ref_idx, ref_d2 = cg.cga_nn_query(a, small)
    torch.cuda.synchronize()
    assert torch.equal(got_idx, ref_idx) and torch.equal(got_d2, ref_d2)


@pytest.mark.parametrize("prep", [(3,), (2, 5), "tree"])
def test_noalloc_uses_the_prepared_search(cg, prep):
    """On a handle prepared with coarse levels or the occupancy tree the call
    answers exactly as cga_nn_query does on it (two calls in a row)."""
    from paper_2110_11616_gb300 import synth as sy
    scene = sy.superellipsoid_scene(n_objects=12, seed=409, extent=100.0)
    pts = sy.sample_surfaces(scene, 400_000, seed=410)
    g = cg.grid_from_box([0.0] * 3, 100.0, 12)
    a = cg.cga_build(torch.from_numpy(pts).cuda(), g)
    cg.cga_nn_prepare(a, prep)
    for seed in (411, 412):
        q = torch.from_numpy(sy.uniform_queries(50_000, seed, [-10.0] * 3, 120.0)).cuda()
        got_idx, got_d2 = call_noalloc(cg, a, q)
        ref_idx, ref_d2 = cg.cga_nn_query(a, q)
        torch.cuda.synchronize()
        assert torch.equal(got_idx, ref_idx) and torch.equal(got_d2, ref_d2)
