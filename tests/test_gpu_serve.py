"""Served loop: every request's result is the same in the continuous-batching
mix as when it runs alone through the plain single calls (bit for bit; all
outputs are integers), under a tight and a loose memory budget, and the
per-request timestamps are ordered."""
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


def make_pool(cg, k=6):
    g = cg.grid_from_box([-128.0] * 3, 256.0, 16)
    sizes = synth.log_uniform_ints(k, 3_000, 200_000, seed=77)
    pool, worlds = [], []
    for i, n in enumerate(sizes):
        scene = synth.lidar_sweeps(1, 64, max(1, int(n) // 64), seed=500 + i, n_boxes=8)
        pool.append(cg.cga_build(dev(scene.sweeps[0]), g, xform=scene.poses[0]))
        worlds.append(scene.world)
    return g, pool, worlds


def make_requests(worlds, n_req, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for r in range(n_req):
        if rng.random() < 0.7:
            a = int(rng.integers(len(worlds)))
            m = int(np.exp(rng.uniform(0, np.log(40_000))))
            q = synth.jitter_queries(worlds[a], m, 0.2, seed=seed * 1000 + r)
            reqs.append(("nn", a, q))
        else:
            a, b = (int(v) for v in rng.integers(len(worlds), size=2))
            reqs.append(("mp", a, b, ["xy", "xz", "yz"][int(rng.integers(3))]))
    return reqs


def run_alone(cg, pool, req):
    if req[0] == "nn":
        idx, d2 = cg.cga_nn_query(pool[req[1]], dev(req[2]))
        torch.cuda.synchronize()
        return idx.cpu().numpy(), d2.cpu().numpy()
    m = cg.cga_merge(pool[req[1]], pool[req[2]])
    p = cg.cga_project(m, req[3])
    return m.download(), p.download()


@pytest.mark.parametrize("budget_mb,slots,max_batch", [(2048, 4, 16), (24, 2, 3)])
def test_mix_equals_alone(cg, budget_mb, slots, max_batch):
    g, pool, worlds = make_pool(cg)
    reqs = make_requests(worlds, 60, seed=budget_mb)
    server = cg.Server(pool, memory_budget=budget_mb << 20, slots=slots, max_batch=max_batch)
    tickets = {}
    for req in reqs:
        if req[0] == "nn":
            q = dev(req[2])
            m = q.shape[0]
            idx = torch.empty(m, dtype=torch.int32, device="cuda")
            d2 = torch.empty(m, dtype=torch.int64, device="cuda")
            t = server.submit_nn(req[1], q, idx, d2)
            tickets[t] = (req, idx, d2)
        else:
            t = server.submit_merge_project(req[1], req[2], req[3])
            tickets[t] = (req, None, None)
    server.drain()
    done = server.poll(max_n=len(reqs) + 10)
    assert len(done) == len(reqs)
    for c in done:
        assert c["status"] == cg.OK
        assert c["t_submit_ns"] <= c["t_start_ns"] <= c["t_done_ns"]
        req, idx, d2 = tickets[c["ticket"]]
        alone = run_alone(cg, pool, req)
        if req[0] == "nn":
            assert np.array_equal(idx.cpu().numpy(), alone[0])
            assert np.array_equal(d2.cpu().numpy(), alone[1])
        else:
            got_m, got_p = c["merged"].download(), c["projected"].download()
            for k in got_m:
                assert np.array_equal(got_m[k], alone[0][k]), k
            for k in got_p:
                assert np.array_equal(got_p[k], alone[1][k]), k
    server.free()


def test_server_rejects_bad_requests(cg):
    g, pool, worlds = make_pool(cg, k=2)
    other = cg.cga_build(dev(synth.uniform_cube(100, seed=3)), cg.grid_from_box([0] * 3, 1.0, 10))
    server = cg.Server(pool + [other], memory_budget=1 << 20, slots=1, max_batch=4)
    with pytest.raises(cg.CgaError) as e:
        server.submit_merge_project(0, 2, "xy")
    assert e.value.code == cg.ERR_GRID_MISMATCH
    big = torch.zeros((500_000, 3), dtype=torch.float32, device="cuda")
    idx = torch.empty(500_000, dtype=torch.int32, device="cuda")
    d2 = torch.empty(500_000, dtype=torch.int64, device="cuda")
    with pytest.raises(cg.CgaError) as e:
        server.submit_nn(0, big, idx, d2)   # footprint above the 1 MiB budget
    assert e.value.code == cg.ERR_OOM
    server.free()


def test_served_results_match_oracle(cg, orc):
    """Served results against the CPU oracle at serving sizes: a pool of six
    LiDAR and surface clouds of 0.1M to 4M points (16-bit grid), NN requests
    of up to 1M jittered queries and merge + projection requests, all in one
    continuous-batching mix.  Every merge and projection is compared whole
    with orc.merge and orc.project; for every NN request a seeded sample of
    queries is compared with the oracle's window search and every answer is
    checked to be a stored voxel at exactly the reported squared distance."""
    import oracle_threads
    from paper_2110_11616_gb300 import synth_gpu
    g = cg.grid_from_box([-128.0] * 3, 256.0, 16)
    og = orc.grid_from_box([-128.0] * 3, 256.0, 16)
    sizes = [100_000, 4_000_000, 350_000, 1_500_000, 800_000, 2_500_000]
    pool, opool, pts = [], [], []
    for i, n in enumerate(sizes):
        p = (synth_gpu.lidar_cloud(n, seed=700 + i) if i % 2 == 0 else
             synth_gpu.surface_cloud(n, seed=700 + i, n_objects=40))
        if i % 2 == 1:  # surface clouds centred in the LiDAR box
            p = (p - 50.0).contiguous()
        pool.append(cg.cga_build(p, g))
        ph = p.cpu().numpy()
        opool.append(orc.build(ph, og))
        pts.append(p)
    rng = np.random.default_rng(701)
    reqs = []
    for r in range(24):
        if r % 3 != 2:
            a = int(rng.integers(len(pool)))
            m = 1_000_000 if r == 0 else int(np.exp(rng.uniform(0, np.log(1_000_000))))
            q = synth_gpu.jitter_queries(pts[a], m, 0.2, seed=7000 + r)
            reqs.append(("nn", a, q))
        else:
            a, b = (int(v) for v in rng.integers(len(pool), size=2))
            reqs.append(("mp", a, b, ["xy", "xz", "yz"][int(rng.integers(3))]))
    server = cg.Server(pool, memory_budget=8 << 30, slots=4, max_batch=16)
    tickets = {}
    for req in reqs:
        if req[0] == "nn":
            m = req[2].shape[0]
            idx = torch.empty(m, dtype=torch.int32, device="cuda")
            d2 = torch.empty(m, dtype=torch.int64, device="cuda")
            tickets[server.submit_nn(req[1], req[2], idx, d2)] = (req, idx, d2)
        else:
            tickets[server.submit_merge_project(req[1], req[2], req[3])] = (req, None, None)
    server.drain()
    done = server.poll(max_n=len(reqs) + 10)
    assert len(done) == len(reqs)
    decoded = {}
    for c in done:
        assert c["status"] == cg.OK
        req, idx, d2 = tickets[c["ticket"]]
        if req[0] == "nn":
            a = req[1]
            oa = opool[a]
            qh = req[2].cpu().numpy()
            gi = idx.cpu().numpy().view(np.uint32)
            gd = d2.cpu().numpy().view(np.uint64)
            pick = np.random.default_rng(702 + c["ticket"]).choice(
                len(qh), size=min(3000, len(qh)), replace=False)
            oi, od = oracle_threads.nn_window(orc, oa, og, qh[pick])
            np.testing.assert_array_equal(gd[pick], od, err_msg=f"request {c['ticket']} dist2")
            np.testing.assert_array_equal(gi[pick], oi, err_msg=f"request {c['ticket']} idx")
            if a not in decoded:
                decoded[a] = orc.decode(oa).astype(np.int64)
            qv, ok = orc.query_voxels(og, qh)
            assert ok.all() and np.all(gi < oa.u)
            rd = ((qv - decoded[a][gi]) ** 2).sum(1).astype(np.uint64)
            np.testing.assert_array_equal(rd, gd, err_msg=f"request {c['ticket']} consistency")
        else:
            om = orc.merge(opool[req[1]], opool[req[2]])
            got_m = c["merged"].download()
            for k in ("X_index", "X_pointer", "Y_index", "Y_pointer", "Z_index"):
                np.testing.assert_array_equal(got_m[k], getattr(om, k), err_msg=f"merge {k}")
            op = orc.project(om, req[3])
            got_p = c["projected"].download()
            for k in ("U_index", "U_pointer", "V_index"):
                np.testing.assert_array_equal(got_p[k], getattr(op, k), err_msg=f"{req[3]} {k}")
    server.free()
