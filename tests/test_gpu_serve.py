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
