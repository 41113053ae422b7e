"""GPU parity of the Value array (Sec. V): per-voxel attribute rows of
builds (average or first point) and merges (base or average) equal the CPU
oracle's byte for byte, together with the geometry."""
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


def dev_u8(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint8)).cuda()


def check(cg, gpu, o, ov, what=""):
    d = gpu.download()
    for lv in LEVELS:
        np.testing.assert_array_equal(d[lv], getattr(o, lv), err_msg=f"{what} {lv}")
    v = cg.cga_values(gpu)
    np.testing.assert_array_equal(v.cpu().numpy(), ov, err_msg=f"{what} values")


def cloud(n, seed, channels, lo=-0.02, extent=1.04):
    pts = synth.uniform_cube(n, seed=seed, lo=lo, extent=extent)
    attr = np.random.default_rng(seed + 1).integers(0, 256, size=(n, channels), dtype=np.uint8)
    return pts, attr


@pytest.mark.parametrize("policy", ["average", "first"])
@pytest.mark.parametrize("n,bits", [(0, 10), (1, 10), (TILE + 3, 10), (50_000, 5), (100_000, 16),
                                    (70_000, 12)])
@pytest.mark.parametrize("channels", [1, 3, 4])
def test_build_values_parity(cg, orc, policy, n, bits, channels):
    pts, attr = cloud(n, 7 * n + bits + channels, channels)
    g, og = cg.grid_from_box([0, 0, 0], 1.0, bits), orc.grid_from_box([0, 0, 0], 1.0, bits)
    a = cg.cga_build_values(dev(pts), dev_u8(attr), g, policy=policy)
    o, ov = orc.build_values(pts, attr, og, policy=policy)
    check(cg, a, o, ov, f"{policy} n={n} b={bits} c={channels}")


@pytest.mark.parametrize("policy", ["average", "first"])
def test_build_values_with_transform(cg, orc, policy):
    pts, attr = cloud(60_000, 3, 3)
    X = synth.rigid_xform(seed=4)
    g, og = cg.grid_from_box([0, 0, 0], 1.0, 8), orc.grid_from_box([0, 0, 0], 1.0, 8)
    a = cg.cga_build_values(dev(pts), dev_u8(attr), g, xform=X, policy=policy)
    o, ov = orc.build_values(pts, attr, og, xform=X, policy=policy)
    check(cg, a, o, ov, policy)


def test_many_points_in_one_voxel(cg, orc):
    n = 300_000
    pts = np.full((n, 3), 0.5, np.float32)
    attr = np.stack([np.full(n, 255), np.arange(n) % 256, np.arange(n) % 7], 1).astype(np.uint8)
    g, og = cg.grid_from_box([0, 0, 0], 1.0, 10), orc.grid_from_box([0, 0, 0], 1.0, 10)
    for policy in ("average", "first"):
        a = cg.cga_build_values(dev(pts), dev_u8(attr), g, policy=policy)
        o, ov = orc.build_values(pts, attr, og, policy=policy)
        check(cg, a, o, ov, policy)


@pytest.mark.parametrize("policy", ["base", "average"])
@pytest.mark.parametrize("bits", [6, 10, 16])
def test_merge_values_parity(cg, orc, policy, bits):
    pts, attr = cloud(40_000, 11 + bits, 3)
    pts2, attr2 = cloud(30_000, 21 + bits, 3)
    X = synth.rigid_xform(seed=bits)
    g, og = cg.grid_from_box([0, 0, 0], 1.0, bits), orc.grid_from_box([0, 0, 0], 1.0, bits)
    a = cg.cga_build_values(dev(pts), dev_u8(attr), g)
    b = cg.cga_build_values(dev(np.concatenate([pts[:20_000], pts2])),
                            dev_u8(np.concatenate([attr2[:20_000], attr2])), g, xform=None)
    oa, ova = orc.build_values(pts, attr, og)
    ob, ovb = orc.build_values(np.concatenate([pts[:20_000], pts2]),
                               np.concatenate([attr2[:20_000], attr2]), og)
    m = cg.cga_merge_values(a, b, policy=policy)
    om, ovm = orc.merge_values(oa, ova, ob, ovb, policy=policy)
    check(cg, m, om, ovm, f"{policy} b={bits}")
    # the twin under a rigid transform (the Sec. II-A use)
    t = cg.cga_build_values(dev(pts), dev_u8(attr), g, xform=X)
    ot, ovt = orc.build_values(pts, attr, og, xform=X)
    m2 = cg.cga_merge_values(a, t, policy=policy)
    om2, ovm2 = orc.merge_values(oa, ova, ot, ovt, policy=policy)
    check(cg, m2, om2, ovm2, f"{policy} twin b={bits}")


@pytest.mark.parametrize("policy", ["base", "average"])
def test_merge_values_identities(cg, orc, policy):
    pts, attr = cloud(20_000, 31, 2)
    g, og = cg.grid_from_box([0, 0, 0], 1.0, 7), orc.grid_from_box([0, 0, 0], 1.0, 7)
    a = cg.cga_build_values(dev(pts), dev_u8(attr), g)
    e = cg.cga_build_values(dev(np.zeros((0, 3))), dev_u8(np.zeros((0, 2))), g)
    oa, ova = orc.build_values(pts, attr, og)
    check(cg, cg.cga_merge_values(a, a, policy=policy), oa, ova, "self")
    check(cg, cg.cga_merge_values(a, e, policy=policy), oa, ova, "with empty")
    check(cg, cg.cga_merge_values(e, a, policy=policy), oa, ova, "empty base")


def test_value_arguments(cg):
    pts, attr = cloud(100, 41, 3)
    g = cg.grid_from_box([0, 0, 0], 1.0, 8)
    with pytest.raises(cg.CgaError):
        cg.cga_build_values(dev(pts), dev_u8(np.zeros((100, 5))), g)
    plain = cg.cga_build(dev(pts), g)
    assert cg.cga_values(plain) is None
    a = cg.cga_build_values(dev(pts), dev_u8(attr), g)
    with pytest.raises(cg.CgaError):
        cg.cga_merge_values(a, plain)
    b2 = cg.cga_build_values(dev(pts), dev_u8(attr[:, :2].copy()), g)
    with pytest.raises(cg.CgaError):
        cg.cga_merge_values(a, b2)
