"""GPU parity of the perspective projection (Eq. 5-6): the z-buffer index and
depth images equal the oracle's bit for bit (the same float operations in the
same order on both sides; cosine and sine are given as floats)."""
import math

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


def angle(theta):
    return float(np.float32(math.cos(theta))), float(np.float32(math.sin(theta)))


def compare(cg, orc, pts, bits, eye, theta, D, W, H, xform=None):
    g, og = cg.grid_from_box([0, 0, 0], 1.0, bits), orc.grid_from_box([0, 0, 0], 1.0, bits)
    a = cg.cga_build(dev(pts), g, xform=xform)
    c, s = angle(theta)
    idx, dep = cg.cga_perspective(a, eye, c, s, D, W, H)
    oi, od = orc.perspective(orc.build(pts, og, xform=xform), eye, c, s, D, W, H)
    np.testing.assert_array_equal(idx.cpu().numpy().view(np.uint32), oi)
    np.testing.assert_array_equal(dep.cpu().numpy(), od)
    return oi


@pytest.mark.parametrize("theta", [0.0, 0.3, -1.1, math.pi / 2, 2.5])
@pytest.mark.parametrize("bits,n", [(8, 20_000), (10, 150_000), (16, 60_000)])
def test_perspective_parity(cg, orc, theta, bits, n):
    pts = synth.uniform_cube(n, seed=bits + n)
    top = float(1 << bits)
    # the camera looks along (sin, 0, cos) after the turn: stand 1.5 grid
    # widths behind the cloud's centre on that line
    c, s = angle(theta)
    eye = [top / 2 - 1.5 * top * s + 0.25, top / 2 - 0.5, top / 2 - 1.5 * top * c]
    oi = compare(cg, orc, pts, bits, eye, theta, 400.0, 320, 240)
    assert (oi != 0xFFFFFFFF).any()


def test_eye_inside_the_cloud(cg, orc):
    # about half the voxels are behind the eye; many share pixels near the centre
    pts = synth.superellipsoid_scene(n_objects=6, seed=9, extent=100.0)
    pts = synth.sample_surfaces(pts, 80_000, seed=10)
    eye = [2048.3, 2048.7, 2048.1]
    for theta in (0.0, 0.8, 3.0):
        compare(cg, orc, pts / 100.0, 12, eye, theta, 500.0, 256, 256)


def test_lidar_frame(cg, orc):
    sc = synth.lidar_sweeps(1, 64, 1024, seed=11, with_world=False)
    pts = (sc.sweeps[0] + 128.0) / 256.0
    compare(cg, orc, pts, 16, [32768.0, 32768.0, 30000.0], 0.4, 800.0, 640, 480)


def test_empty_and_tiny(cg, orc):
    compare(cg, orc, np.zeros((0, 3), np.float32), 8, [0, 0, -10], 0.0, 10.0, 8, 8)
    compare(cg, orc, np.array([[0.5, 0.5, 0.9]], np.float32), 8, [128, 128, 0], 0.0, 10.0, 1, 1)


def test_invalid(cg):
    a = cg.cga_build(dev(np.zeros((1, 3))), cg.grid_from_box([0, 0, 0], 1.0, 8))
    with pytest.raises(cg.CgaError):
        cg.cga_perspective(a, [0, 0, 0], 1.0, 0.0, 0.0, 8, 8)
    with pytest.raises(cg.CgaError):
        cg.cga_perspective(a, [0, 0, 0], float("nan"), 0.0, 1.0, 8, 8)
