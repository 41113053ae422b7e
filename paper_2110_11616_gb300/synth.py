"""Seeded synthetic point clouds, rigid transforms and query sets.

These generators stand in for the paper's datasets (the 8i surface light-field
sequences and the Paris-Lille-3D / GT_Madame LiDAR scans, Sec. VI-B), which are
not used: every input is produced here from a fixed seed.  The module holds no
part of the CGA method itself (no quantization, encoding, sorting or search):
it only draws float32 coordinates and float32 rigid transforms, and both the
CUDA library and the CPU oracle consume its output.

Workload recipes (sizes follow the five benchmark configurations):
  * uniform_cube: n points uniform in a cube (the 100k-point plain case).
  * rigid_xform: axis uniform on the sphere, angle U(0, max_deg), translation
    U(-max_t, max_t)^3; returned as 12 float32 (R row-major, then t).
  * lidar_sweeps: a 64-beam x 2048-step spinning sensor (elevation -25..+3 deg)
    driving ~1 m per frame with yaw changes <= 2 deg; each ray returns the
    nearest hit among a ground plane 1.8 m below the sensor, seeded box
    obstacles and a lognormal background range (median 15 m, capped at 120 m).
    Points are in the sensor frame; the per-sweep pose maps them to the world.
  * superellipsoids: points sampled on the surfaces of seeded superellipsoids
    (exponents U(0.3, 3), semi-axes scale U(1, 10) m, random pose) in a cube.
  * jitter_queries / uniform_queries: NN query sets.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def _rng(seed) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_cube(n: int, seed: int, lo: float = 0.0, extent: float = 1.0) -> np.ndarray:
    r = _rng(seed)
    pts = r.random((n, 3), dtype=np.float64) * extent + lo
    return pts.astype(np.float32)


def _axis_angle(axis, angle) -> np.ndarray:
    x, y, z = axis
    c, s = math.cos(angle), math.sin(angle)
    C = 1.0 - c
    return np.array([
        [c + x * x * C, x * y * C - z * s, x * z * C + y * s],
        [y * x * C + z * s, c + y * y * C, y * z * C - x * s],
        [z * x * C - y * s, z * y * C + x * s, c + z * z * C],
    ])


def rigid_xform(seed: int, max_deg: float = 10.0, max_t: float = 0.05) -> np.ndarray:
    """12 float32: R (3x3 row-major) then t."""
    r = _rng(seed)
    v = r.normal(size=3)
    v /= np.linalg.norm(v)
    ang = math.radians(r.uniform(0.0, max_deg))
    R = _axis_angle(v, ang)
    t = r.uniform(-max_t, max_t, size=3)
    return np.concatenate([R.reshape(9), t]).astype(np.float32)


def pose_xform(yaw: float, tx: float, ty: float, tz: float = 0.0) -> np.ndarray:
    c, s = math.cos(yaw), math.sin(yaw)
    R = np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])
    return np.concatenate([R.reshape(9), [tx, ty, tz]]).astype(np.float32)


def apply_xform64(xform12: np.ndarray, pts: np.ndarray) -> np.ndarray:
    """Float64 R p + t, used only to place query points near world geometry."""
    X = np.asarray(xform12, np.float64)
    R, t = X[:9].reshape(3, 3), X[9:]
    return pts.astype(np.float64) @ R.T + t


@dataclass
class LidarScene:
    sweeps: list  # float32 (beams*steps, 3) per sweep, sensor frame
    poses: list   # float32 xform12 per sweep (sensor -> world)
    box_lo: tuple = (-128.0, -128.0, -128.0)
    extent: float = 256.0
    world: np.ndarray = field(default=None)  # float64 world points, all sweeps


def _ray_box(o, d, lo, hi):
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        t0 = (lo - o) * inv
        t1 = (hi - o) * inv
    tmin = np.nanmax(np.minimum(t0, t1), axis=1)
    tmax = np.nanmin(np.maximum(t0, t1), axis=1)
    hit = (tmax >= np.maximum(tmin, 0.0)) & (tmin > 0.0)
    return np.where(hit, tmin, np.inf)


def lidar_sweeps(n_sweeps: int = 10, beams: int = 64, steps: int = 2048, seed: int = 2,
                 n_boxes: int = 40, with_world: bool = True) -> LidarScene:
    r = _rng(seed)
    elev = np.radians(np.linspace(-25.0, 3.0, beams))
    az = 2.0 * np.pi * np.arange(steps) / steps
    E, A = np.meshgrid(elev, az, indexing="ij")
    d_sensor = np.stack([np.cos(E) * np.cos(A), np.cos(E) * np.sin(A), np.sin(E)],
                        axis=-1).reshape(-1, 3)
    ground_z = -1.8
    cx = r.uniform(-60.0, 60.0, size=n_boxes)
    cy = r.uniform(-60.0, 60.0, size=n_boxes)
    sx = r.uniform(1.0, 6.0, size=n_boxes)
    sy = r.uniform(1.0, 6.0, size=n_boxes)
    sz = r.uniform(1.0, 4.0, size=n_boxes)
    lo_b = np.stack([cx - sx / 2, cy - sy / 2, np.full(n_boxes, ground_z)], axis=1)
    hi_b = np.stack([cx + sx / 2, cy + sy / 2, ground_z + sz], axis=1)
    sweeps, poses, worlds = [], [], []
    yaw, px, py = 0.0, 0.0, 0.0
    for _ in range(n_sweeps):
        pose = pose_xform(yaw, px, py, 0.0)
        P = np.asarray(pose, np.float64)
        R = P[:9].reshape(3, 3)
        o = P[9:]
        d_world = d_sensor @ R.T
        rng_bg = np.minimum(r.lognormal(mean=math.log(15.0), sigma=0.6, size=len(d_sensor)),
                            120.0)
        t_hit = rng_bg
        with np.errstate(divide="ignore", invalid="ignore"):
            t_ground = np.where(d_world[:, 2] < 0, (ground_z - o[2]) / d_world[:, 2], np.inf)
        t_hit = np.minimum(t_hit, t_ground)
        O = np.broadcast_to(o, d_world.shape)
        for b in range(n_boxes):
            t_hit = np.minimum(t_hit, _ray_box(O, d_world, lo_b[b], hi_b[b]))
        t_hit = np.minimum(t_hit, 120.0)
        pts_s = d_sensor * t_hit[:, None]
        sweeps.append(pts_s.astype(np.float32))
        poses.append(pose)
        if with_world:
            worlds.append(apply_xform64(pose, pts_s.astype(np.float32)))
        step = r.uniform(0.8, 1.2)
        px += step * math.cos(yaw)
        py += step * math.sin(yaw)
        yaw += math.radians(r.uniform(-2.0, 2.0))
    scene = LidarScene(sweeps=sweeps, poses=poses)
    if with_world:
        scene.world = np.concatenate(worlds, axis=0)
    return scene


def _random_rotation(r: np.random.Generator) -> np.ndarray:
    q = r.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def _spow(v, e):
    return np.sign(v) * np.abs(v) ** e


@dataclass
class SurfaceScene:
    objects: list  # (e1, e2, axes[3], R[3x3], center[3])
    box_lo: tuple
    extent: float


def superellipsoid_scene(n_objects: int = 200, seed: int = 3, lo: float = 0.0,
                         extent: float = 100.0) -> SurfaceScene:
    r = _rng(seed)
    objs = []
    for _ in range(n_objects):
        e1, e2 = r.uniform(0.3, 3.0, size=2)
        s = r.uniform(1.0, 10.0)
        axes = s * r.uniform(0.5, 1.0, size=3)
        R = _random_rotation(r)
        c = r.uniform(lo + 0.1 * extent, lo + 0.9 * extent, size=3)
        objs.append((e1, e2, axes, R, c))
    return SurfaceScene(objs, (lo, lo, lo), extent)


def sample_surfaces(scene: SurfaceScene, n: int, seed: int) -> np.ndarray:
    """n float32 points on the scene's surfaces, object share ~ its axes^2."""
    r = _rng(seed)
    w = np.array([float(np.mean(o[2]) ** 2) for o in scene.objects])
    counts = r.multinomial(n, w / w.sum())
    out = np.empty((n, 3), np.float32)
    pos = 0
    for (e1, e2, axes, R, c), k in zip(scene.objects, counts):
        if k == 0:
            continue
        eta = r.uniform(-np.pi / 2, np.pi / 2, size=k)
        om = r.uniform(-np.pi, np.pi, size=k)
        ce, se = _spow(np.cos(eta), e1), _spow(np.sin(eta), e1)
        co, so = _spow(np.cos(om), e2), _spow(np.sin(om), e2)
        local = np.stack([axes[0] * ce * co, axes[1] * ce * so, axes[2] * se], axis=1)
        out[pos:pos + k] = (local @ R.T + c).astype(np.float32)
        pos += k
    perm = r.permutation(n)
    return out[perm]


def jitter_queries(world: np.ndarray, m: int, sigma: float, seed: int) -> np.ndarray:
    r = _rng(seed)
    pick = r.integers(0, len(world), size=m)
    return (world[pick] + r.normal(0.0, sigma, size=(m, 3))).astype(np.float32)


def uniform_queries(m: int, seed: int, lo, extent: float) -> np.ndarray:
    r = _rng(seed)
    return (r.random((m, 3)) * extent + np.asarray(lo, np.float64)).astype(np.float32)


def log_uniform_ints(k: int, lo: float, hi: float, seed: int) -> np.ndarray:
    r = _rng(seed)
    return np.exp(r.uniform(math.log(lo), math.log(hi), size=k)).astype(np.int64)
