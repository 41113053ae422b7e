"""Seeded synthetic point clouds generated on the GPU with torch (for the
batched and served workloads, whose 1.7e8-2.4e8 points would take minutes to
draw on the host).  Same recipes as synth.py, scaled to any point count; no
part of the CGA method lives here (only float32 coordinates are drawn).

  lidar_cloud: one spinning-sensor sweep of n returns (64 beams, n/64 azimuth
    steps, elevation -25..+3 deg) placed at a random pose within +-40 m; each
    ray hits the nearest of a ground plane 1.8 m below the sensor, 8 seeded
    boxes, or a lognormal background range (median 15 m) capped at 120 m.
  surface_cloud: n points on 200 superellipsoids (exponents U(0.3, 3),
    semi-axes scale U(1, 10) m, random rotation) in a 100 m cube.
"""
from __future__ import annotations

import math

import torch


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def lidar_cloud(n: int, seed: int, device="cuda") -> torch.Tensor:
    g = _gen(seed, device)
    beams = 64
    steps = max(1, -(-n // beams))
    f64 = dict(dtype=torch.float64, device=device)
    elev = torch.deg2rad(torch.linspace(-25.0, 3.0, beams, **f64))
    az = 2 * math.pi * torch.arange(steps, **f64) / steps
    E, A = torch.meshgrid(elev, az, indexing="ij")
    d = torch.stack([E.cos() * A.cos(), E.cos() * A.sin(), E.sin()], -1).reshape(-1, 3)[:n]
    yaw = float(torch.rand(1, generator=g, **f64).item() * 2 * math.pi)
    ox, oy = (torch.rand(2, generator=g, **f64) * 80 - 40).tolist()
    c, s = math.cos(yaw), math.sin(yaw)
    R = torch.tensor([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]], **f64)
    dw = d @ R.T
    o = torch.tensor([ox, oy, 0.0], **f64)
    t = torch.exp(math.log(15.0) + 0.6 * torch.randn(len(dw), generator=g, **f64)).clamp(max=120.0)
    ground = torch.where(dw[:, 2] < 0, (-1.8 - o[2]) / dw[:, 2], torch.full_like(t, float("inf")))
    t = torch.minimum(t, ground)
    nb = 8
    ctr = torch.rand(nb, 2, generator=g, **f64) * 120 - 60 + o[:2]
    size = torch.rand(nb, 3, generator=g, **f64) * torch.tensor([5.0, 5.0, 3.0], **f64) + 1.0
    lo = torch.cat([ctr - size[:, :2] / 2, torch.full((nb, 1), -1.8, **f64)], 1)
    hi = torch.cat([ctr + size[:, :2] / 2, -1.8 + size[:, 2:]], 1)
    inv = 1.0 / dw
    for b in range(nb):
        t0 = (lo[b] - o) * inv
        t1 = (hi[b] - o) * inv
        tmin = torch.minimum(t0, t1).nan_to_num(nan=-float("inf")).amax(1)
        tmax = torch.maximum(t0, t1).nan_to_num(nan=float("inf")).amin(1)
        hit = (tmax >= tmin.clamp(min=0)) & (tmin > 0)
        t = torch.where(hit, torch.minimum(t, tmin), t)
    return (o + dw * t[:, None]).to(torch.float32).contiguous()


def surface_scene(seed: int, n_objects: int = 200, lo: float = 0.0, extent: float = 100.0,
                  device="cuda") -> dict:
    """Parameters of n_objects seeded superellipsoids inside [lo, lo + extent)^3."""
    g = _gen(seed, device)
    f64 = dict(dtype=torch.float64, device=device)
    e = torch.rand(n_objects, 2, generator=g, **f64) * 2.7 + 0.3
    scale = torch.rand(n_objects, 1, generator=g, **f64) * 9 + 1
    axes = scale * (torch.rand(n_objects, 3, generator=g, **f64) * 0.5 + 0.5)
    q = torch.randn(n_objects, 4, generator=g, **f64)
    q = q / q.norm(dim=1, keepdim=True)
    w, x, y, z = q.unbind(1)
    R = torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], 1),
        torch.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], 1),
        torch.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], 1),
    ], 1)
    ctr = torch.rand(n_objects, 3, generator=g, **f64) * (0.8 * extent) + lo + 0.1 * extent
    return {"e": e, "axes": axes, "R": R, "ctr": ctr}


def sample_scene(scene: dict, n: int, seed: int) -> torch.Tensor:
    """n float32 points on the scene's surfaces (object share ~ mean axis^2)."""
    e, axes, R, ctr = scene["e"], scene["axes"], scene["R"], scene["ctr"]
    device = e.device
    g = _gen(seed, device)
    f64 = dict(dtype=torch.float64, device=device)
    wgt = axes.mean(1) ** 2
    obj = torch.multinomial((wgt / wgt.sum()).float(), n, replacement=True, generator=g)
    eta = (torch.rand(n, generator=g, **f64) - 0.5) * math.pi
    om = (torch.rand(n, generator=g, **f64) * 2 - 1) * math.pi

    def spow(v, p):
        return torch.sign(v) * v.abs() ** p

    e1, e2 = e[obj, 0], e[obj, 1]
    ce, se = spow(eta.cos(), e1), spow(eta.sin(), e1)
    co, so = spow(om.cos(), e2), spow(om.sin(), e2)
    ax = axes[obj]
    local = torch.stack([ax[:, 0] * ce * co, ax[:, 1] * ce * so, ax[:, 2] * se], 1)
    pts = torch.einsum("nij,nj->ni", R[obj], local) + ctr[obj]
    return pts.to(torch.float32).contiguous()


def surface_cloud(n: int, seed: int, n_objects: int = 200, lo: float = 0.0, extent: float = 100.0,
                  device="cuda") -> torch.Tensor:
    """n points of the scene drawn from `seed` (sampled with seed + 1)."""
    return sample_scene(surface_scene(seed, n_objects, lo, extent, device), n, seed + 1)


def jitter_queries(points: torch.Tensor, m: int, sigma: float, seed: int) -> torch.Tensor:
    g = _gen(seed, points.device)
    pick = torch.randint(0, len(points), (m,), generator=g, device=points.device)
    noise = torch.randn(m, 3, generator=g, device=points.device, dtype=torch.float64) * sigma
    return (points[pick].double() + noise).to(torch.float32).contiguous()


def uniform_queries(m: int, seed: int, lo, extent: float, device="cuda") -> torch.Tensor:
    g = _gen(seed, device)
    u = torch.rand(m, 3, generator=g, device=device, dtype=torch.float64)
    return (u * extent + torch.tensor(lo, dtype=torch.float64, device=device)).to(
        torch.float32).contiguous()
