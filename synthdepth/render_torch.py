"""The same seeded sequences rendered with torch (any device), for workloads
too large to ray-cast on the host in reasonable time (HD frames, many
scenes, serving sessions).

Scene, trajectory and placement are those of ``make_sequence`` (see
``sequence_geometry``); the ray cast is the same float64 arithmetic written
with torch ops. The noise (Gaussian sigma = 1.5e-3 z^2 plus 2 % zero pixels)
has the same distribution but comes from torch's generator seeded per
(seed, frame), so noisy frames differ from the host renderer's draws. Noise
free frames agree with the host renderer to float64 rounding.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .configs import Workload, sequence_geometry


@dataclass
class DeviceSequence:
    workload: Workload
    depth: "object"          # torch (N, H, W) float32 metres, 0 = invalid
    poses: np.ndarray        # (N, 4, 4) float64 world->camera
    first_frame: int


def raycast_depth_torch(scene, world_to_cam: np.ndarray, rays):
    """z-depth of the first hit for camera rays ``rays`` ((P, 3) float64
    torch, z = 1) under the room->camera pose ``world_to_cam``."""
    import torch
    M = np.asarray(world_to_cam, dtype=np.float64)
    R = M[:3, :3]
    C = -R.T @ M[:3, 3]
    Rt = torch.as_tensor(R, dtype=torch.float64, device=rays.device)
    dirs = rays @ Rt
    n = dirs.shape[0]
    inf = torch.tensor(float("inf"), dtype=torch.float64, device=rays.device)
    best = torch.full((n,), float("inf"), dtype=torch.float64, device=rays.device)
    for ax in range(3):
        d = dirs[:, ax]
        t_hi = (float(scene.room_hi[ax]) - C[ax]) / d
        t_lo = (float(scene.room_lo[ax]) - C[ax]) / d
        t_exit = torch.where(d > 0, t_hi, torch.where(d < 0, t_lo, inf))
        best = torch.minimum(best, t_exit)
    a = (dirs * dirs).sum(1)
    for centre, radius in scene.spheres:
        oc = C - np.asarray(centre)
        b = 2.0 * (dirs @ torch.as_tensor(oc, dtype=torch.float64, device=rays.device))
        c = float(oc @ oc - radius * radius)
        disc = b * b - 4.0 * a * c
        ok = disc >= 0.0
        sq = torch.sqrt(torch.where(ok, disc, torch.zeros_like(disc)))
        t0 = (-b - sq) / (2.0 * a)
        hit = ok & (t0 > 0.0)
        best = torch.where(hit & (t0 < best), t0, best)
    for lo, hi in scene.boxes:
        tmin = torch.full((n,), -float("inf"), dtype=torch.float64, device=rays.device)
        tmax = torch.full((n,), float("inf"), dtype=torch.float64, device=rays.device)
        for ax in range(3):
            d = dirs[:, ax]
            ta = (float(lo[ax]) - C[ax]) / d
            tb = (float(hi[ax]) - C[ax]) / d
            inside = bool(lo[ax] <= C[ax] <= hi[ax])
            t1 = torch.where(d != 0, torch.minimum(ta, tb), -inf if inside else inf)
            t2 = torch.where(d != 0, torch.maximum(ta, tb), inf if inside else -inf)
            tmin = torch.maximum(tmin, t1)
            tmax = torch.minimum(tmax, t2)
        hit = (tmax >= tmin) & (tmin > 0.0)
        best = torch.where(hit & (tmin < best), tmin, best)
    return torch.where(torch.isfinite(best), best, torch.zeros_like(best))


def make_sequence_torch(w: Workload, n_frames: int | None = None,
                        first_frame: int = 0, device="cuda") -> DeviceSequence:
    """Frames [first_frame, first_frame + n_frames) of ``w`` rendered on
    ``device``."""
    import torch
    scene, poses, world_from_room = sequence_geometry(w, n_frames, first_frame)
    n = len(poses)
    u = torch.arange(w.width, dtype=torch.float64, device=device)
    v = torch.arange(w.height, dtype=torch.float64, device=device)
    vv, uu = torch.meshgrid(v, u, indexing="ij")
    rays = torch.stack([(uu - w.cx) / w.fx, (vv - w.cy) / w.fy,
                        torch.ones_like(uu)], -1).reshape(-1, 3)
    out = torch.empty((n, w.height, w.width), dtype=torch.float32, device=device)
    gen = torch.Generator(device=device)
    for i in range(n):
        d = raycast_depth_torch(scene, poses[i], rays)
        if w.noise:
            gen.manual_seed((w.seed * 1_000_003 + 1000 + first_frame + i) % (1 << 62))
            noise = torch.randn(d.shape, dtype=torch.float64, device=device, generator=gen)
            drop = torch.rand(d.shape, dtype=torch.float64, device=device, generator=gen)
            d = d + noise * (1.5e-3 * d * d)
            d = torch.where(drop < 0.02, torch.zeros_like(d), d)
            d = torch.clamp(d, min=0.0)
        out[i] = d.reshape(w.height, w.width).to(torch.float32)
    poses = poses @ np.linalg.inv(world_from_room)
    return DeviceSequence(workload=w, depth=out, poses=poses, first_frame=first_frame)
