"""Analytic scenes and exact ray casting of z-depth images (float64).

A scene is the inside of an axis-aligned box room plus a few spheres and
axis-aligned boxes. ``raycast_depth`` returns, per pixel centre, the camera-z
coordinate of the first surface hit along the pixel's ray: the quantity a
structured-light depth sensor reports.

Conventions: world frame in metres, y up. Camera frame x right, y down,
z forward; the pose is the 4x4 world->camera matrix.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Scene:
    room_lo: np.ndarray                      # (3,) inner corner of the room
    room_hi: np.ndarray                      # (3,)
    spheres: list = field(default_factory=list)   # [(centre(3,), radius)]
    boxes: list = field(default_factory=list)     # [(lo(3,), hi(3,))]


def make_room_scene(rng: np.random.Generator, n_objects: int,
                    size: tuple = (4.0, 3.0, 3.0),
                    fixed_objects: bool = False,
                    keep_out_radius: float = 0.85) -> Scene:
    """A room of ``size`` metres centred at the origin with seeded objects.

    ``fixed_objects``: one sphere of 0.5 m diameter and one cube of 0.4 m edge
    (the tiny workload); otherwise ``n_objects`` random spheres / boxes of
    0.2-0.6 m extent. All objects stay inside ``keep_out_radius`` of the room
    centre in the horizontal plane, so a camera circling at 1 m never enters
    one.
    """
    half = np.asarray(size, dtype=np.float64) / 2.0
    scene = Scene(room_lo=-half, room_hi=half.copy())

    def place(extent_half):
        # horizontal position with reach inside keep_out_radius
        reach = keep_out_radius - extent_half
        ang = rng.uniform(0.0, 2.0 * np.pi)
        rad = rng.uniform(0.0, max(reach - 0.05, 0.0))
        y = rng.uniform(-half[1] + extent_half, half[1] - extent_half)
        return np.array([rad * np.cos(ang), y, rad * np.sin(ang)])

    if fixed_objects:
        r = 0.25
        c = place(r)
        scene.spheres.append((c, r))
        e = 0.2
        c = place(e * np.sqrt(2.0))
        scene.boxes.append((c - e, c + e))
        return scene
    for _ in range(n_objects):
        if rng.uniform() < 0.5:
            r = rng.uniform(0.1, 0.3)
            scene.spheres.append((place(r), r))
        else:
            e = rng.uniform(0.1, 0.3, size=3)
            c = place(float(np.hypot(e[0], e[2])))
            scene.boxes.append((c - e, c + e))
    return scene


def _pixel_rays(width: int, height: int, fx: float, fy: float, cx: float,
                cy: float) -> np.ndarray:
    """Camera-frame rays with z = 1 through every pixel centre, (H, W, 3)."""
    u = np.arange(width, dtype=np.float64)
    v = np.arange(height, dtype=np.float64)
    uu, vv = np.meshgrid(u, v)
    return np.stack([(uu - cx) / fx, (vv - cy) / fy, np.ones_like(uu)], axis=-1)


def raycast_depth(scene: Scene, world_to_cam: np.ndarray, width: int,
                  height: int, fx: float, fy: float, cx: float,
                  cy: float) -> np.ndarray:
    """Exact z-depth (float64, metres) of the first hit for every pixel.

    Rays are parametrised by camera z: p(t) = C + t * R^T r with r_z = 1, so
    the hit parameter t is directly the depth value. Pixels with no hit
    (impossible inside a closed room) get 0.
    """
    M = np.asarray(world_to_cam, dtype=np.float64)
    R = M[:3, :3]
    t = M[:3, 3]
    C = -R.T @ t                                   # camera centre in world
    rays = _pixel_rays(width, height, fx, fy, cx, cy).reshape(-1, 3)
    dirs = rays @ R                                # R^T r for every row r
    n = dirs.shape[0]
    best = np.full(n, np.inf)

    # room: the camera is inside, the hit is the exit point
    with np.errstate(divide="ignore", invalid="ignore"):
        for ax in range(3):
            d = dirs[:, ax]
            t_hi = (scene.room_hi[ax] - C[ax]) / d
            t_lo = (scene.room_lo[ax] - C[ax]) / d
            t_exit = np.where(d > 0, t_hi, np.where(d < 0, t_lo, np.inf))
            best = np.minimum(best, t_exit)

    for centre, radius in scene.spheres:
        oc = C - np.asarray(centre)
        a = np.einsum("ij,ij->i", dirs, dirs)
        b = 2.0 * (dirs @ oc)
        c = oc @ oc - radius * radius
        disc = b * b - 4.0 * a * c
        ok = disc >= 0.0
        sq = np.sqrt(np.where(ok, disc, 0.0))
        t0 = (-b - sq) / (2.0 * a)
        hit = ok & (t0 > 0.0)
        best = np.where(hit & (t0 < best), t0, best)

    for lo, hi in scene.boxes:
        lo = np.asarray(lo)
        hi = np.asarray(hi)
        tmin = np.full(n, -np.inf)
        tmax = np.full(n, np.inf)
        with np.errstate(divide="ignore", invalid="ignore"):
            for ax in range(3):
                d = dirs[:, ax]
                ta = (lo[ax] - C[ax]) / d
                tb = (hi[ax] - C[ax]) / d
                inside = (C[ax] >= lo[ax]) & (C[ax] <= hi[ax])
                t1 = np.where(d != 0, np.minimum(ta, tb),
                              np.where(inside, -np.inf, np.inf))
                t2 = np.where(d != 0, np.maximum(ta, tb),
                              np.where(inside, np.inf, -np.inf))
                tmin = np.maximum(tmin, t1)
                tmax = np.minimum(tmax, t2)
        hit = (tmax >= tmin) & (tmin > 0.0)
        best = np.where(hit & (tmin < best), tmin, best)

    best = np.where(np.isfinite(best), best, 0.0)
    return best.reshape(height, width)


# Surface colour: a smooth texture of the room-frame position, three
# channels of different spatial frequency and phase (values 28..228).
_TEX_FREQ = np.array([[1.3, 0.4, 0.0], [0.0, 0.7, -1.1], [0.5, 0.0, 0.9]])
_TEX_PHASE = np.array([0.3, 1.7, 2.9])


def surface_colour(points: np.ndarray) -> np.ndarray:
    """Texture value (float64, 0..255 scale) of room-frame points (..., 3)."""
    arg = 2.0 * np.pi * (points @ _TEX_FREQ.T) + _TEX_PHASE
    return 128.0 + 100.0 * np.sin(arg)


def raycast_colour(depth: np.ndarray, world_to_cam: np.ndarray, width: int, height: int,
                   fx: float, fy: float, cx: float, cy: float) -> np.ndarray:
    """Texture value (float64 (H, W, 3)) of the surface point seen by every
    pixel, from the noise-free z-depth of raycast_depth (same conventions)."""
    M = np.asarray(world_to_cam, dtype=np.float64)
    R = M[:3, :3]
    C = -R.T @ M[:3, 3]
    rays = _pixel_rays(width, height, fx, fy, cx, cy).reshape(-1, 3)
    pts = C + depth.reshape(-1, 1) * (rays @ R)
    return surface_colour(pts).reshape(height, width, 3)
