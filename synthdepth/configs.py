"""Workload recipes and sequence generation.

Each workload fixes an image size, pinhole intrinsics, a scene recipe, a
trajectory, a depth-noise model and the fusion parameters (voxel size,
truncation band, hash / pool sizes, storage form). ``make_sequence`` renders
its depth frames deterministically from the seed.

Noise model (Kinect-class sensor): additive Gaussian with standard deviation
1.5e-3 * z^2 metres, then a seeded 2 % of pixels set to 0 (invalid).
"""

from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np

from .scene import raycast_colour, make_room_scene, raycast_depth
from .trajectory import circle_poses, smooth_poses

STORAGE_F32, STORAGE_I16, STORAGE_F16 = 0, 1, 2


@dataclass(frozen=True)
class Workload:
    name: str
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    n_frames: int
    seed: int
    n_objects: int            # 0 with fixed_objects -> sphere + cube
    fixed_objects: bool
    circle: bool              # poses on a 1 m circle (else smooth seeded path)
    noise: bool               # Gaussian z^2 noise + 2 % zero pixels
    voxel_size: float
    mu: float
    max_weight: int
    hash_buckets_log2: int
    entries_per_bucket: int
    excess_entries: int
    pool_blocks: int
    storage: int

    def scene_desc(self) -> dict:
        return dict(voxel_size=self.voxel_size, mu=self.mu,
                    max_weight=self.max_weight,
                    hash_buckets_log2=self.hash_buckets_log2,
                    entries_per_bucket=self.entries_per_bucket,
                    excess_entries=self.excess_entries,
                    pool_blocks=self.pool_blocks, storage=self.storage)

    def intrinsics(self) -> tuple:
        return (self.fx, self.fy, self.cx, self.cy, self.width, self.height)


def workload_tiny(**kw) -> Workload:
    """160x120, 20 noise-free frames on a 1 m circle; room + sphere + cube;
    2 cm voxels, mu 8 cm, hash 2^14 + 2^12 excess, pool 2^14, max weight 100."""
    w = Workload(name="tiny_160x120_2cm", width=160, height=120, fx=131.25,
                 fy=131.25, cx=79.5, cy=59.5, n_frames=20, seed=1410_0925_1,
                 n_objects=0, fixed_objects=True, circle=True, noise=False,
                 voxel_size=0.02, mu=0.08, max_weight=100,
                 hash_buckets_log2=14, entries_per_bucket=2,
                 excess_entries=1 << 12, pool_blocks=1 << 14,
                 storage=STORAGE_F32)
    return replace(w, **kw)


def workload_kinect(**kw) -> Workload:
    """640x480, 300 noisy frames on a seeded smooth path; room + 6 objects;
    5 mm voxels, mu 2 cm, hash 2^20 + 2^17 excess, pool 2^18, float32 sdf."""
    w = Workload(name="kinect_640x480_5mm", width=640, height=480, fx=525.0,
                 fy=525.0, cx=319.5, cy=239.5, n_frames=300,
                 seed=1410_0925_2, n_objects=6, fixed_objects=False,
                 circle=False, noise=True, voxel_size=0.005, mu=0.02,
                 max_weight=100, hash_buckets_log2=20, entries_per_bucket=2,
                 excess_entries=1 << 17, pool_blocks=1 << 18,
                 storage=STORAGE_F32)
    return replace(w, **kw)


def workload_hd(storage: int = STORAGE_I16, **kw) -> Workload:
    """1280x720 (f=1050), 500 noisy frames, same room family; 4 mm voxels,
    mu 1.6 cm, pool 2^21 blocks, hash 2^21 + 2^18 excess; int16 or FP16 sdf."""
    w = Workload(name="hd_1280x720_4mm", width=1280, height=720, fx=1050.0,
                 fy=1050.0, cx=639.5, cy=359.5, n_frames=500,
                 seed=1410_0925_3, n_objects=6, fixed_objects=False,
                 circle=False, noise=True, voxel_size=0.004, mu=0.016,
                 max_weight=100, hash_buckets_log2=21, entries_per_bucket=2,
                 excess_entries=1 << 18, pool_blocks=1 << 21,
                 storage=storage)
    return replace(w, **kw)


_BATCH_IMAGES = [(160, 120, 131.25), (320, 240, 262.5), (640, 480, 525.0)]
_BATCH_VOXELS = [0.004, 0.005, 0.010]
_BATCH_POOL_LOG2 = {0.004: 18, 0.005: 16, 0.010: 14}


def batched_workloads(n_scenes: int = 64, n_frames: int = 100,
                      seed: int = 1410_0925_4,
                      storage: int = STORAGE_I16) -> list:
    """Independent scenes of uneven image and voxel sizes: images uniform over
    {160x120, 320x240, 640x480}, voxels over {4, 5, 10} mm with mu = 4 voxels,
    pools 2^14..2^18 blocks (by voxel size), noise as the Kinect workload."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_scenes):
        W, H, f = _BATCH_IMAGES[int(rng.integers(0, 3))]
        s = _BATCH_VOXELS[int(rng.integers(0, 3))]
        pl = _BATCH_POOL_LOG2[s]
        out.append(Workload(
            name=f"batch{i}_{W}x{H}_{int(round(s * 1000))}mm", width=W,
            height=H, fx=f, fy=f, cx=W / 2 - 0.5, cy=H / 2 - 0.5,
            n_frames=n_frames, seed=seed * 100 + i, n_objects=6,
            fixed_objects=False, circle=False, noise=True, voxel_size=s,
            mu=4 * s, max_weight=100, hash_buckets_log2=pl + 2,
            entries_per_bucket=2, excess_entries=1 << (pl - 1),
            pool_blocks=1 << pl, storage=storage))
    return out


@dataclass
class Sequence:
    workload: Workload
    depth: np.ndarray        # (N, H, W) float32 metres, 0 = invalid
    poses: np.ndarray        # (N, 4, 4) float64 world->camera
    first_frame: int
    colour: np.ndarray | None = None  # (N, H, W, 4) uint8 RGBX registered to depth


def sequence_geometry(w: Workload, n_frames: int | None = None,
                      first_frame: int = 0):
    """The seeded scene and camera poses of frames [first_frame, first_frame +
    n) of ``w``: (scene in room coordinates, (n, 4, 4) room->camera poses,
    4x4 room->world placement). Depends only on ``w.seed``."""
    n = w.n_frames if n_frames is None else n_frames
    rng = np.random.default_rng(w.seed)
    scene = make_room_scene(rng, w.n_objects, fixed_objects=w.fixed_objects)
    total = max(w.n_frames, first_frame + n)
    if w.circle:
        poses = circle_poses(total)
    else:
        poses = smooth_poses(np.random.default_rng([w.seed, 7]), total)
    poses = poses[first_frame:first_frame + n]
    # The room is placed in the world with a seeded rigid transform (a yaw and
    # an offset), so that its walls are not aligned with the voxel lattice.
    world_from_room = room_placement(np.random.default_rng([w.seed, 11]))
    return scene, poses, world_from_room


def make_sequence(w: Workload, n_frames: int | None = None,
                  first_frame: int = 0, colour: bool = False) -> Sequence:
    """Render frames [first_frame, first_frame + n_frames) of workload ``w``.

    The scene and the whole trajectory depend only on ``w.seed``; the noise of
    frame k depends only on (seed, k), so any sub-range is reproducible.
    ``colour``: also render an RGBX colour image registered to each depth
    image (same camera): the surface texture at the pixel's noise-free hit
    point plus N(0, 2^2) sensor noise per channel (seeded by (seed, k)),
    rounded and clipped to 0..255; X = 255.
    """
    scene, poses, world_from_room = sequence_geometry(w, n_frames, first_frame)
    n = len(poses)
    frames = np.empty((n, w.height, w.width), dtype=np.float32)
    rgb = np.empty((n, w.height, w.width, 4), dtype=np.uint8) if colour else None
    for i in range(n):
        d = raycast_depth(scene, poses[i], w.width, w.height, w.fx, w.fy,
                          w.cx, w.cy)
        if colour:
            c = raycast_colour(d, poses[i], w.width, w.height, w.fx, w.fy, w.cx, w.cy)
            crng = np.random.default_rng([w.seed, 5000 + first_frame + i])
            c = c + 2.0 * crng.standard_normal(c.shape)
            rgb[i, ..., :3] = np.clip(np.rint(c), 0, 255).astype(np.uint8)
            rgb[i, ..., 3] = 255
        if w.noise:
            nrng = np.random.default_rng([w.seed, 1000 + first_frame + i])
            d = d + nrng.standard_normal(d.shape) * (1.5e-3 * d * d)
            d = np.where(nrng.uniform(size=d.shape) < 0.02, 0.0, d)
            d = np.maximum(d, 0.0)
        frames[i] = d.astype(np.float32)
    poses = poses @ np.linalg.inv(world_from_room)
    return Sequence(workload=w, depth=frames, poses=poses,
                    first_frame=first_frame, colour=rgb)


def room_placement(rng: np.random.Generator) -> np.ndarray:
    """Seeded 4x4 room->world transform: yaw about the up axis in
    [0, 90) degrees and an offset uniform in [-0.5, 0.5)^3 metres."""
    yaw = rng.uniform(0.0, 0.5 * np.pi)
    c, s = np.cos(yaw), np.sin(yaw)
    T = np.eye(4)
    T[:3, :3] = np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])
    T[:3, 3] = rng.uniform(-0.5, 0.5, size=3)
    return T


_SERVE_IMAGES = [(320, 240, 262.5), (640, 480, 525.0), (1280, 720, 1050.0)]
_SERVE_VOXELS = [0.004, 0.005, 0.006, 0.008, 0.010]
_SERVE_POOL_LOG2 = {0.004: 19, 0.005: 18, 0.006: 18, 0.008: 17, 0.010: 16}


def serving_sessions(rate_per_s: float = 200.0, duration_s: float = 2.0,
                     seed: int = 1410_0925_5, frames=(50, 400), bank: int = 2,
                     storage: int = STORAGE_I16) -> list:
    """Poisson session arrivals: [(arrival_s, Workload)] over ``duration_s``.
    Each session: image uniform over {320x240, 640x480, 1280x720}, voxel
    uniform over {4, 5, 6, 8, 10} mm (mu = 4 voxels, pool by voxel size),
    frame count uniform in ``frames``, and one of ``bank`` seeded sequences
    per image size (sessions of the same image size and bank index share a
    depth sequence; their voxel sizes differ)."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_per_s)
        if t >= duration_s:
            return out
        ii = int(rng.integers(0, len(_SERVE_IMAGES)))
        W, H, f = _SERVE_IMAGES[ii]
        s = _SERVE_VOXELS[int(rng.integers(0, len(_SERVE_VOXELS)))]
        n = int(rng.integers(frames[0], frames[1] + 1))
        b = int(rng.integers(0, bank))
        pl = _SERVE_POOL_LOG2[s]
        out.append((t, Workload(
            name=f"serve_{W}x{H}_{int(round(s * 1000))}mm_b{b}", width=W, height=H,
            fx=f, fy=f, cx=W / 2 - 0.5, cy=H / 2 - 0.5, n_frames=n,
            seed=seed * 10 + 1000 * ii + b, n_objects=6, fixed_objects=False,
            circle=False, noise=True, voxel_size=s, mu=4 * s, max_weight=100,
            hash_buckets_log2=pl + 1, entries_per_bucket=2,
            excess_entries=1 << (pl - 1), pool_blocks=1 << pl, storage=storage)))
