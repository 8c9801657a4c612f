"""Camera trajectories: world->camera 4x4 poses (float64)."""

from __future__ import annotations

import numpy as np


def look_at(centre: np.ndarray, target: np.ndarray,
            up: np.ndarray = np.array([0.0, 1.0, 0.0])) -> np.ndarray:
    """World->camera pose of a camera at ``centre`` looking at ``target``.

    Camera axes: z forward (towards the target), y down (opposite the world up
    vector), x = y cross z (right), so the frame is right-handed.
    """
    centre = np.asarray(centre, dtype=np.float64)
    z = np.asarray(target, dtype=np.float64) - centre
    z /= np.linalg.norm(z)
    x = np.cross(-np.asarray(up, dtype=np.float64), z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z])
    M = np.eye(4)
    M[:3, :3] = R
    M[:3, 3] = -R @ centre
    return M


def circle_poses(n_frames: int, radius: float = 1.0, height: float = 0.0,
                 phase: float = 0.0) -> np.ndarray:
    """``n_frames`` poses evenly spaced on a horizontal circle, each looking at
    the room centre (the tiny workload's known poses)."""
    poses = []
    for k in range(n_frames):
        a = phase + 2.0 * np.pi * k / n_frames
        c = np.array([radius * np.cos(a), height, radius * np.sin(a)])
        poses.append(look_at(c, np.zeros(3)))
    return np.stack(poses)


def smooth_poses(rng: np.random.Generator, n_frames: int, radius: float = 1.0,
                 step_range=(0.01, 0.03)) -> np.ndarray:
    """A seeded smooth trajectory around the room centre.

    Each frame the camera advances by an arc of ``step_range`` metres (seeded
    uniform) along a circle of ``radius``, with slow sinusoidal height and
    look-at-target wobbles. The resulting motion is 1-3 cm and roughly
    0.5-2 degrees per frame.
    """
    arcs = rng.uniform(step_range[0], step_range[1], size=n_frames)
    theta = rng.uniform(0.0, 2.0 * np.pi) + np.concatenate([[0.0], np.cumsum(arcs[:-1])]) / radius
    ph = rng.uniform(0.0, 2.0 * np.pi, size=4)
    k = np.arange(n_frames, dtype=np.float64)
    height = 0.12 * np.sin(2.0 * np.pi * k / 173.0 + ph[0])
    tx = 0.10 * np.sin(2.0 * np.pi * k / 131.0 + ph[1])
    ty = 0.08 * np.sin(2.0 * np.pi * k / 97.0 + ph[2])
    tz = 0.10 * np.sin(2.0 * np.pi * k / 151.0 + ph[3])
    poses = []
    for i in range(n_frames):
        c = np.array([radius * np.cos(theta[i]), height[i], radius * np.sin(theta[i])])
        poses.append(look_at(c, np.array([tx[i], ty[i], tz[i]])))
    return np.stack(poses)
