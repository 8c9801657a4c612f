"""Seeded synthetic RGB-D-like depth sequences.

This package only *generates inputs*: analytic indoor scenes (a box room plus
spheres and axis-aligned boxes), smooth camera trajectories and ray-cast depth
images with Kinect-like noise. It contains none of the fusion method's
arithmetic (no allocation, no signed-distance update), so the oracle and the
CUDA path can both be fed from it without sharing any of the method.

The paper's own inputs (live OpenNI sensors and the recorded "Teddy"
sequence, Section 6) are not available; these sequences stand in for them with
the image sizes, intrinsics, depth ranges and noise of a Kinect-class sensor.
"""

from .scene import Scene, make_room_scene, raycast_depth
from .trajectory import look_at, circle_poses, smooth_poses
from .configs import (Workload, workload_tiny, workload_kinect, workload_hd,
                      batched_workloads, make_sequence, Sequence)

__all__ = [
    "Scene", "make_room_scene", "raycast_depth", "look_at", "circle_poses",
    "smooth_poses", "Workload", "workload_tiny", "workload_kinect",
    "workload_hd", "batched_workloads", "make_sequence", "Sequence",
]
