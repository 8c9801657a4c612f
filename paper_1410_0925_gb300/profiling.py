"""Small, deterministic cases of the measured workloads for ncu captures.

Each driver runs the first N frames of the Kinect-sized sequence (640x480,
5 mm) through one part of the library, eagerly and with a synchronisation
after each call where the counts are read, and prints the counts of every
launch it makes, so that a captured launch can be scaled to the benchmark's
average launch. They time nothing. Usage:

    python -m paper_1410_0925_gb300.profiling --workload kinect --frames 45
    (workloads: kinect, hd, colour, icp, swap, raycast)
"""

from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)

from synthdepth.cache import load_sequence  # noqa: E402

from .workloads import SWAP_CAPACITY, SWAP_MARGIN_PX, Z_NEAR, swap_step_ops  # noqa: E402


def profile_icp(args):
    """Small, deterministic case for ncu: frames 0..N-1 of the Kinect
    sequence fused eagerly, the maps of frame N-1's pose, then three
    reductions of frame N against them; prints the inlier count."""
    import torch
    from paper_1410_0925_gb300 import Icp, Scene, make_intrinsics
    from synthdepth import workload_kinect
    torch.cuda.set_device(0)
    w = workload_kinect()
    seq = load_sequence(w, args.frames + 1)
    n = args.frames
    intr = make_intrinsics(w.fx, w.fy, w.cx, w.cy, w.width, w.height)
    depth = torch.from_numpy(seq.depth[:n + 1]).cuda()
    scene = Scene.from_workload(w)
    scene.integrate_frames(depth[:n], intr, seq.poses[:n])
    icp = Icp()
    V = scene.raycast(intr, seq.poses[n - 1], Z_NEAR)
    N = icp.normals(V)
    out = []
    for _ in range(3):
        s = icp.reduce(depth[n], intr, seq.poses[n - 1], seq.poses[n - 1], V, N, 0.1)
        out.append(float(s[28].item()))
    print(json.dumps({"profile_icp_inliers": out}))


def profile_colour(args):
    """Small, deterministic case for ncu: frames 0..N-1 of the Kinect
    sequence with colour, fused eagerly through tsdf_integrate_rgb; prints
    per-frame counts so a captured launch can be scaled."""
    import torch
    from paper_1410_0925_gb300 import Scene, make_intrinsics
    from synthdepth import workload_kinect
    torch.cuda.set_device(0)
    w = workload_kinect()
    seq = load_sequence(w, args.frames + 1, colour=True)
    intr = make_intrinsics(w.fx, w.fy, w.cx, w.cy, w.width, w.height)
    depth = torch.from_numpy(seq.depth[:args.frames]).cuda()
    col = torch.from_numpy(seq.colour[:args.frames]).cuda()
    scene = Scene.from_workload(w)
    scene.enable_colour()
    per = []
    for i in range(args.frames):
        scene.integrate_rgb(depth[i], col[i], intr, seq.poses[i])
        st = scene.stats()
        per.append({"frame": i, "updated": st["last_updated_voxels"],
                    "visible": st["last_visible_blocks"]})
    print(json.dumps({"profile_frames": per}))


def profile_swap(args):
    """Small, deterministic case for ncu: frames 0..N-1 of the Kinect
    sequence fused with the swap schedule of the swapping workload, then
    three swap-out / swap-in pairs that move blocks both ways (out from a view
    that sees nothing, back from the frames' poses); prints the blocks each
    call moved so a captured launch can be scaled."""
    import torch
    from paper_1410_0925_gb300 import Scene, make_intrinsics
    from synthdepth import workload_kinect
    torch.cuda.set_device(0)
    w = workload_kinect()
    seq = load_sequence(w, args.frames + 1)
    intr = make_intrinsics(w.fx, w.fy, w.cx, w.cy, w.width, w.height)
    n = args.frames
    depth = torch.from_numpy(seq.depth[:n]).cuda()
    scene = Scene.from_workload(w)
    scene.enable_swapping(SWAP_CAPACITY)
    swap_step_ops(scene, depth, intr, seq.poses[:n])
    away = np.array([[-1.0, 0, 0, 0], [0, 1.0, 0, 0], [0, 0, -1.0, -100.0], [0, 0, 0, 1.0]])
    moved = []
    for _ in range(3):
        scene.swap_out(intr, away)
        out_n = scene.swap_stats()["last_out"]
        back = 0
        for i in range(n):
            scene.swap_in(intr, seq.poses[i], SWAP_MARGIN_PX)
            back += scene.swap_stats()["last_in"]
        moved.append({"out": out_n, "in": back})
    print(json.dumps({"profile_swaps": moved, "device_blocks": scene.stats()["allocated_blocks"]}))


def profile_raycast(args):
    """Small, deterministic case for ncu: frames 0..N-1 of the Kinect
    sequence fused eagerly, then three raycasts from the last pose; prints
    each raycast's sample count so a captured launch can be scaled."""
    import torch
    from paper_1410_0925_gb300 import Scene, make_intrinsics
    from synthdepth import workload_kinect
    torch.cuda.set_device(0)
    w = workload_kinect()
    seq = load_sequence(w, args.frames + 1)
    intr = make_intrinsics(w.fx, w.fy, w.cx, w.cy, w.width, w.height)
    depth = torch.from_numpy(seq.depth[:args.frames]).cuda()
    scene = Scene.from_workload(w)
    scene.integrate_frames(depth, intr, seq.poses[:args.frames])
    out = []
    for _ in range(3):
        scene.raycast(intr, seq.poses[args.frames - 1], Z_NEAR)
        out.append(scene.raycast_stats())
    print(json.dumps({"profile_raycasts": out, "allocated": scene.stats()["allocated_blocks"]}))


def profile_fusion(args):
    """Small, deterministic case for ncu: frames 0..N-1 of the Kinect
    sequence, launched eagerly; prints per-frame updated voxels and visible
    blocks so a capture of launch k can be scaled by its own counts."""
    import torch
    from paper_1410_0925_gb300 import Scene, make_intrinsics
    from synthdepth import workload_kinect
    torch.cuda.set_device(0)
    w = workload_kinect()
    seq = load_sequence(w, args.frames + 1)
    intr = make_intrinsics(w.fx, w.fy, w.cx, w.cy, w.width, w.height)
    depth = torch.from_numpy(seq.depth[:args.frames]).cuda()
    scene = Scene.from_workload(w)
    per = []
    for i in range(args.frames):
        scene.integrate(depth[i], intr, seq.poses[i])
        st = scene.stats()
        per.append({"frame": i, "updated": st["last_updated_voxels"],
                    "visible": st["last_visible_blocks"], "new": st["last_new_blocks"],
                    "allocated": st["allocated_blocks"]})
    print(json.dumps({"profile_frames": per}))


def profile_hd(args):
    """Small, deterministic case for ncu: frames 0..N-1 of the 1280x720, 4 mm
    sequence (rendered on the device) fused eagerly in int16 storage; prints
    per-frame counts so a captured launch can be scaled."""
    import torch
    from dataclasses import replace
    from paper_1410_0925_gb300 import Scene, make_intrinsics
    from synthdepth import workload_hd
    from synthdepth.configs import STORAGE_I16
    from synthdepth.render_torch import make_sequence_torch
    torch.cuda.set_device(0)
    # (a pool of 2^19 blocks holds the first frames and keeps the capture's
    # device memory near 1 GB)
    w = replace(workload_hd(), storage=STORAGE_I16, pool_blocks=1 << 19)
    seq = make_sequence_torch(w, n_frames=args.frames, device="cuda")
    intr = make_intrinsics(w.fx, w.fy, w.cx, w.cy, w.width, w.height)
    scene = Scene.from_workload(w)
    per = []
    for i in range(args.frames):
        scene.integrate(seq.depth[i], intr, seq.poses[i])
        st = scene.stats()
        per.append({"frame": i, "updated": st["last_updated_voxels"],
                    "visible": st["last_visible_blocks"], "new": st["last_new_blocks"],
                    "allocated": st["allocated_blocks"]})
    print(json.dumps({"profile_frames": per}))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", choices=["kinect", "hd", "colour", "icp", "swap", "raycast"],
                    default="kinect")
    ap.add_argument("--frames", type=int, default=45)
    args = ap.parse_args(argv)
    {"kinect": profile_fusion, "hd": profile_hd, "colour": profile_colour, "icp": profile_icp,
     "swap": profile_swap, "raycast": profile_raycast}[args.workload](args)


if __name__ == "__main__":
    main()
