"""GPU parity of the raycast (Section 4.4): tsdf_raycast through the C ABI
against the FP64 raycast oracle on identical volumes -- the oracle's own
fused volume (or an analytic one) loaded into the CUDA scene with
tsdf_load_blocks -- pixel by pixel (see parity.compare_raycast)."""

import numpy as np
import pytest

import oracle
from parity import (compare_raycast, f32, oracle_intr, ray_params, run_oracle,
                    storage_arrays)
from synthdepth import make_sequence, workload_kinect, workload_tiny
from synthdepth.configs import STORAGE_F16, STORAGE_F32, STORAGE_I16

pytestmark = pytest.mark.gpu


def _load(w, keys, sdf_values, wts, storage, **over):
    from paper_1410_0925_gb300 import Blocks, Scene
    raw, held = storage_arrays(sdf_values, storage)
    sc = Scene.from_workload(w, storage=storage, **over)
    sc.load_blocks(Blocks(np.asarray(keys, np.int16), raw, np.asarray(wts, np.uint8)))
    return sc, held


def _intr(w, width=None, height=None):
    from paper_1410_0925_gb300 import make_intrinsics
    return make_intrinsics(w.fx, w.fy, w.cx, w.cy, width or w.width, height or w.height)


def _raycast_pair(sc, keys, held, w, pose, z_near=0.2):
    import torch
    H, W = w.height, w.width
    rng = torch.empty((H, W, 2), dtype=torch.float32, device="cuda")
    pts = sc.raycast(_intr(w), pose, z_near=z_near, range_out=rng)
    torch.cuda.synchronize()
    vol = oracle.Volume(keys, held)
    orc = vol.raycast(W, H, oracle_intr(w), pose, ray_params(w, z_near))
    return pts.cpu().numpy(), rng.cpu().numpy(), orc


def _moved(pose, dx=0.031, angle=0.035):
    c, s = np.cos(angle), np.sin(angle)
    dR = np.array([[c, 0, s, dx], [0, 1, 0, -0.012], [-s, 0, c, 0.02], [0, 0, 0, 1.0]])
    return dR @ np.asarray(pose)


@pytest.mark.parametrize("storage", [STORAGE_F32, STORAGE_I16, STORAGE_F16])
def test_raycast_of_fused_volume_matches_oracle(storage):
    w = workload_tiny(storage=storage)
    seq = make_sequence(w, n_frames=6)
    res = run_oracle(w, seq)["res"]
    sc, held = _load(w, res["keys"], res["sdf"], res["w"], storage)
    for pose in (seq.poses[-1], _moved(seq.poses[-1]), seq.poses[0]):
        pts, rng, orc = _raycast_pair(sc, res["keys"], held, w, pose)
        rep = compare_raycast(pts, rng, orc, w.width, w.height, f32(w.voxel_size))
        print(rep)
        assert rep["hits"] > 0.5 * rep["pixels"]
    st = sc.raycast_stats()
    assert st["hits"] == int((pts[..., 3] == 1).sum())
    assert st["guard_stops"] == 0 and st["footprints"] > 0


def test_raycast_kinect_full_resolution():
    """640x480 at 5 mm after three noisy frames (~16k blocks): every pixel
    against the oracle, search ranges included."""
    w = workload_kinect()
    seq = make_sequence(w, n_frames=3)
    res = run_oracle(w, seq)["res"]
    sc, held = _load(w, res["keys"], res["sdf"], res["w"], STORAGE_F32)
    pts, rng, orc = _raycast_pair(sc, res["keys"], held, w, seq.poses[-1])
    rep = compare_raycast(pts, rng, orc, w.width, w.height, f32(w.voxel_size))
    print(rep)
    assert rep["hits"] > 0.9 * rep["pixels"]
    st = sc.raycast_stats()
    ok = orc["flags"] == 0
    # unflagged rays take exactly the oracle's samples
    o_steps = int(orc["steps"][ok].sum())
    assert abs(st["steps"] - int(orc["steps"].sum())) <= 0.02 * o_steps


def _plane(w_s, mu, D, kz, half):
    r = np.arange(-half, half)
    keys = np.array([(x, y, z) for z in kz for y in r for x in r], np.int32)
    loc = np.arange(512)
    z = (8 * keys[:, 2:3] + loc // 64) * w_s
    return keys, np.clip((D - z) / mu, -1.0, 1.0)


def test_raycast_close_up_wide_footprints_and_near_plane():
    """A plane seen from close by with a long focal length: block footprints
    span more than 16 tiles (the list every tile reads); with z_near inside
    the first block layer that layer is clipped, the search starts in the
    second layer, past the surface, and the step back of the coarse search
    finds it."""
    w = workload_tiny(width=128, height=96, fx=120.0, fy=120.0, cx=63.3, cy=47.6,
                      voxel_size=0.02, mu=0.08)
    s = f32(w.voxel_size)
    # the surface more than mu behind the slab's front face, as fusion
    # allocates it (the band reaches mu in front of the surface)
    keys, sdf = _plane(s, f32(w.mu), 8 * 2 * s + 0.1437, kz=(2, 3), half=6)
    sc, held = _load(w, keys, sdf, np.ones(sdf.shape, np.uint8), STORAGE_F32)
    # slightly tilted: seen exactly head-on, every ray would start on the
    # slab's front face (a block boundary, flagged)
    a, b = 0.05, -0.04
    Rx = np.array([[1, 0, 0], [0, np.cos(a), -np.sin(a)], [0, np.sin(a), np.cos(a)]])
    Ry = np.array([[np.cos(b), 0, np.sin(b)], [0, 1, 0], [-np.sin(b), 0, np.cos(b)]])
    pose = np.eye(4)
    pose[:3, :3] = Rx @ Ry
    for z_near in (0.05, 0.371):
        pts, rng, orc = _raycast_pair(sc, keys, held, w, pose, z_near=z_near)
        rep = compare_raycast(pts, rng, orc, w.width, w.height, s)
        print(z_near, rep, sc.raycast_stats())
        if z_near < 0.3:
            assert sc.raycast_stats()["wide_footprints"] > 0
        assert rep["hits"] > 0.9 * rep["pixels"]


def test_raycast_empty_scene_and_bad_arguments():
    import torch
    from paper_1410_0925_gb300 import Scene, TsdfError
    w = workload_tiny()
    sc = Scene.from_workload(w)
    rng = torch.empty((w.height, w.width, 2), dtype=torch.float32, device="cuda")
    pts = sc.raycast(_intr(w), np.eye(4), range_out=rng)
    torch.cuda.synchronize()
    assert (pts == 0).all()
    assert torch.isposinf(rng[..., 0]).all() and torch.isneginf(rng[..., 1]).all()
    assert sc.raycast_stats()["footprints"] == 0
    for z_near in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(TsdfError):
            sc.raycast(_intr(w), np.eye(4), z_near=z_near)
    bad = np.eye(4)
    bad[3, 0] = 0.5
    with pytest.raises(TsdfError):
        sc.raycast(_intr(w), bad)
    flat = torch.empty(w.height * w.width * 4 + 1, dtype=torch.float32, device="cuda")
    with pytest.raises(TsdfError):                      # 4-byte aligned, not 16
        sc.raycast(_intr(w), np.eye(4), points=flat[1:].view(w.height, w.width, 4))
    with pytest.raises(ValueError):
        sc.raycast(_intr(w), np.eye(4), points=torch.empty((2, 2, 4), device="cuda"))


def test_raycast_after_fusion_in_graph_and_independent_of_hash_layout():
    """Raycast straight after tsdf_integrate_frames on the scene stream, the
    same call captured into a CUDA graph and replayed, and the raycast of the
    same blocks loaded into a scene with a 16-bucket hash table (nearly every
    block in an excess chain) give bit-identical images."""
    import torch
    from paper_1410_0925_gb300 import Scene
    w = workload_tiny()
    seq = make_sequence(w, n_frames=8)
    stream = torch.cuda.Stream()
    sc = Scene.from_workload(w, stream=stream)
    depth = torch.from_numpy(np.ascontiguousarray(seq.depth)).cuda()
    torch.cuda.synchronize()
    intr = _intr(w)
    pose = _moved(seq.poses[-1])
    with torch.cuda.stream(stream):
        sc.integrate_frames(depth, intr, seq.poses)
        a = sc.raycast(intr, pose).clone()
        g = torch.cuda.CUDAGraph()
        out = torch.empty_like(a)
        with torch.cuda.graph(g, stream=stream):
            sc.raycast(intr, pose, points=out)
        out.zero_()
        g.replay()
    stream.synchronize()
    assert torch.equal(a, out)
    assert (a[..., 3] == 1).float().mean() > 0.5
    blocks = sc.read_blocks()
    small = Scene.from_workload(w, hash_buckets_log2=4, excess_entries=1 << 14)
    small.load_blocks(blocks)
    b = small.raycast(intr, pose)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
