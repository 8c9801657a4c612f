"""GPU parity of the depth tracker's terms (Section 4.1): tsdf_icp_normals and
tsdf_icp_reduce through the C ABI against the oracle (or_icp_normals,
or_icp_reduce) on the same reference point map (an exact synthetic view) and
depth images; tolerances in parity.compare_icp. A GPU-driven Gauss-Newton
loop recovers a known pose."""

import numpy as np
import pytest

import oracle
from parity import compare_icp
from synthdepth import make_sequence, workload_kinect, workload_tiny
from synthdepth.configs import sequence_geometry
from synthdepth.scene import raycast_depth

pytestmark = pytest.mark.gpu


def _room_view(pose, w):
    scene, _, world_from_room = sequence_geometry(w, 1)
    return raycast_depth(scene, pose @ world_from_room, w.width, w.height, w.fx, w.fy, w.cx, w.cy)


def _points(depth, pose, w):
    u, v = np.meshgrid(np.arange(w.width, dtype=np.float64), np.arange(w.height, dtype=np.float64))
    r = np.stack([(u - w.cx) / w.fx, (v - w.cy) / w.fy, np.ones_like(u)], -1)
    Minv = np.linalg.inv(pose)
    world = (r * depth[..., None]) @ Minv[:3, :3].T + Minv[:3, 3]
    out = np.zeros((w.height, w.width, 4), np.float32)
    ok = depth > 0
    out[ok, :3] = world[ok]
    out[ok, 3] = 1.0
    return out


def _rodrigues(wv):
    th = np.linalg.norm(wv)
    K = np.array([[0, -wv[2], wv[1]], [wv[2], 0, -wv[0]], [-wv[1], wv[0], 0]]) / max(th, 1e-300)
    return np.eye(3) + np.sin(th) * K + (1 - np.cos(th)) * K @ K if th > 0 else np.eye(3)


def _motion(w3, t3):
    D = np.eye(4)
    D[:3, :3] = _rodrigues(np.asarray(w3, np.float64))
    D[:3, 3] = t3
    return D


def _intr(w):
    from paper_1410_0925_gb300 import make_intrinsics
    return make_intrinsics(w.fx, w.fy, w.cx, w.cy, w.width, w.height)


def _f32intr(w):
    return [float(np.float32(x)) for x in (w.fx, w.fy, w.cx, w.cy)]


def _case(w, depth, cur, ref, V, max_dist=0.1):
    import torch
    from paper_1410_0925_gb300 import Icp
    icp = Icp()
    Vd = torch.from_numpy(V).cuda()
    Nd = icp.normals(Vd)
    dd = torch.from_numpy(np.ascontiguousarray(depth, np.float32)).cuda()
    sums = icp.reduce(dd, _intr(w), cur, ref, Vd, Nd, max_dist).cpu().numpy()
    No = oracle.icp_normals(V)
    orc = oracle.icp_reduce(depth, _f32intr(w), cur, ref, V, No, float(np.float32(max_dist)))
    return icp, Nd.cpu().numpy(), No, sums, orc


def test_normals_match_oracle():
    w = workload_tiny()
    ref = make_sequence(w, n_frames=1).poses[0]
    V = _points(_room_view(ref, w), ref, w)
    _, Ng, No, _, _ = _case(w, _room_view(ref, w), ref, ref, V)
    ok = No[..., 3] == 1
    assert np.array_equal(Ng[..., 3] == 1, ok) and ok.sum() > 10000
    assert np.abs(Ng[ok][:, :3] - No[ok][:, :3]).max() < 1e-4
    assert (Ng[~ok] == 0).all()


@pytest.mark.parametrize("offset", [0.0, 1.0])
def test_terms_match_oracle_tiny(offset):
    w = workload_tiny()
    ref = make_sequence(w, n_frames=1).poses[0]
    V = _points(_room_view(ref, w), ref, w)
    true = _motion(np.array([0.012, -0.02, 0.008]) * offset, np.array([0.02, -0.012, 0.015]) * offset) @ ref
    depth = _room_view(true, w).astype(np.float32)
    _, _, _, sums, orc = _case(w, depth, ref, ref, V)
    rep = compare_icp(sums, orc)
    print(rep)
    assert rep["inliers"] > 10000


def test_terms_match_oracle_kinect_noisy_frame():
    """640x480: a noisy frame of the Kinect sequence against the exact view of
    the previous frame's pose, from that pose."""
    w = workload_kinect()
    seq = make_sequence(w, n_frames=2)
    ref = seq.poses[0]
    V = _points(_room_view(ref, w), ref, w)
    _, _, _, sums, orc = _case(w, seq.depth[1], ref, ref, V)
    rep = compare_icp(sums, orc)
    print(rep)
    assert rep["inliers"] > 200000


def test_gpu_gauss_newton_recovers_the_pose_and_is_deterministic():
    import torch
    from paper_1410_0925_gb300 import Icp
    w = workload_tiny()
    ref = make_sequence(w, n_frames=1).poses[0]
    V = torch.from_numpy(_points(_room_view(ref, w), ref, w)).cuda()
    stream = torch.cuda.Stream()
    icp = Icp(stream=stream)
    N = icp.normals(V)
    true = _motion([0.012, -0.02, 0.008], [0.02, -0.012, 0.015]) @ ref
    depth = torch.from_numpy(_room_view(true, w).astype(np.float32)).cuda()
    torch.cuda.synchronize()
    cur = ref.copy()
    for _ in range(8):
        with torch.cuda.stream(stream):
            s = icp.reduce(depth, _intr(w), cur, ref, V, N)
        stream.synchronize()
        Hm, g = Icp.system(s)
        xi = -np.linalg.solve(Hm, g)
        cur = cur @ np.linalg.inv(_motion(xi[:3], xi[3:]))
    err = np.linalg.inv(cur) @ true
    assert np.linalg.norm(err[:3, 3]) < 1e-3 and np.abs(err[:3, :3] - np.eye(3)).max() < 1e-3
    # same inputs, same sums, eagerly and replayed from a CUDA graph
    with torch.cuda.stream(stream):
        a = icp.reduce(depth, _intr(w), ref, ref, V, N).clone()
        g = torch.cuda.CUDAGraph()
        out = torch.zeros_like(a)
        with torch.cuda.graph(g, stream=stream):
            icp.reduce(depth, _intr(w), ref, ref, V, N, sums=out)
        g.replay()
    stream.synchronize()
    assert torch.equal(a, out)
    assert icp.kernel_launches() > 8


def test_icp_bad_arguments():
    import torch
    from paper_1410_0925_gb300 import Icp, TsdfError
    w = workload_tiny()
    icp = Icp()
    V = torch.zeros((w.height, w.width, 4), device="cuda")
    N = icp.normals(V)
    assert (N == 0).all()
    d = torch.ones((w.height, w.width), device="cuda")
    bad = np.eye(4)
    bad[3, 2] = 1.0
    with pytest.raises(TsdfError):
        icp.reduce(d, _intr(w), bad, np.eye(4), V, N)
    with pytest.raises(TsdfError):
        icp.reduce(d, _intr(w), np.eye(4), np.eye(4), V, N, max_dist=0.0)
    flat = torch.zeros(w.height * w.width * 4 + 1, device="cuda")
    with pytest.raises(TsdfError):
        icp.reduce(d, _intr(w), np.eye(4), np.eye(4), flat[1:].view(w.height, w.width, 4), N)
    s = icp.reduce(d, _intr(w), np.eye(4), np.eye(4), V, N)
    assert float(s[28]) == 0.0


def _step_host(pose, sums):
    Hm = np.zeros((6, 6))
    t = 0
    for a in range(6):
        for b in range(a, 6):
            Hm[a, b] = Hm[b, a] = sums[t]
            t += 1
    xi = -np.linalg.solve(Hm, np.asarray(sums[21:27]))
    return pose @ np.linalg.inv(_motion(xi[:3], xi[3:]))


def test_device_solve_matches_the_host_step_on_oracle_terms():
    """The device's Cholesky solve and pose update, fed the oracle's terms,
    give the pose a host solve of the same terms gives."""
    import torch
    from paper_1410_0925_gb300 import Icp
    w = workload_tiny()
    ref = make_sequence(w, n_frames=1).poses[0]
    V = _points(_room_view(ref, w), ref, w)
    true = _motion([0.012, -0.02, 0.008], [0.02, -0.012, 0.015]) @ ref
    depth = _room_view(true, w).astype(np.float32)
    orc = oracle.icp_reduce(depth, _f32intr(w), ref, ref, V, oracle.icp_normals(V), 0.1)
    icp = Icp()
    pose = torch.from_numpy(ref.copy()).cuda()
    icp.solve(torch.from_numpy(orc["sums"]).cuda(), pose)
    got = pose.cpu().numpy()
    want = _step_host(ref, orc["sums"])
    assert np.abs(got - want).max() < 1e-12
    assert icp.status() == 0
    # too few inliers: the pose is kept and the status says so
    empty = torch.zeros(29, dtype=torch.float64, device="cuda")
    icp.solve(empty, pose)
    assert np.array_equal(pose.cpu().numpy(), got) and icp.status() == 2


def test_device_tracking_recovers_the_pose_in_a_graph():
    import torch
    from paper_1410_0925_gb300 import Icp
    w = workload_tiny()
    ref = make_sequence(w, n_frames=1).poses[0]
    V = torch.from_numpy(_points(_room_view(ref, w), ref, w)).cuda()
    stream = torch.cuda.Stream()
    icp = Icp(stream=stream)
    N = icp.normals(V)
    true = _motion([0.012, -0.02, 0.008], [0.02, -0.012, 0.015]) @ ref
    depth = torch.from_numpy(_room_view(true, w).astype(np.float32)).cuda()
    start = torch.from_numpy(ref.copy()).cuda()
    pose = start.clone()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        icp.track(depth, _intr(w), pose, ref, V, N, 0.1, iterations=8)
    stream.synchronize()
    est = pose.cpu().numpy()
    err = np.linalg.inv(est) @ true
    assert np.linalg.norm(err[:3, 3]) < 1e-3 and np.abs(err[:3, :3] - np.eye(3)).max() < 1e-3
    assert icp.status() == 0
    # the same iterations driven from the host give the same pose
    cur = ref.copy()
    for _ in range(8):
        with torch.cuda.stream(stream):
            s = icp.reduce(depth, _intr(w), cur, ref, V, N)
        stream.synchronize()
        cur = _step_host(cur, s.cpu().numpy())
    assert np.abs(cur - est).max() < 1e-5
    # captured once, replayed twice from the start pose
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(g, stream=stream):
            pose.copy_(start)
            icp.track(depth, _intr(w), pose, ref, V, N, 0.1, iterations=8)
        for _ in range(2):
            pose.zero_()
            g.replay()
    stream.synchronize()
    assert torch.equal(pose.cpu(), torch.from_numpy(est))


def test_depth_hierarchy_matches_oracle_bit_exact():
    import torch
    from paper_1410_0925_gb300 import Icp
    w = workload_kinect()
    seq = make_sequence(w, n_frames=1)          # noisy, with dropped pixels
    icp = Icp()
    d0 = torch.from_numpy(seq.depth[0]).cuda()
    d1 = icp.downsample(d0)
    d2 = icp.downsample(d1)
    o1 = oracle.icp_downsample(seq.depth[0])
    o2 = oracle.icp_downsample(o1)
    assert np.array_equal(d1.cpu().numpy(), o1) and np.array_equal(d2.cpu().numpy(), o2)
    assert d2.shape == (120, 160) and (o1 == 0).mean() < 0.01


def test_coarse_to_fine_tracking_recovers_the_pose():
    import torch
    from dataclasses import replace
    from paper_1410_0925_gb300 import Icp
    w = workload_tiny(width=320, height=240, fx=262.5, fy=262.5, cx=159.5, cy=119.5)
    ref = make_sequence(w, n_frames=1).poses[0]
    true = _motion([0.03, -0.04, 0.02], [0.05, -0.03, 0.04]) @ ref
    icp = Icp()
    depth = [torch.from_numpy(_room_view(true, w).astype(np.float32)).cuda()]
    for _ in range(2):
        depth.append(icp.downsample(depth[-1]))
    pose = torch.from_numpy(ref.copy()).cuda()
    for level in (2, 1, 0):
        il = Icp.level_intrinsics(_intr(w), level)
        wl = replace(w, width=il.width, height=il.height, fx=il.fx, fy=il.fy, cx=il.cx, cy=il.cy)
        V = torch.from_numpy(_points(_room_view(ref, wl), ref, wl)).cuda()
        N = icp.normals(V)
        icp.track(depth[level], il, pose, ref, V, N, 0.2, iterations=6)
    est = pose.cpu().numpy()
    err = np.linalg.inv(est) @ true
    assert np.linalg.norm(err[:3, 3]) < 2e-3 and np.abs(err[:3, :3] - np.eye(3)).max() < 2e-3
    assert icp.status() == 0
