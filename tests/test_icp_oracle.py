"""Pins of the depth-tracker oracle (Section 4.1: point-to-plane terms).

I1  closed form: reference plane z = 1 seen head-on, new depth a constant
    1.02 from the same pose: every pixel keeps its reference pixel, r =
    0.02 (normal sign s), J = (P x N, N), so E = 4e-4 per inlier, the
    translation-z gradient is 0.02 per inlier and the Hessian entries are
    sums over the normalised image coordinates.
I2  the distance threshold: below 0.02 every pixel is rejected.
I3  zero residual: the depth image of the reference view itself against its
    own maps gives E ~ 0 and g ~ 0 and one inlier per pixel with a normal.
I4  pose recovery: Gauss-Newton steps on the oracle's terms bring a pose
    estimate that is off by a known small motion back onto the true pose of
    an exact synthetic view (a room with objects).
I5  normals: a plane gives its unit normal; a sphere gives radial normals.
I6  a pixel whose reference projection sits on a rounding boundary is
    flagged and its slack covers the change.
"""

import numpy as np

import oracle
from synthdepth import make_sequence, workload_tiny
from synthdepth.scene import raycast_depth

W, H, F = 40, 30, 36.0
CX, CY = 19.3, 14.6


def _rays(w, h, f, cx, cy):
    u, v = np.meshgrid(np.arange(w, dtype=np.float64), np.arange(h, dtype=np.float64))
    return np.stack([(u - cx) / f, (v - cy) / f, np.ones_like(u)], -1)


def _points_from_depth(depth, pose, f, cx, cy):
    """World point map (H, W, 4) float32 of a z-depth image seen from pose."""
    h, w = depth.shape
    r = _rays(w, h, f, cx, cy)
    cam = r * depth[..., None]
    Minv = np.linalg.inv(pose)
    world = cam @ Minv[:3, :3].T + Minv[:3, 3]
    out = np.zeros((h, w, 4), np.float32)
    ok = depth > 0
    out[ok, :3] = world[ok]
    out[ok, 3] = 1.0
    return out


def test_i1_plane_closed_form():
    V = _points_from_depth(np.ones((H, W)), np.eye(4), F, CX, CY)
    N = oracle.icp_normals(V)
    interior = N[..., 3] == 1
    assert interior.sum() == (W - 2) * (H - 2)
    s = N[interior][:, 2]
    assert np.allclose(np.abs(s), 1.0) and np.allclose(N[interior][:, :2], 0.0)
    depth = np.full((H, W), 1.02, np.float32)
    out = oracle.icp_reduce(depth, (F, F, CX, CY), np.eye(4), np.eye(4), V, N, max_dist=0.1)
    Hm, g = oracle.icp_system(out["sums"])
    n = interior.sum()
    assert out["sums"][28] == n
    d32 = float(np.float32(1.02)) - 1.0                      # the float depth's offset
    r = _rays(W, H, F, CX, CY)[interior]
    xn, yn = r[:, 0], r[:, 1]
    np.testing.assert_allclose(out["sums"][27], n * d32 ** 2, rtol=1e-9)
    np.testing.assert_allclose(g[5], n * d32, rtol=1e-9)      # J_tz r = s (d s) = d
    # J = (P x N, N), P = 1.02 (xn, yn, 1), N = (0, 0, s)
    P32 = float(np.float32(1.02))
    np.testing.assert_allclose(Hm[0, 0], np.sum((P32 * yn) ** 2), rtol=1e-9)
    np.testing.assert_allclose(Hm[1, 1], np.sum((P32 * xn) ** 2), rtol=1e-9)
    np.testing.assert_allclose(Hm[0, 1], -np.sum(P32 ** 2 * xn * yn), rtol=1e-9, atol=1e-9)
    assert abs(Hm[2, 2]) < 1e-12 and Hm[5, 5] == n
    np.testing.assert_allclose(Hm[0, 5], np.sum(P32 * yn), rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(g[0], np.sum(P32 * yn * d32), rtol=1e-9, atol=1e-12)
    assert out["flags"].sum() == 0


def test_i2_distance_threshold():
    V = _points_from_depth(np.ones((H, W)), np.eye(4), F, CX, CY)
    N = oracle.icp_normals(V)
    depth = np.full((H, W), 1.02, np.float32)
    out = oracle.icp_reduce(depth, (F, F, CX, CY), np.eye(4), np.eye(4), V, N, max_dist=0.019)
    assert out["sums"][28] == 0 and out["sums"][27] == 0


def _room_view(pose, w):
    from synthdepth.configs import sequence_geometry
    scene, _, world_from_room = sequence_geometry(w, 1)
    # poses here are world->camera in the world frame; the scene is in room
    # coordinates: camera_from_room = pose @ world_from_room
    return raycast_depth(scene, pose @ world_from_room, w.width, w.height, w.fx, w.fy,
                         w.cx, w.cy)


def test_i3_zero_residual_on_own_view():
    w = workload_tiny()
    seq = make_sequence(w, n_frames=1)
    pose = seq.poses[0]
    depth = _room_view(pose, w).astype(np.float32)
    V = _points_from_depth(depth.astype(np.float64), pose, w.fx, w.cx, w.cy)
    N = oracle.icp_normals(V)
    out = oracle.icp_reduce(depth, (w.fx, w.fy, w.cx, w.cy), pose, pose, V, N, max_dist=0.1)
    n_norm = int((N[..., 3] == 1).sum())
    assert out["sums"][28] >= n_norm - out["flags"].sum() and n_norm > 10000
    assert out["sums"][27] < 1e-9 * n_norm
    assert np.abs(out["sums"][21:27]).max() < 1e-4


def _rodrigues(wv):
    th = np.linalg.norm(wv)
    if th < 1e-15:
        return np.eye(3)
    k = wv / th
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + np.sin(th) * K + (1 - np.cos(th)) * K @ K


def test_i4_gauss_newton_recovers_the_pose():
    w = workload_tiny()
    seq = make_sequence(w, n_frames=1)
    ref = seq.poses[0]
    depth_ref = _room_view(ref, w)
    V = _points_from_depth(depth_ref, ref, w.fx, w.cx, w.cy)
    N = oracle.icp_normals(V)
    # true pose: the camera moved by a small known motion
    D = np.eye(4)
    D[:3, :3] = _rodrigues(np.array([0.012, -0.02, 0.008]))
    D[:3, 3] = [0.02, -0.012, 0.015]
    true = D @ ref
    depth = _room_view(true, w).astype(np.float32)
    cur = ref.copy()
    for _ in range(8):
        out = oracle.icp_reduce(depth, (w.fx, w.fy, w.cx, w.cy), cur, ref, V, N, max_dist=0.1)
        Hm, g = oracle.icp_system(out["sums"])
        xi = -np.linalg.solve(Hm, g)
        # the step moves world points: P' = exp(w) P + t, i.e. the camera-to-
        # world transform is premultiplied by that motion
        step = np.eye(4)
        step[:3, :3] = _rodrigues(xi[:3])
        step[:3, 3] = xi[3:]
        cur = cur @ np.linalg.inv(step)
    err = np.linalg.inv(cur) @ true
    assert np.linalg.norm(err[:3, 3]) < 1e-3          # < 1 mm
    assert np.abs(err[:3, :3] - np.eye(3)).max() < 1e-3
    # and it did move: the start was 2.8 cm and ~1.4 degrees off
    assert np.linalg.norm((np.linalg.inv(ref) @ true)[:3, 3]) > 0.02


def test_i5_normals_of_plane_and_sphere():
    # sphere of radius 0.5 centred 1.5 m ahead, seen head-on
    u, v = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    r = _rays(W, H, F, CX, CY)
    d = r / np.linalg.norm(r, axis=-1, keepdims=True)
    c = np.array([0.0, 0.0, 1.5])
    b = d @ c
    disc = b ** 2 - (c @ c - 0.25)
    t = b - np.sqrt(np.maximum(disc, 0))
    depth = np.where(disc > 0, t * d[..., 2], 0.0)
    V = _points_from_depth(depth, np.eye(4), F, CX, CY)
    N = oracle.icp_normals(V)
    ok = N[..., 3] == 1
    assert ok.sum() > 200
    radial = V[..., :3].astype(np.float64) - c
    radial /= np.linalg.norm(radial, axis=-1, keepdims=True)
    cosang = np.abs(np.einsum("ijk,ijk->ij", N[..., :3], radial))[ok]
    assert np.quantile(cosang, 0.5) > 0.9999 and cosang.min() > 0.99


def _sphere_depth(pose):
    r = _rays(W, H, F, CX, CY)
    Minv = np.linalg.inv(pose)
    d = r @ Minv[:3, :3].T
    n = np.linalg.norm(d, axis=-1, keepdims=True)
    d = d / n
    C = Minv[:3, 3]
    c = np.array([0.0, 0.0, 1.5])
    oc = C - c
    b = d @ oc
    disc = b ** 2 - (oc @ oc - 0.25)
    t = -b - np.sqrt(np.maximum(disc, 0))
    return np.where(disc > 0, t / n[..., 0], 0.0)   # camera z = t / |r|


def test_i6_rounding_boundary_is_flagged_with_slack():
    # the current view is the plane z = 1; the reference camera sits 0.5 / F
    # to the side, so every current point projects exactly onto a rounding
    # boundary of the reference view, whose map (a sphere) differs from
    # pixel to pixel
    ref = np.eye(4)
    ref[0, 3] = 0.5 / F
    V = _points_from_depth(_sphere_depth(ref), ref, F, CX, CY)
    N = oracle.icp_normals(V)
    depth = np.ones((H, W), np.float32)
    out = oracle.icp_reduce(depth, (F, F, CX, CY), np.eye(4), ref, V, N, max_dist=10.0)
    with_normal = N[..., 3] == 1
    assert out["flags"][with_normal].mean() > 0.9
    assert (out["slack"] >= 0).all() and out["slack"][28] <= out["flags"].sum()
    assert out["slack"][27] > 0 and out["slack"][0] > 0
    # a quarter pixel off the boundary nothing is flagged
    ref[0, 3] = 0.25 / F
    V = _points_from_depth(_sphere_depth(ref), ref, F, CX, CY)
    out0 = oracle.icp_reduce(depth, (F, F, CX, CY), np.eye(4), ref, V, oracle.icp_normals(V),
                             max_dist=10.0)
    assert out0["flags"].sum() == 0 and (out0["slack"] == 0).all()


def test_i7_depth_hierarchy_level():
    # hand-made 4x4: blocks with 4, 3, 1 and 0 valid depths
    d = np.array([[1.0, 2.0, 5.0, 0.0],
                  [3.0, 4.0, np.nan, 7.0],
                  [0.0, -1.0, 0.0, 0.0],
                  [0.0, 6.5, 0.0, np.inf]], np.float32)
    out = oracle.icp_downsample(d)
    assert out.shape == (2, 2)
    assert out[0, 0] == np.float32(2.5)               # (1 + 2 + 3 + 4) / 4
    assert out[0, 1] == np.float32(6.0)               # (5 + 7) / 2
    assert out[1, 0] == np.float32(6.5) and out[1, 1] == 0.0
    # odd sizes drop the last row / column; the coarse pixel centres follow
    # (cx - 1/2) / 2; a block's value is the mean of its four depths
    w = 41
    u, v = np.meshgrid(np.arange(w, dtype=np.float64), np.arange(31, dtype=np.float64))
    f, cx, cy = 40.0, 20.3, 15.1
    plane = (1.0 / (1.0 + 0.2 * (u - cx) / f)).astype(np.float32)   # x = -5 z + 5, tilted
    c = oracle.icp_downsample(plane)
    assert c.shape == (15, 20)
    uc = np.arange(20, dtype=np.float64)
    x_fine = (2 * uc + 0.5 - cx) / f
    x_coarse = (uc - (cx - 0.5) / 2) / (f / 2)
    assert np.allclose(x_fine, x_coarse)              # the intrinsics of the coarse level
    want = (plane[0, 0:40:2] + plane[0, 1:40:2] + plane[1, 0:40:2] + plane[1, 1:40:2]) / 4
    np.testing.assert_allclose(c[0], want, rtol=1e-6)
