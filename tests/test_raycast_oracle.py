"""Pins of the raycast oracle (Section 4.4) against what geometry fixes.

The volumes here are analytic: a plane's or a sphere's truncated distance
sampled at the voxel lattice, so the surface every ray must find is known in
closed form. The pins:
  - plane seen head-on: the central ray lands on the plane exactly, every
    other ray within the two-refinement-step residual (1 - cos a)^2 voxels
    (a = angle between ray and plane normal); every pixel finds it;
  - plane seen from behind its band (values negative on the camera side):
    WRONG_SIDE everywhere, no surface;
  - thin slab entered by a coarse step past the surface: the step back
    makes every pixel find the surface;
  - sphere: hits on the sphere within the same residual, rays that pass
    more than a voxel outside it find nothing, rays more than a voxel inside
    all hit;
  - search range: the closed-form footprint of one block; the near-plane
    rules; a brute-force ray / box test showing the range contains every
    block a ray meets;
  - trilinear read: exact on an affine field, unreadable next to a missing
    block;
  - ambiguity flags: a sample on a block boundary is flagged.
"""

import numpy as np
import pytest

import oracle
from oracle import RayParams, Volume

LOCAL = np.arange(512)
LX, LY, LZ = LOCAL % 8, (LOCAL // 8) % 8, LOCAL // 64


def field_volume(keys, fn, s):
    """sdf[n][512] = fn(x, y, z) at the world positions v * s of every voxel."""
    keys = np.asarray(keys, dtype=np.int64).reshape(-1, 3)
    x = (8 * keys[:, 0:1] + LX) * s
    y = (8 * keys[:, 1:2] + LY) * s
    z = (8 * keys[:, 2:3] + LZ) * s
    return keys.astype(np.int32), fn(x, y, z)


def slab_keys(kz, half_blocks):
    r = np.arange(-half_blocks, half_blocks)
    return np.array([(x, y, z) for z in kz for y in r for x in r], np.int32)


def intr_of(f, cx, cy):
    return [f, f, cx, cy]


def rays(W, H, f, cx, cy):
    u, v = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    r = np.stack([(u - cx) / f, (v - cy) / f, np.ones_like(u)], -1).reshape(-1, 3)
    return r / np.linalg.norm(r, axis=1, keepdims=True)


def rot(ax, ay):
    cx_, sx_ = np.cos(ax), np.sin(ax)
    cy_, sy_ = np.cos(ay), np.sin(ay)
    Rx = np.array([[1, 0, 0], [0, cx_, -sx_], [0, sx_, cx_]])
    Ry = np.array([[cy_, 0, sy_], [0, 1, 0], [-sy_, 0, cy_]])
    return Rx @ Ry


def pose_from(R, t):
    M = np.eye(4)
    M[:3, :3] = R
    M[:3, 3] = t
    return M


S, MU = 0.02, 0.08  # mu = 4 voxels
W, H, F, CX, CY = 64, 48, 60.0, 32.0, 24.0


def plane_volume(D, sign=1.0, kz=(11, 12, 13), half_blocks=10):
    keys = slab_keys(kz, half_blocks)
    return field_volume(keys, lambda x, y, z: np.clip(sign * (D - z) / MU, -1.0, 1.0), S)


def test_plane_head_on_closed_form():
    D = 8 * 12 * S + 0.5 * 8 * S + 0.0037  # inside block layer 12 (z in [1.92, 2.08])
    keys, sdf = plane_volume(D)
    vol = Volume(keys, sdf)
    p = RayParams(voxel_size=S, mu=MU)
    out = vol.raycast(W, H, intr_of(F, CX, CY), np.eye(4), p)
    pts = out["points"]
    assert (pts[:, 3] == 1.0).all(), "every ray meets the plane"
    d = rays(W, H, F, CX, CY)
    # the point lies on its ray
    cross = np.cross(pts[:, :3], d)
    assert np.abs(cross).max() < 1e-9
    # depth within the residual of two refinement steps
    cos_a = d[:, 2]
    err = np.abs(pts[:, 2] - D)
    assert (err <= (1 - cos_a) ** 2 * S + 1e-9).all(), err.max()
    centre = int(CY) * W + int(CX)
    assert abs(pts[centre, 2] - D) < 1e-12
    # error multiplier: the central ray meets the plane head-on, so every
    # value-sized step maps t onto the plane whatever its error (|1 + mu
    # dsdf/dt| = 0) and leaves only the sensitivity of the value it read
    # (mu sqrt(3) / mu + 1) and the final point's own error (+1)
    assert abs(out["gain"][centre] - (2.0 + np.sqrt(3.0))) < 1e-9
    assert (out["gain"] >= 2.0).all()
    # the residual is not trivially zero off-axis (the pin has teeth)
    assert err.max() > 1e-6


def test_plane_seen_from_behind_is_wrong_side():
    D = 8 * 12 * S + 0.5 * 8 * S + 0.0037
    keys, sdf = plane_volume(D, sign=-1.0)
    vol = Volume(keys, sdf)
    out = vol.raycast(W, H, intr_of(F, CX, CY), np.eye(4), RayParams(voxel_size=S, mu=MU))
    assert (out["points"][:, 3] == 0.0).all()
    assert (out["steps"] > 0).all()            # the march ran and stopped early
    assert out["steps"].max() < 20


def test_step_back_finds_surface_past_first_coarse_sample():
    # a slab three blocks thick whose surface lies 6 voxels behind its front
    # face: a coarse step lands past it on many rays; stepping back one block
    # and searching in steps of mu finds it on every ray
    kz = (12, 13, 14)
    z_front = 8 * 12 * S
    D = z_front + 6 * S
    keys, sdf = plane_volume(D, kz=kz, half_blocks=16)
    vol = Volume(keys, sdf)
    R = rot(0.21, -0.13)
    cam = np.array([0.03, -0.05, 0.0])       # camera centre in the world
    M = pose_from(R, -R @ cam)
    out = vol.raycast(W, H, intr_of(F, 31.3, 23.6), M, RayParams(voxel_size=S, mu=MU))
    pts = out["points"]
    assert (pts[:, 3] == 1.0).all()
    # world ray directions and the plane's residual bound
    d = rays(W, H, F, 31.3, 23.6) @ R  # R^T applied to each row
    cos_a = np.abs(d[:, 2])
    err = np.abs(pts[:, 2] - D)
    assert (err <= (1 - cos_a) ** 2 * S + 1e-9).all(), err.max()


def test_thin_slab_at_negative_coordinates():
    # camera looking down -z at a slab one block thick (world z in
    # [-1.92, -1.76]) with the surface in its middle: negative block and voxel
    # coordinates throughout (floor, not truncation, finds the blocks)
    Dw = -1.84 - 0.0037
    keys = slab_keys((-12,), 12)
    keys, sdf = field_volume(keys, lambda x, y, z: np.clip((z - Dw) / MU, -1.0, 1.0), S)
    vol = Volume(keys, sdf)
    M = pose_from(np.diag([-1.0, 1.0, -1.0]), np.zeros(3))
    out = vol.raycast(W, H, intr_of(F, 31.3, 23.6), M, RayParams(voxel_size=S, mu=MU))
    pts = out["points"]
    assert (pts[:, 3] == 1.0).all()
    cos_a = rays(W, H, F, 31.3, 23.6)[:, 2]
    err = np.abs(pts[:, 2] - Dw)
    assert (err <= (1 - cos_a) ** 2 * S + 1e-9).all(), err.max()


def sphere_case():
    c = np.array([0.021, -0.013, 1.0])
    R = 0.25
    rng = np.arange(-10, 10)
    keys = []
    for bz in rng:
        for by in rng:
            for bx in rng:
                lo = np.array([bx, by, bz]) * 8 * S
                hi = lo + 8 * S
                dmin = np.linalg.norm(np.maximum(0, np.maximum(lo - c, c - hi)))
                dmax = np.linalg.norm(np.maximum(np.abs(lo - c), np.abs(hi - c)))
                if dmin <= R + 2 * MU and dmax >= R - 2 * MU:
                    keys.append((bx, by, bz))
    keys, sdf = field_volume(
        np.array(keys),
        lambda x, y, z: np.clip((np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) - R)
                                / MU, -1.0, 1.0), S)
    return c, R, keys, sdf


def test_sphere_hits_lie_on_the_sphere():
    c, R, keys, sdf = sphere_case()
    vol = Volume(keys, sdf)
    Wd, Hd, f, cx, cy = 48, 40, 40.0, 23.7, 19.6
    out = vol.raycast(Wd, Hd, intr_of(f, cx, cy), np.eye(4), RayParams(voxel_size=S, mu=MU))
    pts = out["points"]
    d = rays(Wd, Hd, f, cx, cy)
    along = d @ c
    miss = np.sqrt(np.maximum(0.0, c @ c - along ** 2))     # closest approach to the centre
    inside = miss < R - S
    outside = miss > R + S
    assert inside.sum() > 100 and outside.sum() > 100
    assert (pts[inside, 3] == 1.0).all()
    assert (pts[outside, 3] == 0.0).all()
    hit = pts[:, 3] == 1.0
    # exact first intersection along each hit ray
    t_star = along - np.sqrt(np.maximum(0.0, R ** 2 - miss ** 2))
    t_hit = np.einsum("ij,ij->i", pts[:, :3], d)
    assert np.abs(np.cross(pts[hit, :3], d[hit])).max() < 1e-9
    normal = (t_star[:, None] * d - c) / R
    cos_a = np.abs(np.einsum("ij,ij->i", normal, d))
    good = hit & inside & (cos_a > 0.5)
    bound = ((1 - cos_a) ** 2 + 0.05) * S
    assert (np.abs(t_hit - t_star)[good] <= bound[good]).all()
    # any hit is within a voxel of the sphere
    assert (np.abs(np.linalg.norm(pts[hit, :3] - c, axis=1) - R) < S).all()


def test_range_of_one_block_closed_form():
    key = np.array([[2, -1, 6]], np.int32)          # box x [.32,.48] y [-.16,0] z [.96,1.12]
    vol = Volume(key, np.ones((1, 512)))
    Wd, Hd, f, cx, cy = 100, 80, 100.0, 50.3, 40.7
    rng, fl = vol.expected_depth(Wd, Hd, intr_of(f, cx, cy), np.eye(4),
                                 RayParams(voxel_size=S, mu=MU))
    x0, x1, y0, y1, z0, z1 = 0.32, 0.48, -0.16, 0.0, 0.96, 1.12
    # x > 0: the leftmost corner is far, the rightmost near; y <= 0: the top
    # corner is near, the bottom corner (y = 0) projects to cy at any depth
    umin, umax = f * x0 / z1 + cx, f * x1 / z0 + cx
    vmin, vmax = f * y0 / z0 + cy, cy
    u = np.arange(Wd)[None, :]
    v = np.arange(Hd)[:, None]
    cov = (u >= umin) & (u <= umax) & (v >= vmin) & (v <= vmax)
    assert cov.sum() > 50
    assert np.allclose(rng[cov, 0], z0, atol=1e-12) and np.allclose(rng[cov, 1], z1, atol=1e-12)
    assert np.isposinf(rng[~cov, 0]).all() and np.isneginf(rng[~cov, 1]).all()
    assert (fl == 0).all()


def test_range_near_plane_rules():
    # z_near clips whole blocks: wholly nearer, or straddling, covers nothing
    p = RayParams(voxel_size=S, mu=MU, z_near=0.5)
    intr = intr_of(10.0, 8.0, 6.0)
    for key in ([0, 0, 1], [0, 0, 2], [-1, -1, 3]):     # z in [.16,.32], [.32,.48], [.48,.64]
        vol = Volume(np.array([key], np.int32), np.ones((1, 512)))
        rng, fl = vol.expected_depth(16, 12, intr, np.eye(4), p)
        assert np.isposinf(rng[..., 0]).all() and (fl == 0).all()
    # wholly beyond it: box x, y in [-.16, 0], z in [.64, .8]; u in
    # [10 (-.16) / .64 + 8, 8] = [5.5, 8], v in [3.5, 6]
    vol = Volume(np.array([[-1, -1, 4]], np.int32), np.ones((1, 512)))
    rng, fl = vol.expected_depth(16, 12, intr, np.eye(4), p)
    cov = np.zeros((12, 16), bool)
    cov[4:7, 6:9] = True
    assert np.isposinf(rng[~cov, 0]).all()
    assert np.allclose(rng[cov, 0], 0.64) and np.allclose(rng[cov, 1], 0.8)
    # a block whose nearest corner sits within delta_z of z_near is flagged
    # where it would decide a pixel's range
    p2 = RayParams(voxel_size=S, mu=MU, z_near=0.64 + 2e-6)
    rng, fl = vol.expected_depth(16, 12, intr, np.eye(4), p2)
    assert (fl[cov] == oracle.RAY_RANGE_AMBIGUOUS).all() and (fl[~cov] == 0).all()


def test_range_contains_every_block_a_ray_meets():
    rs = np.random.default_rng(5)
    keys = np.unique(rs.integers(-4, 5, size=(60, 3)) + np.array([0, 0, 8]), axis=0).astype(np.int32)
    vol = Volume(keys, np.ones((len(keys), 512)))
    R = rot(0.1, -0.07)
    M = pose_from(R, np.array([0.02, -0.03, 0.05]))
    Wd, Hd, f, cx, cy = 40, 30, 30.0, 19.3, 14.8
    p = RayParams(voxel_size=S, mu=MU, z_near=0.3)
    rng, _ = vol.expected_depth(Wd, Hd, intr_of(f, cx, cy), M, p)
    Mi = np.linalg.inv(M)
    O = Mi[:3, 3]
    met = 0
    for j in range(Wd * Hd):
        u, v = j % Wd, j // Wd
        E = Mi[:3, :3] @ np.array([(u - cx) / f, (v - cy) / f, 1.0])  # world per unit depth
        lo_b = keys * 8 * S
        hi_b = lo_b + 8 * S
        with np.errstate(divide="ignore", invalid="ignore"):
            ta = (lo_b - O) / E
            tb = (hi_b - O) / E
        t0 = np.nanmax(np.minimum(ta, tb), axis=1)
        t1 = np.nanmin(np.maximum(ta, tb), axis=1)
        hit = (t1 >= t0) & (t1 >= p.z_near)
        if not hit.any():
            continue
        met += 1
        z_in = np.maximum(t0[hit], p.z_near)
        assert rng[v, u, 0] <= z_in.min() + 1e-9
        assert rng[v, u, 1] >= t1[hit].max() - 1e-9
    assert met > 200


def test_trilinear_read_exact_on_affine_field():
    keys = slab_keys((0, 1), 2)
    a = np.array([0.3, -0.7, 0.11])
    keys, sdf = field_volume(keys, lambda x, y, z: a[0] * x + a[1] * y + a[2] * z + 0.05, 1.0)
    vol = Volume(keys, sdf)
    rs = np.random.default_rng(1)
    for _ in range(200):
        P = rs.uniform([-16, -16, 0], [15, 15, 15])
        got = vol.read(P)
        assert got is not None and abs(got - (a @ P + 0.05)) < 1e-12
    # the last cell before a missing block is unreadable, the one before it readable
    assert vol.read([0.5, 0.5, 15.5]) is None
    assert vol.read([0.5, 0.5, 14.5]) is not None
    assert vol.read([15.5, 0.5, 3.0]) is None


def test_sample_on_block_boundary_is_flagged():
    # head-on slab: every ray's first sample lies on the slab's front face
    D = 8 * 12 * S + 0.5 * 8 * S + 0.0037
    keys, sdf = plane_volume(D)
    vol = Volume(keys, sdf)
    out = vol.raycast(W, H, intr_of(F, CX, CY), np.eye(4), RayParams(voxel_size=S, mu=MU))
    assert (out["flags"] & oracle.RAY_MARCH_AMBIGUOUS).all()
    # a tilted view of the same slab is mostly unflagged
    R = rot(0.21, -0.13)
    out = vol.raycast(W, H, intr_of(F, 31.3, 23.6), pose_from(R, np.zeros(3)),
                      RayParams(voxel_size=S, mu=MU))
    assert (out["flags"] != 0).mean() < 0.1


def test_pixel_subset_matches_full_image():
    D = 8 * 12 * S + 0.5 * 8 * S + 0.0037
    keys, sdf = plane_volume(D)
    vol = Volume(keys, sdf)
    p = RayParams(voxel_size=S, mu=MU)
    full = vol.raycast(W, H, intr_of(F, 31.3, 23.6), np.eye(4), p)
    pix = np.array([0, 5, W * H - 1, 17 * W + 3])
    sub = vol.raycast(W, H, intr_of(F, 31.3, 23.6), np.eye(4), p, pixels=pix)
    assert np.array_equal(sub["points"], full["points"][pix])
    with pytest.raises(ValueError):
        vol.raycast(W, H, intr_of(F, 31.3, 23.6), np.eye(4), p, pixels=np.array([W * H]))
