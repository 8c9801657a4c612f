"""Pins of the oracle's colour fusion (the voxel type's clr / w_color of
Section 3.1, averaged like the depth by the integration of Section 4.3).

C1  a constant colour on the closed-form plane: every voxel the depth rule
    updates holds exactly that colour with weight min(frames, maxW); every
    other voxel keeps colour 0, weight 0.
C2  hand-derived averages: two frames of constant colours give
    floor((c1 + c2) / 2 + 1/2) per channel (ties round up); a run of frames
    through the weight cap follows the arithmetic worked out below.
C3  a per-pixel texture: after one frame each updated voxel holds the colour
    of the pixel its centre projects to (nearest pixel), channel by channel.
C4  depth-only frames leave colours alone; colour frames leave depth results
    identical to depth-only fusion.
"""

import numpy as np
import pytest

import oracle
from synthdepth import look_at, make_sequence, workload_tiny

W, H, F, CX, CY = 64, 48, 60.0, 31.5, 23.5
S, MU = 0.01, 0.04
POSE = look_at(np.array([0.31, -0.22, 0.13]), np.array([0.9, 0.35, 1.4]))


def _plane_run(colours, max_weight=100, depth=1.0):
    o = oracle.Oracle(oracle.OracleParams(voxel_size=S, mu=MU, max_weight=max_weight))
    d = np.full((H, W), depth, np.float32)
    for c in colours:
        img = np.empty((H, W, 4), np.uint8)
        img[...] = np.asarray(c, np.uint8)
        o.integrate_rgb(d, img, (F, F, CX, CY), POSE)
    return o.read(), o.read_colour()


def test_c1_constant_colour_on_plane():
    c = (200, 17, 93, 5)
    r, col = _plane_run([c] * 4, max_weight=3)
    upd = r["w"] > 0
    assert upd.sum() > 1000 and (~upd).sum() > 1000
    assert (col[upd][:, :3] == np.array(c[:3], np.uint8)).all()
    assert (col[upd][:, 3] == 3).all()                 # min(4 frames, maxW 3)
    assert (col[~upd] == 0).all()
    assert np.array_equal(col[..., 3], r["w"])         # same voxels, same count


def test_c2_hand_derived_averages():
    # two frames: (10 + 13) / 2 = 11.5 -> 12 (tie up); (255 + 0) / 2 = 127.5
    # -> 128; (7 + 7) / 2 = 7
    r, col = _plane_run([(10, 255, 7, 0), (13, 0, 7, 0)])
    upd = r["w"] == 2
    assert upd.sum() > 1000
    assert (col[upd][:, :3] == np.array([12, 128, 7], np.uint8)).all()
    assert (col[upd][:, 3] == 2).all()
    # maxW = 3, colours 0, 0, 0, 90, 90 in one channel:
    #   w 0 -> 0, w 1 -> 0, w 2 -> 0 (weight now 3 = cap)
    #   (3 * 0 + 90) / 4 = 22.5 -> 23, weight stays 3
    #   (3 * 23 + 90) / 4 = 159 / 4 = 39.75 -> 40
    # and in another channel 250, 250, 250, 1, 1:
    #   (3 * 250 + 1) / 4 = 187.75 -> 188; (3 * 188 + 1) / 4 = 141.25 -> 141
    seq = [(0, 250, 60, 0)] * 3 + [(90, 1, 61, 0)] * 2
    r, col = _plane_run(seq, max_weight=3)
    upd = r["w"] == 3
    assert upd.sum() > 1000
    # third channel: 60 x3, then (3 * 60 + 61) / 4 = 60.25 -> 60, again 60
    assert (col[upd][:, :3] == np.array([40, 141, 60], np.uint8)).all()
    assert (col[upd][:, 3] == 3).all()


def test_c3_texture_lookup_at_nearest_pixel():
    rng = np.random.default_rng(3)
    img = rng.integers(0, 256, size=(H, W, 4), dtype=np.uint8)
    o = oracle.Oracle(oracle.OracleParams(voxel_size=S, mu=MU))
    o.integrate_rgb(np.full((H, W), 1.0, np.float32), img, (F, F, CX, CY), POSE)
    r, col = o.read(), o.read_colour()
    # project every voxel centre by plain geometry
    R = POSE[:3, :3]
    l = np.arange(512)
    local = np.stack([l % 8, (l // 8) % 8, l // 64], axis=1)
    P = (r["keys"][:, None, :] * 8 + local[None]) * S
    cam = P @ R.T + POSE[:3, 3]
    x = F * cam[..., 0] / cam[..., 2] + CX
    y = F * cam[..., 1] / cam[..., 2] + CY
    upd = (r["w"] == 1) & (r["vflag"] == 0)
    assert upd.sum() > 1000
    ix = np.floor(x[upd] + 0.5).astype(int)
    iy = np.floor(y[upd] + 0.5).astype(int)
    assert np.array_equal(col[upd][:, :3], img[iy, ix, :3])


def test_c4_colour_and_depth_are_independent():
    w = workload_tiny()
    seq = make_sequence(w, n_frames=4, colour=True)
    p = oracle.OracleParams(voxel_size=float(np.float32(w.voxel_size)),
                            mu=float(np.float32(w.mu)))
    intr = [float(np.float32(v)) for v in (w.fx, w.fy, w.cx, w.cy)]
    a = oracle.Oracle(p)
    b = oracle.Oracle(p)
    for i in range(4):
        a.integrate(seq.depth[i], intr, seq.poses[i])
        b.integrate_rgb(seq.depth[i], seq.colour[i], intr, seq.poses[i])
    ra, rb = a.read(), b.read()
    for k in ("keys", "sdf", "w", "vflag"):
        assert np.array_equal(ra[k], rb[k])
    assert (a.read_colour() == 0).all()
    cb = b.read_colour()
    assert np.array_equal(cb[..., 3], rb["w"])
    # a depth-only frame afterwards changes depth weights, not colours
    b.integrate(seq.depth[1], intr, seq.poses[1])
    rb2, cb2 = b.read(), b.read_colour()
    before = {tuple(k): i for i, k in enumerate(rb["keys"].tolist())}
    for j, k in enumerate(rb2["keys"].tolist()):
        if tuple(k) in before:
            assert np.array_equal(cb2[j], cb[before[tuple(k)]])
        else:
            assert (cb2[j] == 0).all()
    assert not np.array_equal(rb2["w"][:len(rb["w"])], rb["w"]) or len(rb2["w"]) != len(rb["w"])


def test_colour_input_shape_checked():
    o = oracle.Oracle(oracle.OracleParams(voxel_size=S, mu=MU))
    with pytest.raises(ValueError):
        o.integrate_rgb(np.ones((H, W), np.float32), np.zeros((H, W, 3), np.uint8),
                        (F, F, CX, CY), POSE)
