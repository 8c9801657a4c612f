"""Pins of the swapping oracle (Section 5): the visibility rule on hand-placed
blocks, lossless round trips, the secondary integration against the running
average it must reproduce, its integer arithmetic on hand-derived voxels, and
the capacity and pool rules against brute force.

Plain CPU tests; each pin is fixed by geometry, arithmetic or an identity,
not by the oracle's own output.
"""

import numpy as np
import pytest

import oracle
from synthdepth import workload_tiny
from synthdepth.configs import make_sequence

BIG = 10 ** 9


def f32(x):
    return float(np.float32(x))


@pytest.fixture(scope="module")
def tiny():
    w = workload_tiny()
    return w, make_sequence(w, colour=True)


def params(w, storage=0, pool=0):
    return oracle.OracleParams(voxel_size=f32(w.voxel_size), mu=f32(w.mu),
                               max_weight=w.max_weight, storage=storage, pool_blocks=pool)


def intr_of(w):
    return tuple(f32(v) for v in (w.fx, w.fy, w.cx, w.cy))


# a view that sees nothing: rotated half a turn about y and moved 100 m back,
# so every point with world z > -100 m has camera z < 0
AWAY = np.array([[-1.0, 0, 0, 0], [0, 1.0, 0, 0], [0, 0, -1.0, -100.0], [0, 0, 0, 1.0]])


def swap_in_all(o, w, seq):
    """Bring every host block back: visible from some pose with a huge margin."""
    for P in seq.poses:
        o.swap_in(w.width, w.height, intr_of(w), P, 1e9, 0.0, BIG)


def fused(w, seq, frames, storage=0, pool=0):
    o = oracle.Oracle(params(w, storage, pool))
    for t in frames:
        o.integrate_rgb(seq.depth[t], seq.colour[t], intr_of(w), seq.poses[t])
    return o


def same_map(a, b):
    ra, rb = a.read(), b.read()
    assert np.array_equal(ra["keys"], rb["keys"])
    assert np.array_equal(ra["w"], rb["w"])
    assert np.array_equal(ra["sdf"], rb["sdf"])
    assert np.array_equal(a.read_colour(), b.read_colour())


# ---------------------------------------------------------------------------
# visibility

P1 = oracle.OracleParams(voxel_size=0.01, mu=0.04, max_weight=100, storage=0)
K1 = (100.0, 100.0, 80.0, 60.0)  # fx, fy, cx, cy of a 160 x 120 view
I4 = np.eye(4)


def vis(key, margin=0.0, max_depth=0.0, pose=I4):
    return oracle.block_visible(P1, 160, 120, K1, pose, key, margin, max_depth)


def test_visibility_hand_placed_blocks():
    # block (0, 0, 12): box [0, .08]^2 x [.96, 1.04] straight ahead
    assert vis((0, 0, 12)) == (True, False)
    # behind the camera
    assert vis((0, 0, -14)) == (False, False)
    # a camera inside block (0, 0, 0): corners on both sides of its plane
    inside = np.eye(4)
    inside[:3, 3] = -0.04
    assert vis((0, 0, 0), pose=inside) == (True, False)
    # block (11, 0, 12): x in [.88, .96], z in [.96, 1.04]; its leftmost
    # projected corner is u = 100 * .88 / 1.04 + 80 = 164.615..., the grown
    # image's right edge is 159.5 + margin
    umin = 100 * 0.88 / 1.04 + 80
    assert vis((11, 0, 12)) == (False, False)
    assert vis((11, 0, 12), margin=5.2) == (True, False)
    assert vis((11, 0, 12), margin=umin - 159.5 - 0.01) == (False, False)
    assert vis((11, 0, 12), margin=umin - 159.5 + 0.01) == (True, False)
    # on the bound itself: flagged
    assert vis((11, 0, 12), margin=umin - 159.5)[1]
    # depth limit: the nearest corner is at z = .96
    assert vis((0, 0, 12), max_depth=0.95) == (False, False)
    assert vis((0, 0, 12), max_depth=0.97) == (True, False)
    assert vis((0, 0, 12), max_depth=0.96)[1]
    # a block touching the camera plane (z in [-.08, 0]) is flagged
    assert vis((0, 0, -1))[1]


def test_visibility_contains_every_projection():
    """A block with some point projecting into the image (z > 0) is visible
    (the corner box holds every projection of the block)."""
    rng = np.random.default_rng(3)
    pose = np.eye(4)
    c, s_ = np.cos(0.3), np.sin(0.3)
    pose[:3, :3] = [[c, 0, s_], [0, 1, 0], [-s_, 0, c]]
    pose[:3, 3] = [0.1, -0.05, 0.2]
    for _ in range(300):
        key = rng.integers(-20, 20, 3)
        pts = (8 * (key + rng.random((64, 3)))) * 0.01
        q = pts @ pose[:3, :3].T + pose[:3, 3]
        front = q[:, 2] > 1e-3
        u = 100 * q[front, 0] / q[front, 2] + 80
        v = 100 * q[front, 1] / q[front, 2] + 60
        inside = ((u > -0.5) & (u < 159.5) & (v > -0.5) & (v < 119.5)).any()
        visible, _ = vis(key, pose=pose)
        if inside:
            assert visible, key


def test_band_blocks_are_visible(tiny):
    """Every block a frame's bands allocate is visible from that frame."""
    w, seq = tiny
    for t in (0, 7):
        o = oracle.Oracle(params(w))
        o.integrate(seq.depth[t], intr_of(w), seq.poses[t])
        for key in o.read()["keys"]:
            visible, amb = oracle.block_visible(params(w), w.width, w.height, intr_of(w),
                                                seq.poses[t], key)
            assert visible or amb, key


# ---------------------------------------------------------------------------
# round trips

def test_round_trip_is_lossless(tiny):
    w, seq = tiny
    a = fused(w, seq, range(10))
    b = fused(w, seq, range(10))
    n = b.num_blocks()
    assert b.swap_out(w.width, w.height, intr_of(w), AWAY, 0.0, 0.0, BIG) == n
    assert b.num_blocks() == 0 and b.num_host_blocks() == n
    host = b.read_host()
    assert (host["bflag"] & oracle.BLOCK_SWAPPED).all()
    swap_in_all(b, w, seq)
    assert b.num_host_blocks() == 0
    same_map(a, b)
    # and fusion goes on identically
    for t in range(10, 20):
        a.integrate_rgb(seq.depth[t], seq.colour[t], intr_of(w), seq.poses[t])
        b.integrate_rgb(seq.depth[t], seq.colour[t], intr_of(w), seq.poses[t])
    same_map(a, b)


@pytest.mark.parametrize("storage", [0, 1, 2])
def test_swap_in_before_integration_loses_nothing(tiny, storage):
    """Swap in what the view sees before fusing, swap out what it does not
    after: every update lands on a device block, so the map equals fusion
    without swapping, bit for bit, and no block needs a merge."""
    w, seq = tiny
    a = oracle.Oracle(params(w, storage))
    b = oracle.Oracle(params(w, storage))
    moved = merged = 0
    for t in range(seq.depth.shape[0]):
        n, m = b.swap_in(w.width, w.height, intr_of(w), seq.poses[t], 0.0, 0.0, BIG)
        moved += n
        merged += m
        a.integrate_rgb(seq.depth[t], seq.colour[t], intr_of(w), seq.poses[t])
        b.integrate_rgb(seq.depth[t], seq.colour[t], intr_of(w), seq.poses[t])
        moved += b.swap_out(w.width, w.height, intr_of(w), seq.poses[t], 0.0, 0.0, BIG)
    assert moved > 1000 and merged == 0
    swap_in_all(b, w, seq)
    same_map(a, b)


# ---------------------------------------------------------------------------
# secondary integration

def test_merge_equals_running_average(tiny):
    """Frames 0-9 fused, everything swapped out, frame 10 fused into fresh
    blocks, then merged: without the weight cap the weighted mean of the two
    running averages is the running average of all eleven frames, so every
    merged block equals fusion without swapping (FP64, float storage)."""
    w, seq = tiny
    s = fused(w, seq, range(10))
    z = fused(w, seq, range(11))
    s.swap_out(w.width, w.height, intr_of(w), AWAY, 0.0, 0.0, BIG)
    s.integrate_rgb(seq.depth[10], seq.colour[10], intr_of(w), seq.poses[10])
    fresh = {tuple(k) for k in s.read()["keys"].tolist()}
    # the fresh blocks are exactly the blocks frame 10's bands meet
    alone = fused(w, seq, [10])
    assert fresh == {tuple(k) for k in alone.read()["keys"].tolist()}
    n, m = s.swap_in(w.width, w.height, intr_of(w), seq.poses[10], 0.0, 0.0, BIG)
    assert m == len(fresh) - len(fresh - {tuple(k) for k in fused(w, seq, range(10)).read()["keys"].tolist()})
    rs, rz = s.read(), z.read()
    zi = {tuple(k): i for i, k in enumerate(rz["keys"].tolist())}
    assert rz["w"].max() < w.max_weight
    checked = 0
    for i, k in enumerate(rs["keys"].tolist()):
        if tuple(k) not in fresh:
            continue
        j = zi[tuple(k)]
        assert np.array_equal(rs["w"][i], rz["w"][j]), k
        assert np.abs(rs["sdf"][i] - rz["sdf"][j]).max() < 1e-12, k
        checked += 1
    assert checked == len(fresh)


def plane_scene(storage, d_a, d_b, rgb_a, rgb_b, pool=0):
    """A 160 x 120 camera at the origin looking down +z (cx = 80, cy = 60, so
    voxel (0, 0, z) projects onto pixel (80, 60) exactly); frame A sees a
    plane at depth d_a, then everything is swapped out, frame B sees a plane
    at d_b, then everything is swapped back in."""
    p = oracle.OracleParams(voxel_size=0.01, mu=0.04, max_weight=100, storage=storage,
                            pool_blocks=pool)
    o = oracle.Oracle(p)
    for d, c in ((d_a, rgb_a), (d_b, rgb_b)):
        depth = np.full((120, 160), d, np.float32)
        col = np.zeros((120, 160, 4), np.uint8)
        col[..., :3] = c
        o.integrate_rgb(depth, col, K1, I4)
        if d == d_a:
            o.swap_out(160, 120, K1, AWAY, 0.0, 0.0, BIG)
    n, m = o.swap_in(160, 120, K1, I4, 0.0, 0.0, BIG)
    assert m > 0
    return o


def voxel_state(o, vox):
    r = o.read()
    key = np.asarray(vox) // 8
    i = np.nonzero((r["keys"] == key).all(1))[0][0]
    lx, ly, lz = np.asarray(vox) - 8 * key
    li = lx + 8 * ly + 64 * lz
    return r["sdf"][i, li], r["w"][i, li], o.read_colour()[i, li]


def test_int16_merge_truncates_toward_zero():
    # voxel (0, 0, 100) sits at camera depth 1.0 on pixel (80, 60). Frame A:
    # eta / mu * 32767 = -3.5 (+- 0.03 from the float32 depth), stored -3;
    # frame B: the plane through the voxel, stored 0. Merge: (-3 + 0) / 2 =
    # -1.5, truncated toward zero: -1 (floor would give -2).
    d_a = np.float32(1.0 - 3.5 * 0.04 / 32767)
    o = plane_scene(1, d_a, np.float32(1.0), (10, 20, 30), (11, 21, 200))
    sdf, wt, rgbw = voxel_state(o, (0, 0, 100))
    assert wt == 2
    assert round(sdf * 32767) == -1
    # colour: per channel (10 + 11) / 2 = 10.5 -> 11, 20.5 -> 21, 115 -> 115
    assert rgbw.tolist() == [11, 21, 115, 2]


def test_float_merge_is_the_weighted_mean():
    # frame A at depth 1.02: f = .02 / .04 = 0.5 at voxel z = 1.0; frame B at
    # depth 1.0: f = 0. Merge (1 * .5 + 1 * 0) / 2 = .25; and a voxel that
    # frame A updated twice is impossible here, so use the weight cap check
    # below for unequal weights.
    o = plane_scene(0, np.float32(1.02), np.float32(1.0), (0, 0, 0), (0, 0, 0))
    sdf, wt, _ = voxel_state(o, (0, 0, 100))
    f_a = (float(np.float32(1.02)) - 1.0) / 0.04
    assert wt == 2 and abs(sdf - 0.5 * f_a) < 1e-12


def test_unequal_weights_and_cap(tiny):
    """Host weight 9 (nine frames), device weight 1: the merged value is
    (9 F_h + F_d) / 10; with maxW = 5 the weight is capped at 5 but the
    average still uses the uncapped sum of the capped stored weights."""
    w, seq = tiny
    for max_w in (100, 5):
        p = oracle.OracleParams(voxel_size=f32(w.voxel_size), mu=f32(w.mu), max_weight=max_w,
                                storage=0)
        s = oracle.Oracle(p)
        h = oracle.Oracle(p)
        d = oracle.Oracle(p)
        for t in range(9):
            s.integrate(seq.depth[t], intr_of(w), seq.poses[t])
            h.integrate(seq.depth[t], intr_of(w), seq.poses[t])
        s.swap_out(w.width, w.height, intr_of(w), AWAY, 0.0, 0.0, BIG)
        s.integrate(seq.depth[9], intr_of(w), seq.poses[9])
        d.integrate(seq.depth[9], intr_of(w), seq.poses[9])
        s.swap_in(w.width, w.height, intr_of(w), seq.poses[9], 0.0, 0.0, BIG)
        rs, rh, rd = s.read(), h.read(), d.read()
        hi = {tuple(k): i for i, k in enumerate(rh["keys"].tolist())}
        di = {tuple(k): i for i, k in enumerate(rd["keys"].tolist())}
        n = 0
        for i, k in enumerate(rs["keys"].tolist()):
            k = tuple(k)
            if k not in hi or k not in di:
                continue
            wh, wd = rh["w"][hi[k]].astype(int), rd["w"][di[k]].astype(int)
            fh, fd = rh["sdf"][hi[k]], rd["sdf"][di[k]]
            both = (wh > 0) & (wd > 0)
            exp = np.where(both, (wh * fh + wd * fd) / np.maximum(wh + wd, 1),
                           np.where(wd > 0, fd, fh))
            expw = np.minimum(wh + wd, max_w)
            assert np.array_equal(rs["w"][i], expw)
            assert np.abs(rs["sdf"][i] - exp).max() < 1e-12
            n += int(both.sum())
        assert n > 1000


# ---------------------------------------------------------------------------
# capacity and pool rules

def test_capacity_takes_smallest_keys(tiny):
    w, seq = tiny
    full = fused(w, seq, range(8))
    part = fused(w, seq, range(8))
    view = seq.poses[15]
    n_all = full.swap_out(w.width, w.height, intr_of(w), view, 0.0, 0.0, BIG)
    assert n_all > 200
    assert part.swap_out(w.width, w.height, intr_of(w), view, 0.0, 0.0, 150) == 150
    moved = sorted(tuple(k) for k in full.read_host()["keys"].tolist())
    assert [tuple(k) for k in part.read_host()["keys"].tolist()] == moved[:150]
    # swap-in: the smallest keys of what an unbounded call brings back
    view_in = seq.poses[0]
    a = full.swap_in(w.width, w.height, intr_of(w), view_in, 0.0, 0.0, BIG)[0]
    before = {tuple(k) for k in part.read_host()["keys"].tolist()}
    assert a > 40
    n = part.swap_in(w.width, w.height, intr_of(w), view_in, 0.0, 0.0, 40)[0]
    after = {tuple(k) for k in part.read_host()["keys"].tolist()}
    back = sorted(before - after)
    # the candidates: host blocks that the unbounded call brought back
    cand = sorted(before & {tuple(k) for k in full.read()["keys"].tolist()})
    assert n == len(back) == min(40, len(cand)) and len(cand) > 0
    assert back == cand[:len(back)]


def test_prefetch_needs_a_full_call_of_free_blocks(tiny):
    w, seq = tiny
    n_blocks = fused(w, seq, range(5)).num_blocks()
    for spare, expect_prefetch in ((100, True), (99, False)):
        o = fused(w, seq, range(5), pool=n_blocks + spare)
        o.swap_out(w.width, w.height, intr_of(w), AWAY, 0.0, 0.0, BIG)
        # all device blocks are free again; the pool has n_blocks + spare
        n, m = o.swap_in(w.width, w.height, intr_of(w), seq.poses[0], 0.0, 0.0,
                         n_blocks + 100)
        assert m == 0
        assert (n > 0) == expect_prefetch


def test_pending_merge_is_not_swapped_out(tiny):
    """A block with a fresh device block and a host copy stays on the device
    until it is merged."""
    w, seq = tiny
    o = fused(w, seq, range(3))
    o.swap_out(w.width, w.height, intr_of(w), AWAY, 0.0, 0.0, BIG)
    host = {tuple(k) for k in o.read_host()["keys"].tolist()}
    o.integrate(seq.depth[3], intr_of(w), seq.poses[3])
    dev = {tuple(k) for k in o.read()["keys"].tolist()}
    pending = dev & host
    assert pending and dev - host
    # only the blocks new in frame 3 (no host copy) leave
    assert o.swap_out(w.width, w.height, intr_of(w), AWAY, 0.0, 0.0, BIG) == len(dev - host)
    assert {tuple(k) for k in o.read()["keys"].tolist()} == pending
