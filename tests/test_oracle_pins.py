"""Pins of the FP64 oracle against facts other than itself.

P1  closed form for a fronto-parallel plane (sdf = clamp((D - z)/mu, -1, 1),
    w = min(frames, maxW)), under a general rotated+translated pose, in all
    three storage forms.
P2  translating plane: unit-weight mean before the weight cap, the closed
    form of the exponential moving average after it.
P3  block form == dense-volume form (Section 3.2 vs 3.3) on the tiny workload.
P4  brute-force sampling of every band segment reproduces the block set.
P5  invariants over a whole sequence (weights capped and monotone, sdf in
    [-1, 1], the block set never shrinks).
P6  the single-voxel re-simulation and single-block hit scan agree with the
    full oracle, and contain both outcomes of a planted ambiguity.
"""

import numpy as np
import pytest

import oracle
from synthdepth import look_at, make_sequence, workload_tiny
from synthdepth.configs import room_placement  # noqa: F401  (documented input)


def f32(x):
    return float(np.float32(x))


def _camera_axes(pose):
    """Camera centre and axes from a world->camera pose by geometry:
    the rows of the rotation are the camera axes in world coordinates."""
    R = pose[:3, :3]
    C = -np.linalg.solve(R, pose[:3, 3])
    return C, R[0], R[1], R[2]


def _voxel_positions(keys, s):
    l = np.arange(512)
    local = np.stack([l % 8, (l // 8) % 8, l // 64], axis=1)
    vox = keys[:, None, :] * 8 + local[None, :, :]
    return vox, vox * s


GEN_POSE = look_at(np.array([0.31, -0.22, 0.13]), np.array([0.9, 0.35, 1.4]))


@pytest.mark.parametrize("storage", [oracle.STORAGE_F32, oracle.STORAGE_I16,
                                     oracle.STORAGE_F16])
def test_p1_fronto_parallel_plane(storage):
    W, H, f, D = 64, 48, 60.0, 1.0
    cx, cy = 31.5, 23.5
    s, mu, maxW, n = 0.01, 0.04, 3, 5
    o = oracle.Oracle(oracle.OracleParams(voxel_size=s, mu=mu, max_weight=maxW,
                                          storage=storage))
    depth = np.full((H, W), D, np.float32)
    for _ in range(n):
        o.integrate(depth, (f, f, cx, cy), GEN_POSE)
    r = o.read()
    assert len(r["keys"]) > 50
    C, ax, ay, az = _camera_axes(GEN_POSE)
    _, P = _voxel_positions(r["keys"], s)
    rel = P - C
    z = rel @ az
    x = f * (rel @ ax) / z + cx
    y = f * (rel @ ay) / z + cy
    eta = D - z
    m = 1e-6
    inside = (z > m) & (x > 1 + m) & (x < W - 2 - m) & (y > 1 + m) & (y < H - 2 - m)
    outside = (z < -m) | (x < 1 - m) | (x > W - 2 + m) | (y < 1 - m) | (y > H - 2 + m)
    upd = inside & (eta > -mu + 1e-9)
    skip = outside | (inside & (eta < -mu - 1e-9))
    assert upd.sum() > 1000 and skip.sum() > 1000
    f_ = np.minimum(1.0, eta / mu)
    if storage == oracle.STORAGE_I16:
        want = np.trunc(f_ * 32767.0) / 32767.0
    elif storage == oracle.STORAGE_F16:
        want = f_.astype(np.float16).astype(np.float64)
    else:
        want = f_
    np.testing.assert_allclose(r["sdf"][upd], want[upd], rtol=0, atol=1e-12)
    assert (r["w"][upd] == min(n, maxW)).all()
    assert (r["sdf"][skip] == 1.0).all() and (r["w"][skip] == 0).all()
    # every allocated block's camera-z extent overlaps the band [D-mu, D+mu]
    corners = np.array([[i, j, k] for i in (0, 8) for j in (0, 8) for k in (0, 8)])
    cz = ((r["keys"][:, None, :] * 8 + corners[None]) * s - C) @ az
    assert (cz.min(1) <= D + mu + 1e-9).all() and (cz.max(1) >= D - mu - 1e-9).all()


def test_p2_translating_plane_mean_then_ema():
    W, H, f = 48, 36, 45.0
    cx, cy = 23.5, 17.5
    s, mu, maxW = 0.01, 0.04, 5
    depths = [1.0 + 0.0123 * ((-1) ** t) * (t % 4) - 0.004 * t for t in range(14)]
    o = oracle.Oracle(oracle.OracleParams(voxel_size=s, mu=mu, max_weight=maxW))
    for d in depths:
        o.integrate(np.full((H, W), d, np.float32), (f, f, cx, cy), GEN_POSE)
    r = o.read()
    C, ax, ay, az = _camera_axes(GEN_POSE)
    _, P = _voxel_positions(r["keys"], s)
    rel = P - C
    z = rel @ az
    x = f * (rel @ ax) / z + cx
    y = f * (rel @ ay) / z + cy
    m = 1e-6
    inside = (z > m) & (x > 1 + m) & (x < W - 2 - m) & (y > 1 + m) & (y < H - 2 - m)
    Dt = np.array([float(np.float32(d)) for d in depths])
    checked = 0
    a = maxW / (maxW + 1.0)
    for b in range(len(r["keys"])):
        t0 = r["t_alloc"][b]
        for li in np.nonzero(inside[b])[0][::7]:
            eta = Dt[t0:] - z[b, li]
            if np.any(np.abs(eta + mu) < 1e-9):
                continue
            fs = np.minimum(1.0, eta[eta >= -mu] / mu)
            k = len(fs)
            if k == 0:
                assert r["w"][b, li] == 0 and r["sdf"][b, li] == 1.0
                continue
            if k <= maxW:
                want = fs.mean()
            else:
                head = fs[:maxW].mean()
                tail = fs[maxW:]
                j = np.arange(len(tail))
                want = a ** len(tail) * head + (1 - a) * np.sum(a ** (len(tail) - 1 - j) * tail)
            assert r["w"][b, li] == min(k, maxW)
            assert abs(r["sdf"][b, li] - want) < 1e-12
            checked += 1
    assert checked > 500


@pytest.fixture(scope="module")
def tiny_run():
    w = workload_tiny()
    seq = make_sequence(w)
    p = oracle.OracleParams(voxel_size=f32(w.voxel_size), mu=f32(w.mu),
                            max_weight=w.max_weight)
    intr = tuple(f32(v) for v in (w.fx, w.fy, w.cx, w.cy))
    o = oracle.Oracle(p)
    snaps = []
    for i in range(seq.depth.shape[0]):
        o.integrate(seq.depth[i], intr, seq.poses[i])
        if i in (0, 5, 12, 19):
            snaps.append((i, o.read()))
    return dict(w=w, seq=seq, p=p, intr=intr, res=o.read(), snaps=snaps,
                ghosts=o.ghosts())


def test_p3_block_form_equals_dense_volume(tiny_run):
    res, seq, p, intr = tiny_run["res"], tiny_run["seq"], tiny_run["p"], tiny_run["intr"]
    kmin = res["keys"].min(0) - 1
    kmax = res["keys"].max(0) + 1
    origin = 8 * kmin
    size = 8 * (kmax - kmin + 1)
    d = oracle.DenseOracle(p, origin, size)
    for i in range(seq.depth.shape[0]):
        assert d.integrate(seq.depth[i], intr, seq.poses[i]) == 0
    sdf, w = d.read()
    vox, _ = _voxel_positions(res["keys"], 1.0)
    idx = vox.astype(np.int64) - origin
    ds = sdf[idx[..., 2], idx[..., 1], idx[..., 0]]
    dw = w[idx[..., 2], idx[..., 1], idx[..., 0]]
    assert np.array_equal(ds, res["sdf"])
    assert np.array_equal(dw, res["w"])
    mask = np.zeros(w.shape, bool)
    mask[idx[..., 2], idx[..., 1], idx[..., 0]] = True
    assert (w[~mask] == 0).all() and (sdf[~mask] == 1.0).all()


def _point_box_distance(pts, lo, hi):
    d = np.maximum(np.maximum(lo - pts, 0.0), pts - hi)
    return np.sqrt((d * d).sum(-1))


def test_p4_band_blocks_by_sampling():
    w = workload_tiny(width=40, height=30, fx=131.25 / 4, fy=131.25 / 4,
                      cx=19.5, cy=14.5)
    seq = make_sequence(w, n_frames=3)
    s, mu = f32(w.voxel_size), f32(w.mu)
    intr = tuple(f32(v) for v in (w.fx, w.fy, w.cx, w.cy))
    for t in range(3):
        o = oracle.Oracle(oracle.OracleParams(voxel_size=s, mu=mu))
        o.integrate(seq.depth[t], intr, seq.poses[t])
        A = {tuple(k) for k in o.read()["keys"]}
        Minv = np.linalg.inv(seq.poses[t])
        H, W = seq.depth[t].shape
        v, u = np.mgrid[0:H, 0:W]
        d = seq.depth[t].astype(np.float64)
        ok = d > 0
        rays = np.stack([(u - intr[2]) / intr[0], (v - intr[3]) / intr[1],
                         np.ones_like(d)], -1)[ok]
        dd = d[ok]
        ns = 1001
        sig = dd[:, None] - mu + (2 * mu) * np.linspace(0, 1, ns)[None, :]
        q = rays[:, None, :] * sig[..., None]
        pts = q @ Minv[:3, :3].T + Minv[:3, 3]
        pts = pts.reshape(-1, 3)
        S = {tuple(k) for k in np.unique(np.floor(pts / (8 * s)).astype(np.int64), axis=0)}
        assert S <= A, "a sampled band point lies in an unallocated block"
        missing = A - S
        # the segment's spacing between samples bounds how far a block that
        # the sampling missed can be from the nearest sample
        h = (2 * mu * np.linalg.norm(rays, axis=1).max() * 1.0001) / (ns - 1)
        for k in missing:
            lo = np.array(k) * 8 * s
            dist = _point_box_distance(pts, lo, lo + 8 * s).min()
            assert dist <= h, (k, dist, h)
        assert len(missing) < 0.05 * len(A)


def test_p5_invariants(tiny_run):
    w, snaps = tiny_run["w"], tiny_run["snaps"]
    prev = None
    for i, r in snaps:
        assert (r["w"] <= w.max_weight).all()
        assert (r["w"] <= i + 1).all()
        assert (r["sdf"] >= -1.0).all() and (r["sdf"] <= 1.0).all()
        assert (r["sdf"][r["w"] == 0] == 1.0).all()
        assert (r["t_alloc"] <= i).all()
        keys = {tuple(k) for k in r["keys"]}
        if prev is not None:
            pkeys, pr = prev
            assert pkeys <= keys, "a block disappeared"
            # weights never decrease below the cap
            idx = {tuple(k): j for j, k in enumerate(r["keys"])}
            rows = [idx[tuple(k)] for k in pr["keys"]]
            assert (r["w"][rows] >= pr["w"]).all()
        prev = (keys, r)
    # canonical order: strictly increasing (x, y, z)
    k = snaps[-1][1]["keys"]
    order = np.lexsort((k[:, 2], k[:, 1], k[:, 0]))
    assert np.array_equal(order, np.arange(len(k)))


def test_p6_resimulation_agrees_with_full_oracle(tiny_run):
    res, seq, p, intr = tiny_run["res"], tiny_run["seq"], tiny_run["p"], tiny_run["intr"]
    rng = np.random.default_rng(3)
    blocks = rng.choice(len(res["keys"]), 24, replace=False)
    for b in blocks:
        key = res["keys"][b]
        hits = oracle.block_hit_frames(key, seq.depth, intr, seq.poses, p)
        exact = np.nonzero(hits & oracle.HIT_EXACT)[0]
        assert exact[0] == res["t_alloc"][b]
        for li in rng.choice(512, 12, replace=False):
            vox = key * 8 + np.array([li % 8, (li // 8) % 8, li // 64])
            c = oracle.voxel_candidates(vox, seq.depth, intr, seq.poses, p, hits)
            assert c is not None
            cs, cw = c
            if res["vflag"][b, li] == 0 and res["bflag"][b] == 0:
                assert len(cs) == 1
                assert cs[0] == res["sdf"][b, li] and cw[0] == res["w"][b, li]
            else:
                assert any(cs[j] == res["sdf"][b, li] and cw[j] == res["w"][b, li]
                           for j in range(len(cs)))
    # ghosts never have an exact hit
    for key in tiny_run["ghosts"][:10]:
        hits = oracle.block_hit_frames(key, seq.depth, intr, seq.poses, p)
        assert not (hits & oracle.HIT_EXACT).any()


def test_p6_planted_rounding_ambiguity_gives_both_outcomes():
    """Voxel (0,0,64) projects to x = cx = 4.5 exactly, so (int)(x + 0.5)
    sits on the boundary between columns 4 and 5; the re-simulation must
    report both the column-5 outcome (the FP64 choice) and the column-4 one."""
    s, mu = 0.015625, 0.0625
    p = oracle.OracleParams(voxel_size=s, mu=mu)
    depth = np.full((1, 10, 10), 1.03125, np.float32)
    depth[0, :, 4] = 1.125
    intr = (100.0, 100.0, 4.5, 4.3)
    poses = np.eye(4)[None]
    o = oracle.Oracle(p)
    o.integrate(depth[0], intr, poses[0])
    r = o.read()
    b = np.nonzero((r["keys"] == [0, 0, 8]).all(1))[0][0]
    assert r["vflag"][b, 0] == 1
    assert r["sdf"][b, 0] == 0.5 and r["w"][b, 0] == 1
    hits = oracle.block_hit_frames([0, 0, 8], depth, intr, poses, p)
    cs, cw = oracle.voxel_candidates([0, 0, 64], depth, intr, poses, p, hits)
    got = sorted(zip(cs.tolist(), cw.tolist()))
    assert got == [(0.5, 1), (1.0, 1)]
