"""The swap kernels' visibility test, compiled for the host
(tsdf_swap_visibility; no GPU needed), against the oracle's visibility rule
(Section 5): the kernels evaluate five linear functions of the block origin in
FP64 where the oracle projects all eight corners, so the two must agree on
every block the oracle does not flag."""

import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module")
def lib():
    from paper_1410_0925_gb300 import build
    build.build()
    from paper_1410_0925_gb300.tsdf import load_library
    return load_library()


def _pose(rng):
    a = rng.normal(size=3)
    a *= rng.uniform(0, np.pi) / np.linalg.norm(a)
    th = np.linalg.norm(a)
    k = a / th
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    R = np.eye(3) + np.sin(th) * K + (1 - np.cos(th)) * K @ K
    M = np.eye(4)
    M[:3, :3] = R
    M[:3, 3] = rng.uniform(-1.5, 1.5, 3)
    return M


def test_kernel_visibility_matches_the_oracle(lib):
    from paper_1410_0925_gb300 import make_intrinsics, swap_visibility
    rng = np.random.default_rng(5)
    n_checked = n_flagged = n_vis = 0
    for trial in range(24):
        voxel = float(np.float32(rng.choice([0.004, 0.005, 0.01, 0.02])))
        W, H = [(160, 120), (640, 480), (1280, 720)][trial % 3]
        f = float(np.float32(rng.uniform(0.7, 1.3) * W))
        cx, cy = float(np.float32(W / 2 - 0.5)), float(np.float32(H / 2 - 0.5))
        intr = make_intrinsics(f, f, cx, cy, W, H)
        M = _pose(rng)
        margin = float(rng.choice([0.0, 2.0, 16.0, 100.0]))
        max_depth = float(rng.choice([0.0, 0.0, 1.0, 3.0]))
        # blocks anywhere within a few metres, and blocks around points in
        # front of the camera (near the image edges as often as inside)
        reach = int(4.0 / (8 * voxel))
        anywhere = rng.integers(-reach, reach + 1, (200, 3))
        z = rng.uniform(0.05, 5.0, 200)
        q = np.stack([rng.uniform(-0.8, 0.8, 200) * z * W / f,
                      rng.uniform(-0.8, 0.8, 200) * z * H / f, z], -1)
        world = (q - M[:3, 3]) @ M[:3, :3]
        ahead = np.floor(world / (8 * voxel)).astype(np.int64)
        keys = np.concatenate([anywhere, ahead]).astype(np.int16)
        got = swap_visibility(voxel, intr, M, keys, margin, max_depth)
        p = oracle.OracleParams(voxel_size=voxel, mu=4 * voxel, max_weight=100, storage=0)
        for k, g in zip(keys, got):
            vis, amb = oracle.block_visible(p, W, H, (f, f, cx, cy), M, k, margin, max_depth)
            if amb:
                n_flagged += 1
                continue
            assert g == vis, (trial, k.tolist(), g, vis)
            n_checked += 1
            n_vis += vis
    assert n_checked > 9000 and n_flagged < 0.01 * n_checked
    assert 0.2 * n_checked < n_vis < 0.8 * n_checked


def test_kernel_visibility_on_the_edges(lib):
    """Blocks straddling the camera plane, exactly behind it, and a margin
    placed on a block edge from both sides."""
    from paper_1410_0925_gb300 import make_intrinsics, swap_visibility
    intr = make_intrinsics(100.0, 100.0, 80.0, 60.0, 160, 120)
    I4 = np.eye(4)
    inside = np.eye(4)
    inside[:3, 3] = -0.04
    keys = np.array([[0, 0, 12], [0, 0, -14], [11, 0, 12]], np.int16)
    assert swap_visibility(0.01, intr, I4, keys).tolist() == [True, False, False]
    assert swap_visibility(0.01, intr, inside, keys[:1] * 0).tolist() == [True]
    umin = 100 * 0.88 / 1.04 + 80
    assert swap_visibility(0.01, intr, I4, keys[2:], umin - 159.5 + 0.01).tolist() == [True]
    assert swap_visibility(0.01, intr, I4, keys[2:], umin - 159.5 - 0.01).tolist() == [False]
    assert swap_visibility(0.01, intr, I4, keys[:1], 0.0, 0.95).tolist() == [False]
    assert swap_visibility(0.01, intr, I4, keys[:1], 0.0, 0.97).tolist() == [True]


def test_kernel_visibility_rejects_bad_views(lib):
    from paper_1410_0925_gb300 import TsdfError, make_intrinsics, swap_visibility
    intr = make_intrinsics(100.0, 100.0, 80.0, 60.0, 160, 120)
    keys = np.zeros((1, 3), np.int16)
    bad = np.eye(4)
    bad[3, 3] = 2.0
    for args in ((0.01, intr, bad, keys), (0.0, intr, np.eye(4), keys),
                 (0.01, intr, np.eye(4), keys, -1.0), (0.01, intr, np.eye(4), keys, 0.0, np.nan)):
        with pytest.raises(TsdfError):
            swap_visibility(*args)
