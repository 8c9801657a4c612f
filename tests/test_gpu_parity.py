"""GPU parity: the CUDA fusion path (through the C ABI) against the FP64 oracle
on the same seeded inputs. See tests/parity.py for the comparison rules."""

import numpy as np
import pytest

from parity import (TOL, compare, flag_bound, run_gpu, run_oracle, oracle_params,
                    oracle_intr)
from synthdepth import make_sequence, workload_kinect, workload_tiny
from synthdepth.configs import STORAGE_F16, STORAGE_F32, STORAGE_I16

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny_seq():
    return make_sequence(workload_tiny())


@pytest.mark.parametrize("storage", [STORAGE_F32, STORAGE_I16, STORAGE_F16])
def test_tiny_sequence_matches_oracle(tiny_seq, storage):
    w = workload_tiny(storage=storage)
    orc = run_oracle(w, tiny_seq)
    scene, blocks, stats, status = run_gpu(w, tiny_seq)
    assert status == 0
    rep = compare(blocks, orc, tiny_seq, w, storage)   # every flagged voxel re-simulated
    print(rep)
    assert rep["flagged_checked"] == rep["flagged_voxels"]
    assert rep["flagged_fraction"] <= flag_bound(20)
    assert rep["ghosts_on_gpu"] <= 0.01 * rep["gpu_blocks"]
    assert rep["unresolved"] == 0
    assert stats["frames"] == 20 and stats["allocated_blocks"] == len(blocks.keys)
    assert stats["total_updated_voxels"] > 0


def test_kinect_frames_full_resolution():
    """640x480, 5 mm, noisy, first 6 frames: several thousand blocks, tiles
    of the allocation grid with a ragged right column of the 16x16 tiling."""
    w = workload_kinect()
    seq = make_sequence(w, n_frames=6)
    orc = run_oracle(w, seq)
    scene, blocks, stats, status = run_gpu(w, seq)
    assert status == 0
    rep = compare(blocks, orc, seq, w, STORAGE_F32)
    print(rep)
    assert rep["oracle_blocks"] > 5000
    assert rep["flagged_checked"] == rep["flagged_voxels"]
    assert rep["flagged_fraction"] <= flag_bound(6)
    assert rep["ghosts_on_gpu"] <= 0.01 * rep["gpu_blocks"]
    assert rep["unresolved"] == 0


def test_kinect_120_frames_element_by_element():
    """640x480, 5 mm, noisy, the first 120 frames of the benchmark's
    sequence, so that voxels reach the weight cap (100): every voxel of every
    block compared (weights bit-exact and sdf within 1e-5 on the strict set),
    a 3000-voxel sample of the flagged ones against the re-simulation."""
    w = workload_kinect()
    seq = make_sequence(w, n_frames=120)
    orc = run_oracle(w, seq)
    scene, blocks, stats, status = run_gpu(w, seq)
    assert status == 0
    rep = compare(blocks, orc, seq, w, STORAGE_F32, max_candidates=3000)
    print(rep)
    assert rep["max_weight"] == w.max_weight
    assert rep["flagged_fraction"] <= flag_bound(120)
    assert rep["strict_voxels"] > 0.8 * 512 * rep["oracle_blocks"]
    assert rep["ghosts_on_gpu"] <= 0.01 * rep["gpu_blocks"]
    assert rep["unresolved"] == 0


def test_ragged_image_and_odd_intrinsics():
    w = workload_tiny(width=157, height=93, fx=120.0, fy=119.0, cx=77.3, cy=45.9)
    seq = make_sequence(w, n_frames=5)
    orc = run_oracle(w, seq)
    scene, blocks, stats, status = run_gpu(w, seq)
    assert status == 0
    rep = compare(blocks, orc, seq, w, STORAGE_F32)
    print(rep)
    assert rep["oracle_blocks"] > 500


@pytest.mark.parametrize("storage", [STORAGE_F32, STORAGE_I16, STORAGE_F16])
def test_large_image_depth_max_pyramid_in_global_memory(storage):
    """2000x1500 images: the depth-max pyramid (15,479 cells over three
    levels) exceeds the integration kernel's shared-memory copy, so its block
    selection reads the pyramid from global memory; the result must still
    match the oracle."""
    w = workload_tiny(width=2000, height=1500, fx=1640.625, fy=1640.625, cx=999.5, cy=749.5,
                      storage=storage)
    seq = make_sequence(w, n_frames=3)
    orc = run_oracle(w, seq)
    scene, blocks, stats, status = run_gpu(w, seq)
    assert status == 0
    rep = compare(blocks, orc, seq, w, storage, max_candidates=3000)
    print(rep)
    assert rep["oracle_blocks"] > 1000
    assert rep["flagged_fraction"] <= flag_bound(3)
    assert rep["unresolved"] == 0


def test_tiny_hash_table_equals_large_one(tiny_seq):
    """16 buckets of 2 entries force nearly every block into the excess
    chains; the canonical result must be bit-identical, and every block must
    be retrievable through bucket + chain (Section 3.3 retrieval)."""
    w = workload_tiny()
    _, big, _, st_big = run_gpu(w, tiny_seq)
    scene, small, stats, st_small = run_gpu(w, tiny_seq, hash_buckets_log2=4,
                                            excess_entries=1 << 13)
    assert st_big == 0 and st_small == 0
    assert stats["excess_used"] > 0.9 * len(small.keys)
    assert np.array_equal(big.keys, small.keys)
    assert np.array_equal(big.w, small.w)
    assert np.array_equal(big.sdf, small.sdf)
    ptrs = scene.lookup(small.keys)
    assert (ptrs >= 0).all() and len(np.unique(ptrs)) == len(ptrs)
    absent = small.keys.astype(np.int32) + np.array([0, 0, 20000])
    absent = absent[np.abs(absent[:, 2]) < 32767].astype(np.int16)
    assert (scene.lookup(absent) == -1).all()


def test_runs_are_bit_identical(tiny_seq):
    w = workload_tiny()
    outs = [run_gpu(w, tiny_seq)[1] for _ in range(3)]
    for o in outs[1:]:
        assert np.array_equal(o.keys, outs[0].keys)
        assert np.array_equal(o.w, outs[0].w)
        assert np.array_equal(o.sdf, outs[0].sdf)


def test_empty_and_invalid_depth():
    import torch
    from paper_1410_0925_gb300 import Scene, make_intrinsics
    w = workload_tiny()
    scene = Scene.from_workload(w)
    intr = make_intrinsics(w.fx, w.fy, w.cx, w.cy, w.width, w.height)
    pose = np.eye(4)
    for val in (0.0, float("nan"), float("inf"), -1.0):
        d = torch.full((w.height, w.width), val, dtype=torch.float32, device="cuda")
        scene.integrate(d, intr, pose)
    st = scene.stats()
    assert st["allocated_blocks"] == 0 and st["total_updated_voxels"] == 0
    assert st["frames"] == 4
    blocks = scene.read_blocks()
    assert len(blocks.keys) == 0


def test_invalid_arguments_rejected():
    import torch
    from paper_1410_0925_gb300 import Scene, TsdfError, make_intrinsics
    with pytest.raises(TsdfError):
        Scene(voxel_size=-1.0, mu=0.02)
    with pytest.raises(TsdfError):
        Scene(voxel_size=0.01, mu=0.04, max_weight=300)
    scene = Scene(voxel_size=0.01, mu=0.04, hash_buckets_log2=10, excess_entries=64,
                  pool_blocks=128)
    d = torch.ones((10, 10), dtype=torch.float32, device="cuda")
    bad_pose = np.eye(4)
    bad_pose[3, 0] = 1.0
    with pytest.raises(TsdfError):
        scene.integrate(d, make_intrinsics(10, 10, 5, 5, 10, 10), bad_pose)
    with pytest.raises(TsdfError):
        scene.integrate(d, make_intrinsics(10, 10, 5, 5, 2, 10), np.eye(4))
    # loading a weight above the scene's cap (integration never makes one)
    from paper_1410_0925_gb300 import Blocks
    keys = np.zeros((1, 3), np.int16)
    sdf = np.ones((1, 512), np.float32)
    w = np.zeros((1, 512), np.uint8)
    w[0, 7] = 101
    with pytest.raises(TsdfError):
        scene.load_blocks(Blocks(keys, sdf, w))
    w[0, 7] = 100
    scene.load_blocks(Blocks(keys, sdf, w))
    assert scene.num_blocks() == 1


def test_pool_exhaustion_keeps_smallest_keys(tiny_seq):
    """With a 300-block pool the first frame needs more blocks than exist;
    the smallest keys (canonical order) are allocated, the call reports
    POOL_EXHAUSTED, and integration of the allocated blocks continues."""
    from paper_1410_0925_gb300.tsdf import TSDF_ERR_POOL_EXHAUSTED
    w = workload_tiny(pool_blocks=300)
    seq = make_sequence(w, n_frames=3)
    orc = run_oracle(w, seq, pool_blocks=300)
    assert orc["statuses"][0] == 1
    scene, blocks, stats, status = run_gpu(w, seq)
    assert status == TSDF_ERR_POOL_EXHAUSTED
    assert len(blocks.keys) == 300
    assert np.array_equal(blocks.keys.astype(np.int32), orc["res"]["keys"])
    rep = compare(blocks, orc, seq, w, STORAGE_F32)
    assert rep["oracle_blocks"] == 300
    # the scene stays usable and the status was cleared by reporting it
    scene.sync()


def test_excess_exhaustion_reported_and_scene_usable(tiny_seq):
    from paper_1410_0925_gb300.tsdf import TSDF_ERR_EXCESS_EXHAUSTED
    w = workload_tiny()
    scene, blocks, stats, status = run_gpu(w, tiny_seq, hash_buckets_log2=4,
                                           excess_entries=64)
    assert status == TSDF_ERR_EXCESS_EXHAUSTED
    assert stats["excess_used"] == 64
    assert len(blocks.keys) == 32 + 64          # every bucket entry + excess entry
    orc = run_oracle(w, tiny_seq)
    assert {tuple(k) for k in blocks.keys.tolist()} <= {tuple(k) for k in orc["res"]["keys"].tolist()}
    assert (scene.lookup(blocks.keys) >= 0).all()
    scene.sync()


def test_resume_from_readback_equals_uninterrupted(tiny_seq):
    import torch
    from paper_1410_0925_gb300 import Scene, make_intrinsics
    for storage in (STORAGE_F32, STORAGE_I16):
        w = workload_tiny(storage=storage)
        intr = make_intrinsics(w.fx, w.fy, w.cx, w.cy, w.width, w.height)
        depth = torch.from_numpy(tiny_seq.depth).cuda()
        full = Scene.from_workload(w)
        for i in range(20):
            full.integrate(depth[i], intr, tiny_seq.poses[i])
        ref = full.read_blocks()
        first = Scene.from_workload(w)
        for i in range(10):
            first.integrate(depth[i], intr, tiny_seq.poses[i])
        snap = first.read_blocks()
        resumed = Scene.from_workload(w)
        resumed.load_blocks(snap)
        again = resumed.read_blocks()
        assert np.array_equal(again.keys, snap.keys) and np.array_equal(again.sdf, snap.sdf)
        for i in range(10, 20):
            resumed.integrate(depth[i], intr, tiny_seq.poses[i])
        got = resumed.read_blocks()
        assert np.array_equal(got.keys, ref.keys)
        assert np.array_equal(got.w, ref.w)
        assert np.array_equal(got.sdf, ref.sdf)


def test_host_depth_path_equals_device_path(tiny_seq):
    """Host (pinned) depth, device depth, and a scene that switches from one
    to the other between frames all give the same result."""
    from paper_1410_0925_gb300 import Scene, make_intrinsics
    import torch
    w = workload_tiny()
    intr = make_intrinsics(w.fx, w.fy, w.cx, w.cy, w.width, w.height)
    a = Scene.from_workload(w)
    b = Scene.from_workload(w)
    c = Scene.from_workload(w)
    dev = torch.from_numpy(tiny_seq.depth).cuda()
    pinned = torch.from_numpy(tiny_seq.depth).pin_memory()
    for i in range(8):
        a.integrate(dev[i], intr, tiny_seq.poses[i])
        b.integrate(pinned[i], intr, tiny_seq.poses[i])
        c.integrate(dev[i] if i < 4 else pinned[i], intr, tiny_seq.poses[i])
    ra, rb, rc = a.read_blocks(), b.read_blocks(), c.read_blocks()
    for r in (rb, rc):
        assert np.array_equal(ra.keys, r.keys) and np.array_equal(ra.sdf, r.sdf)
        assert np.array_equal(ra.w, r.w)


def test_kinect_full_sequence_sampled():
    """The benchmark's workload (640x480, 5 mm, 300 frames) in the bench's
    launch configuration: global invariants on every voxel, and sampled
    blocks checked voxel by voxel against the oracle's single-voxel
    re-simulation over all 300 frames."""
    import oracle
    w = workload_kinect()
    seq = make_sequence(w)
    scene, blocks, stats, status = run_gpu(w, seq)
    assert status == 0
    vals = blocks.sdf_values()
    assert (blocks.w <= w.max_weight).all()
    assert (vals >= -1.0).all() and (vals <= 1.0).all()
    assert (vals[blocks.w == 0] == 1.0).all()
    assert stats["allocated_blocks"] == len(blocks.keys) > 20000
    p = oracle_params(w)
    intr = oracle_intr(w)
    rng = np.random.default_rng(11)
    rows = rng.choice(len(blocks.keys), 24, replace=False)
    checked = 0
    for r in rows:
        key = blocks.keys[r].astype(np.int32)
        hits = oracle.block_hit_frames(key, seq.depth, intr, seq.poses, p)
        assert hits.any(), f"GPU block {key.tolist()} is met by no band segment"
        for li in rng.choice(512, 24, replace=False):
            vox = key * 8 + np.array([li % 8, (li // 8) % 8, li // 64])
            c = oracle.voxel_candidates(vox, seq.depth, intr, seq.poses, p, hits, max_out=256)
            if c is None:
                continue
            cs, cw = c
            gs, gw = vals[r, li], blocks.w[r, li]
            assert any(cw[i] == gw and abs(cs[i] - gs) <= TOL[STORAGE_F32] for i in range(len(cs))), \
                (vox.tolist(), gs, gw, list(zip(cs.tolist(), cw.tolist())))
            checked += 1
    assert checked > 0.9 * 24 * 24


def test_stage_timing_eager_and_captured(tiny_seq):
    """Stage timing works for eagerly launched frames and inside a captured
    CUDA graph, and reports increasing stage boundaries."""
    import torch
    from paper_1410_0925_gb300 import Scene, make_intrinsics
    w = workload_tiny()
    intr = make_intrinsics(w.fx, w.fy, w.cx, w.cy, w.width, w.height)
    depth = torch.from_numpy(tiny_seq.depth).cuda()
    stream = torch.cuda.Stream()
    scene = Scene.from_workload(w, stream=stream)
    for only in (False, True):
        scene.timing_begin(4, only)
        for i in range(4):
            scene.integrate(depth[i], intr, tiny_seq.poses[i])
        t = scene.timing_read()
        assert t.shape == (4, 3)
        cols = [1, 2] if only else [0, 1, 2]
        sub = t[:, cols]
        assert np.isfinite(sub).all() and (np.diff(sub, axis=1) >= 0).all()
        scene.timing_end()
    scene.integrate(depth[4], intr, tiny_seq.poses[4])  # sizes buffers before capture
    scene.timing_begin(3, False)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        for i in range(5, 8):
            scene.integrate(depth[i], intr, tiny_seq.poses[i])
    with torch.cuda.stream(stream):
        g.replay()
    t = scene.timing_read()
    assert t.shape == (3, 3) and np.isfinite(t).all() and (np.diff(t.reshape(-1)) >= 0).all()
    scene.timing_end()
