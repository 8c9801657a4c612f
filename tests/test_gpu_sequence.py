"""Pipelined sequences (tsdf_integrate_frames): frame t + 1's allocation
overlaps frame t's integration on a second stream; the results must equal
frame-by-frame fusion bit for bit, eagerly and inside a CUDA graph."""

import numpy as np
import pytest

from synthdepth import make_sequence, workload_kinect, workload_tiny
from synthdepth.configs import STORAGE_F32, STORAGE_I16

pytestmark = pytest.mark.gpu


def _intr(w):
    from paper_1410_0925_gb300 import make_intrinsics
    return make_intrinsics(w.fx, w.fy, w.cx, w.cy, w.width, w.height)


def _alone(w, depth, poses):
    from paper_1410_0925_gb300 import Scene
    sc = Scene.from_workload(w)
    for i in range(depth.shape[0]):
        sc.integrate(depth[i], _intr(w), poses[i])
    return sc.read_blocks(), sc.stats()


def _same(a, b):
    assert np.array_equal(a.keys, b.keys)
    assert np.array_equal(a.w, b.w)
    assert np.array_equal(a.sdf, b.sdf)


@pytest.mark.parametrize("storage", [STORAGE_F32, STORAGE_I16])
def test_sequence_equals_frame_by_frame(storage):
    import torch
    from paper_1410_0925_gb300 import Scene
    w = workload_tiny(storage=storage)
    seq = make_sequence(w, n_frames=9)
    depth = torch.from_numpy(seq.depth).cuda()
    ref, st = _alone(w, depth, seq.poses)
    sc = Scene.from_workload(w)
    sc.integrate_frames(depth[:4], _intr(w), seq.poses[:4])
    sc.integrate(depth[4], _intr(w), seq.poses[4])      # mixed with single frames
    sc.integrate_frames(depth[5:], _intr(w), seq.poses[5:])
    _same(sc.read_blocks(), ref)
    got = sc.stats()
    for k in ("frames", "allocated_blocks", "total_updated_voxels", "total_visible_blocks",
              "last_updated_voxels"):
        assert got[k] == st[k], k


def test_sequence_in_cuda_graph_kinect_prefix():
    """40 Kinect frames in one captured sequence (reset first), replayed
    twice: equal to frame-by-frame fusion."""
    import torch
    from paper_1410_0925_gb300 import Scene
    w = workload_kinect()
    seq = make_sequence(w, n_frames=40)
    depth = torch.from_numpy(seq.depth).cuda()
    ref, st = _alone(w, depth, seq.poses)
    stream = torch.cuda.Stream()
    sc = Scene.from_workload(w, stream=stream)
    with torch.cuda.stream(stream):
        sc.integrate_frames(depth[:2], _intr(w), seq.poses[:2])  # sizes the buffers
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        sc.reset()
        sc.integrate_frames(depth, _intr(w), seq.poses)
    for _ in range(2):
        with torch.cuda.stream(stream):
            g.replay()
        _same(sc.read_blocks(), ref)
        assert sc.stats()["total_updated_voxels"] == st["total_updated_voxels"]


def test_sequence_of_mixed_image_sizes():
    import torch
    from paper_1410_0925_gb300 import Scene
    a = workload_tiny()
    b = workload_tiny(width=157, height=93, fx=120.0, fy=119.0, cx=77.3, cy=45.9)
    sa, sb = make_sequence(a, n_frames=3), make_sequence(b, n_frames=3)
    frames = [torch.from_numpy(sa.depth[0]).cuda(), torch.from_numpy(sb.depth[1]).cuda(),
              torch.from_numpy(sa.depth[2]).cuda()]
    intrs = [_intr(a), _intr(b), _intr(a)]
    poses = [sa.poses[0], sb.poses[1], sa.poses[2]]
    ref = Scene.from_workload(a)
    for f, i, p in zip(frames, intrs, poses):
        ref.integrate(f, i, p)
    sc = Scene.from_workload(a)
    sc.integrate_frames(frames, intrs, poses)
    _same(sc.read_blocks(), ref.read_blocks())


def test_sequence_from_host_depth_equals_device_depth():
    """tsdf_integrate_frames with depth in pinned host memory (the library
    copies every frame through its staging ring on a copy stream, ahead of
    the allocation stream): equal to the same sequence from device depth,
    over several calls in a row (the ring is reused across calls), with
    mixed host and device frames in one call and with pageable host memory."""
    import torch
    from paper_1410_0925_gb300 import Scene
    w = workload_kinect()
    seq = make_sequence(w, n_frames=12)
    dev = torch.from_numpy(seq.depth).cuda()
    ref = Scene.from_workload(w)
    ref.integrate_frames(dev, _intr(w), seq.poses)
    pinned = torch.from_numpy(seq.depth).pin_memory()
    sc = Scene.from_workload(w)
    sc.integrate_frames(pinned[:5], _intr(w), seq.poses[:5])
    mixed = [dev[5], pinned[6], dev[7]]
    sc.integrate_frames(mixed, _intr(w), seq.poses[5:8])
    sc.integrate_frames(torch.from_numpy(seq.depth[8:]), _intr(w), seq.poses[8:])
    _same(sc.read_blocks(), ref.read_blocks())
    assert sc.stats()["total_updated_voxels"] == ref.stats()["total_updated_voxels"]


def test_batch_from_host_depth_equals_device_depth():
    """A batch whose frames are in pinned host memory (each launch copies them
    into the scenes' staging buffers before its allocation stage), eagerly
    and captured as a multi-frame graph step: equal to the same batch from
    device depth."""
    import torch
    from paper_1410_0925_gb300 import Batch, Scene
    a = workload_tiny()
    b = workload_tiny(width=157, height=93, fx=120.0, fy=119.0, cx=77.3, cy=45.9)
    ws = [a, b]
    seqs = [make_sequence(w, n_frames=4) for w in ws]
    dev = [torch.from_numpy(s.depth).cuda() for s in seqs]
    host = [torch.from_numpy(s.depth).pin_memory() for s in seqs]
    ref = [Scene.from_workload(w) for w in ws]
    rb = Batch(2)
    for i in range(4):
        rb.integrate([(sc, d[i], _intr(w), s.poses[i]) for sc, d, w, s in zip(ref, dev, ws, seqs)])
    stream = torch.cuda.Stream()
    scenes = [Scene.from_workload(w, stream=stream) for w in ws]
    hb = Batch(2, tables=4, stream=stream)
    items = lambda i: [(sc, h[i], _intr(w), s.poses[i])  # noqa: E731
                       for sc, h, w, s in zip(scenes, host, ws, seqs)]
    for i in range(4):
        hb.integrate(items(i))
    for sc, r in zip(scenes, ref):
        _same(sc.read_blocks(), r.read_blocks())
    hb.cursor = 0  # waits for the eager launches' table copies (no waits under capture)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        for sc in scenes:
            sc.reset()
        for i in range(4):
            hb.prepare(items(i))
            hb.launch()
    with torch.cuda.stream(stream):
        g.replay()
    for sc, r in zip(scenes, ref):
        _same(sc.read_blocks(), r.read_blocks())
