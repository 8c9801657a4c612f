"""Batched step: many independent scenes of uneven image sizes, voxel sizes,
pools and storage forms per launch. Each scene's result inside the batch must
be bit-identical to fusing it alone with tsdf_integrate (same kernels' rule,
same decisions), eagerly, under CUDA-graph capture and replay, and whatever
launch shapes the autotuner picks."""

import numpy as np
import pytest

from synthdepth import make_sequence, workload_tiny
from synthdepth.configs import STORAGE_F16, STORAGE_F32, STORAGE_I16

pytestmark = pytest.mark.gpu

N_FRAMES = 6


def _workloads():
    return [
        workload_tiny(),
        workload_tiny(name="b1", width=157, height=93, fx=120.0, fy=119.0, cx=77.3, cy=45.9,
                      voxel_size=0.015, mu=0.06, storage=STORAGE_I16, seed=11),
        workload_tiny(name="b2", width=320, height=240, fx=262.5, fy=262.5, cx=159.5, cy=119.5,
                      voxel_size=0.01, mu=0.04, storage=STORAGE_F16, seed=12, pool_blocks=1 << 15,
                      hash_buckets_log2=15),
        workload_tiny(name="b3", voxel_size=0.025, mu=0.1, seed=13, hash_buckets_log2=6,
                      excess_entries=1 << 13),
        workload_tiny(name="b4", width=64, height=48, fx=52.5, fy=52.5, cx=31.5, cy=23.5,
                      seed=14, storage=STORAGE_I16),
    ]


@pytest.fixture(scope="module")
def data():
    import torch
    ws = _workloads()
    seqs = [make_sequence(w, n_frames=N_FRAMES) for w in ws]
    depth = [torch.from_numpy(s.depth).cuda() for s in seqs]
    return ws, seqs, depth


def _intr(w):
    from paper_1410_0925_gb300 import make_intrinsics
    return make_intrinsics(w.fx, w.fy, w.cx, w.cy, w.width, w.height)


def _alone(ws, seqs, depth):
    from paper_1410_0925_gb300 import Scene
    out = []
    for w, s, d in zip(ws, seqs, depth):
        sc = Scene.from_workload(w)
        for i in range(N_FRAMES):
            sc.integrate(d[i], _intr(w), s.poses[i])
        out.append((sc.read_blocks(), sc.stats()))
    return out


def _same(a, b):
    assert np.array_equal(a.keys, b.keys)
    assert np.array_equal(a.w, b.w)
    assert np.array_equal(a.sdf, b.sdf)


def test_batch_equals_scenes_alone(data):
    import torch
    from paper_1410_0925_gb300 import Batch, Scene
    ws, seqs, depth = data
    ref = _alone(ws, seqs, depth)
    stream = torch.cuda.Stream()
    batch = Batch(8, stream=stream)
    scenes = [Scene.from_workload(w) for w in ws]
    for i in range(N_FRAMES):
        batch.integrate([(sc, d[i], _intr(w), s.poses[i])
                         for sc, d, w, s in zip(scenes, depth, ws, seqs)])
    for sc, (rb, st) in zip(scenes, ref):
        got = sc.read_blocks()
        _same(got, rb)
        gst = sc.stats()
        assert gst["frames"] == N_FRAMES
        assert gst["total_updated_voxels"] == st["total_updated_voxels"]
        assert gst["allocated_blocks"] == st["allocated_blocks"]
    assert batch.kernel_launches() > 0


def test_batch_in_cuda_graph_with_new_frames(data):
    import torch
    from paper_1410_0925_gb300 import Batch, Scene
    ws, seqs, depth = data
    ref = _alone(ws, seqs, depth)
    stream = torch.cuda.Stream()
    batch = Batch(8, stream=stream)
    scenes = [Scene.from_workload(w) for w in ws]
    items = lambda i: [(sc, d[i], _intr(w), s.poses[i])  # noqa: E731
                       for sc, d, w, s in zip(scenes, depth, ws, seqs)]
    batch.integrate(items(0))       # sizes every scene's buffers, eagerly
    stream.synchronize()
    batch.prepare(items(1))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        batch.launch()
    # capture does not execute: frame 1 runs at the first replay
    with torch.cuda.stream(stream):
        g.replay()
    for i in range(2, N_FRAMES):
        stream.synchronize()
        batch.prepare(items(i))
        with torch.cuda.stream(stream):
            g.replay()
    for sc, (rb, _) in zip(scenes, ref):
        _same(sc.read_blocks(), rb)


def test_multi_frame_step_in_one_graph(data):
    """A whole step (reset every scene, then all frames, one table per
    frame) captured once and replayed twice gives the per-scene results."""
    import torch
    from paper_1410_0925_gb300 import Batch, Scene
    ws, seqs, depth = data
    ref = _alone(ws, seqs, depth)
    stream = torch.cuda.Stream()
    batch = Batch(8, tables=N_FRAMES, stream=stream)
    scenes = [Scene.from_workload(w, stream=stream) for w in ws]
    items = lambda i: [(sc, d[i], _intr(w), s.poses[i])  # noqa: E731
                       for sc, d, w, s in zip(scenes, depth, ws, seqs)]
    batch.integrate(items(0))       # sizes every scene's buffers, eagerly
    stream.synchronize()
    assert batch.cursor == 1 % N_FRAMES
    batch.cursor = 0
    batch.timing_begin(N_FRAMES)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        for sc in scenes:
            sc.reset()
        for i in range(N_FRAMES):
            batch.prepare(items(i))
            batch.launch()
    assert batch.cursor == 0
    for _ in range(2):
        with torch.cuda.stream(stream):
            g.replay()
        t = batch.timing_read()            # stage boundaries of every launch
        assert t.shape == (N_FRAMES, 3)
        assert np.isfinite(t).all() and (np.diff(t.reshape(-1)) >= 0).all()
        for sc, (rb, st) in zip(scenes, ref):
            _same(sc.read_blocks(), rb)
            assert sc.stats()["total_updated_voxels"] == st["total_updated_voxels"]
    batch.timing_end()


def test_autotuned_batch_gives_the_same_result(data):
    import torch
    from paper_1410_0925_gb300 import Batch, Scene
    ws, seqs, depth = data
    ref = _alone(ws, seqs, depth)
    stream = torch.cuda.Stream()
    # tune on scratch scenes, then run the real ones with the chosen config
    scratch = [Scene.from_workload(w) for w in ws]
    tuner = Batch(8, stream=stream)
    tuner.prepare([(sc, d[0], _intr(w), s.poses[0])
                   for sc, d, w, s in zip(scratch, depth, ws, seqs)])
    best, ms = tuner.autotune(steps=2)
    assert best["integrate_kernel"] in ("staged", "general") and ms > 0
    assert best["alloc_tile"] in ("16x16", "16x8", "32x8")
    assert 1 <= best["integrate_ctas_per_sm"] <= 8
    batch = Batch(8, stream=stream)
    batch.set_config(**best)
    scenes = [Scene.from_workload(w) for w in ws]
    for i in range(N_FRAMES):
        batch.integrate([(sc, d[i], _intr(w), s.poses[i])
                         for sc, d, w, s in zip(scenes, depth, ws, seqs)])
    for sc, (rb, _) in zip(scenes, ref):
        _same(sc.read_blocks(), rb)


def test_batch_rejects_bad_input(data):
    import torch
    from paper_1410_0925_gb300 import Batch, Scene, TsdfError
    ws, seqs, depth = data
    sc = Scene.from_workload(ws[0])
    batch = Batch(2)
    with pytest.raises(TsdfError):
        batch.launch()                             # nothing prepared
    with pytest.raises(TsdfError):
        Batch(1024, tables=2048)                   # more than 2^20 slots
    item = (sc, depth[0][0], _intr(ws[0]), seqs[0].poses[0])
    with pytest.raises(TsdfError):
        batch.integrate([item, item])              # the same scene twice
    other = [Scene.from_workload(ws[0]) for _ in range(3)]
    with pytest.raises(TsdfError):
        batch.integrate([(o, depth[0][0], _intr(ws[0]), seqs[0].poses[0]) for o in other])
    with pytest.raises(ValueError):
        batch.integrate([(sc, depth[0][0].double(), _intr(ws[0]), seqs[0].poses[0])])


def test_pipelined_batch_equals_scenes_alone(data):
    """Pipelined launches (launch k + 1's allocation overlapping launch k's
    integration), eager with a join and as a captured multi-frame step,
    give the per-scene results."""
    import torch
    from paper_1410_0925_gb300 import Batch, Scene, TsdfError
    ws, seqs, depth = data
    ref = _alone(ws, seqs, depth)
    stream = torch.cuda.Stream()
    with pytest.raises(TsdfError):
        Batch(8, tables=1, stream=stream).set_config(8, pipelined=True,
                                                     integrate_kernel="general")  # needs two tables
    batch = Batch(8, tables=3, stream=stream)
    batch.set_config(8, pipelined=True, integrate_kernel="general")
    scenes = [Scene.from_workload(w, stream=stream) for w in ws]
    for i in range(N_FRAMES):
        batch.integrate([(sc, d[i], _intr(w), s.poses[i])
                         for sc, d, w, s in zip(scenes, depth, ws, seqs)])
    batch.join()
    for sc, (rb, st) in zip(scenes, ref):
        _same(sc.read_blocks(), rb)
        assert sc.stats()["total_updated_voxels"] == st["total_updated_voxels"]
    gbatch = Batch(8, tables=N_FRAMES, stream=stream)
    gbatch.set_config(pipelined=True, integrate_kernel="staged", alloc_tile="32x8")
    items = lambda i: [(sc, d[i], _intr(w), s.poses[i])  # noqa: E731
                       for sc, d, w, s in zip(scenes, depth, ws, seqs)]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        for sc in scenes:
            sc.reset()
        for i in range(N_FRAMES):
            gbatch.prepare(items(i))
            gbatch.launch()
        gbatch.join()
    for _ in range(2):
        with torch.cuda.stream(stream):
            g.replay()
        for sc, (rb, _) in zip(scenes, ref):
            _same(sc.read_blocks(), rb)


@pytest.mark.parametrize("kernel,threads,ctas", [("staged", 512, 1), ("staged", 256, 1),
                                                 ("general", 256, 2), ("general", 256, 8)])
@pytest.mark.parametrize("tile", ["16x16", "16x8", "32x8"])
def test_every_schedule_gives_the_scenes_alone(data, kernel, threads, ctas, tile):
    """The schedules the autotuner chooses among (integration kernel design,
    CTA size, CTAs per SM, allocation tile) change nothing in the result:
    bit-identical to each scene fused alone."""
    import torch
    from paper_1410_0925_gb300 import Batch, Scene
    ws, seqs, depth = data
    ref = _alone(ws, seqs, depth)
    batch = Batch(8, stream=torch.cuda.Stream())
    batch.set_config(ctas, integrate_kernel=kernel, integrate_threads=threads, alloc_tile=tile)
    cfg = batch.config()
    assert (cfg["integrate_kernel"], cfg["alloc_tile"]) == (kernel, tile)
    scenes = [Scene.from_workload(w) for w in ws]
    for i in range(N_FRAMES):
        batch.integrate([(sc, d[i], _intr(w), s.poses[i])
                         for sc, d, w, s in zip(scenes, depth, ws, seqs)])
    for sc, (rb, st) in zip(scenes, ref):
        _same(sc.read_blocks(), rb)
        assert sc.stats()["total_updated_voxels"] == st["total_updated_voxels"]


def test_invalid_schedules_are_refused(data):
    from paper_1410_0925_gb300 import Batch, TsdfError
    batch = Batch(4)
    for kw in (dict(integrate_kernel="staged", integrate_ctas_per_sm=2),
               dict(integrate_kernel="staged", integrate_threads=384),
               dict(integrate_kernel="general", integrate_ctas_per_sm=9),
               dict(alloc_tile=3)):
        with pytest.raises(TsdfError):
            batch.set_config(**kw)
