"""The input generators: the torch renderer reproduces the host renderer's
noise-free frames, keeps its noise statistics, and both are seeded."""

import numpy as np
import pytest

from synthdepth import make_sequence, workload_kinect, workload_tiny
from synthdepth.configs import batched_workloads

torch = pytest.importorskip("torch")


def test_torch_renderer_matches_host_renderer_noise_free():
    from synthdepth.render_torch import make_sequence_torch
    w = workload_tiny()
    a = make_sequence(w, n_frames=3, first_frame=5)
    b = make_sequence_torch(w, n_frames=3, first_frame=5, device="cpu")
    assert np.array_equal(a.poses, b.poses)
    assert np.abs(a.depth - b.depth.numpy()).max() <= 1e-6


def test_torch_renderer_noise_statistics_and_seeding():
    from synthdepth.render_torch import make_sequence_torch
    w = workload_kinect(width=160, height=120, fx=131.25, fy=131.25, cx=79.5, cy=59.5)
    clean = make_sequence_torch(w, n_frames=2, device="cpu")
    clean_w = workload_kinect(width=160, height=120, fx=131.25, fy=131.25, cx=79.5,
                              cy=59.5, noise=False)
    ref = make_sequence_torch(clean_w, n_frames=2, device="cpu").depth.numpy()
    d = clean.depth.numpy()
    zero = d == 0
    assert 0.012 < zero.mean() < 0.03                     # 2 % dropped pixels
    z = ref[~zero]
    r = (d[~zero] - z) / (1.5e-3 * z * z)                # standardised noise
    assert abs(r.mean()) < 0.05 and 0.95 < r.std() < 1.05
    again = make_sequence_torch(w, n_frames=2, device="cpu").depth.numpy()
    assert np.array_equal(d, again)


def test_batched_workloads_cover_the_stated_mix():
    ws = batched_workloads()
    assert len(ws) == 64
    assert {(w.width, w.height) for w in ws} == {(160, 120), (320, 240), (640, 480)}
    assert {w.voxel_size for w in ws} == {0.004, 0.005, 0.010}
    assert all(abs(w.mu - 4 * w.voxel_size) < 1e-12 for w in ws)
    assert {w.pool_blocks for w in ws} <= {1 << 14, 1 << 16, 1 << 18}
