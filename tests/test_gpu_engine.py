"""The processing pipeline of one camera (Section 2.1) through tsdf_engine_*:
tracking against the model rendered from the last pose, fusion at the
tracked pose. Checked against what the synthetic sequence fixes: its true
poses (the tracked trajectory stays on them) and the model fused with them."""

import numpy as np
import pytest

from synthdepth import make_sequence, workload_kinect

pytestmark = pytest.mark.gpu


def _intr(w):
    from paper_1410_0925_gb300 import make_intrinsics
    return make_intrinsics(w.fx, w.fy, w.cx, w.cy, w.width, w.height)


def _pose_error(est, true):
    e = np.linalg.inv(est) @ true
    ang = np.degrees(np.arccos(np.clip((np.trace(e[:3, :3]) - 1) / 2, -1, 1)))
    return np.linalg.norm(e[:3, 3]), ang


def test_engine_tracks_the_sequence_and_fuses_the_same_model():
    import torch
    from paper_1410_0925_gb300 import Engine, Scene
    w = workload_kinect()
    n = 20
    seq = make_sequence(w, n_frames=n, colour=True)
    depth = torch.from_numpy(seq.depth).cuda()
    col = torch.from_numpy(seq.colour).cuda()
    eng = Engine(w.scene_desc(), _intr(w), seq.poses[0], levels=3, iterations=(4, 4, 6),
                 colour=True)
    worst_t, worst_a = 0.0, 0.0
    for i in range(n):
        pose = eng.process(depth[i], col[i])
        t, a = _pose_error(pose, seq.poses[i])
        worst_t, worst_a = max(worst_t, t), max(worst_a, a)
    print(f"worst tracking error {worst_t * 1e3:.2f} mm, {worst_a:.3f} deg")
    assert worst_t < 0.01 and worst_a < 1.0, (worst_t, worst_a)
    assert eng.tracker_status() == 0
    # the model against fusion at the true poses
    ref = Scene.from_workload(w)
    for i in range(n):
        ref.integrate(depth[i], _intr(w), seq.poses[i])
    got = eng.scene().read_blocks()
    want = ref.read_blocks()
    a = {tuple(k) for k in got.keys.tolist()}
    b = {tuple(k) for k in want.keys.tolist()}
    # millimetre pose differences move the blocks a segment only grazes
    assert len(a & b) / len(a | b) > 0.9                      # 0.936 measured
    assert eng.scene().stats()["frames"] == n
    rgbw = eng.scene().read_colour()
    assert rgbw[..., 3].max() > 0 and rgbw[..., :3].max() > 0


def test_engine_first_frame_and_errors():
    import torch
    from paper_1410_0925_gb300 import Engine, TsdfError
    w = workload_kinect()
    seq = make_sequence(w, n_frames=1)
    d = torch.from_numpy(seq.depth[0]).cuda()
    eng = Engine(w.scene_desc(), _intr(w), seq.poses[0], levels=1, iterations=(10,))
    pose = eng.process(d)
    assert np.array_equal(pose, seq.poses[0])                 # frame 0 keeps the initial pose
    assert eng.scene().stats()["allocated_blocks"] > 0
    with pytest.raises(TsdfError):
        eng.process(d, torch.zeros((w.height, w.width, 4), dtype=torch.uint8, device="cuda"))
    for kw in (dict(levels=0), dict(levels=5), dict(max_dist=0.0), dict(z_near=-1.0),
               dict(levels=2, iterations=(101, 0))):
        with pytest.raises(TsdfError):
            Engine(w.scene_desc(), _intr(w), seq.poses[0], **kw)
