"""The serving loop on the GPU: sessions that arrive while others are being
fused are admitted as memory frees up, share batched steps, and each
session's result equals the same session fused alone, bit for bit."""

import numpy as np
import pytest

from synthdepth import make_sequence, workload_tiny
from synthdepth.configs import STORAGE_F16, STORAGE_I16

pytestmark = pytest.mark.gpu

N_FRAMES = 8


def _workloads():
    return [
        workload_tiny(name="s0"),
        workload_tiny(name="s1", width=157, height=93, fx=120.0, fy=119.0, cx=77.3, cy=45.9,
                      voxel_size=0.015, mu=0.06, storage=STORAGE_I16, seed=21),
        workload_tiny(name="s2", voxel_size=0.025, mu=0.1, seed=22, storage=STORAGE_F16),
        workload_tiny(name="s3", seed=23, storage=STORAGE_I16),
        workload_tiny(name="s4", width=320, height=240, fx=262.5, fy=262.5, cx=159.5,
                      cy=119.5, voxel_size=0.01, mu=0.04, seed=24, pool_blocks=1 << 15,
                      hash_buckets_log2=15),
        # same buffer sizes as s0 with another voxel size: may reuse s0's scene
        workload_tiny(name="s5", voxel_size=0.03, mu=0.12, seed=25),
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


def test_sessions_alone_and_in_the_mix(data):
    import torch
    from paper_1410_0925_gb300 import Scene, Server, scene_device_bytes
    from paper_1410_0925_gb300.tsdf import SESSION_FINISHED, SESSION_QUEUED
    ws, seqs, depth = data
    alone, alone_stats = [], []
    for w, s, d in zip(ws, seqs, depth):
        sc = Scene.from_workload(w)
        for i in range(N_FRAMES):
            sc.integrate(d[i], _intr(w), s.poses[i])
        alone.append(sc.read_blocks())
        alone_stats.append(sc.stats())
    cost = [scene_device_bytes(w.width, w.height, **w.scene_desc()) for w in ws]
    budget = sorted(cost)[-1] + sorted(cost)[-2] + min(cost)   # room for about three
    stream = torch.cuda.Stream()
    srv = Server(budget, max_active=4, max_queued_frames=2, max_inflight_steps=2, stream=stream)
    sid = {}
    next_frame = {}
    results = {}
    tickets = set()
    saw_waiting = False
    saw_active = 0
    it = 0
    while len(results) < len(ws):
        # one new session every third iteration, while earlier ones run
        k = it // 3
        if it % 3 == 0 and k < len(ws):
            sid[k] = srv.open_workload(ws[k])
            next_frame[k] = 0
        # clients keep up to two frames queued
        for j, s in sid.items():
            if j in results:
                continue
            info = srv.session_info(s)
            while next_frame[j] < N_FRAMES and info["frames_submitted"] - info["frames_launched"] < 2:
                t = srv.submit(s, depth[j][next_frame[j]], _intr(ws[j]), seqs[j].poses[next_frame[j]])
                tickets.add(t)
                next_frame[j] += 1
                info = srv.session_info(s)
                if next_frame[j] == N_FRAMES:
                    srv.close_session(s)
            if info["state"] == SESSION_QUEUED:
                saw_waiting = True
        st = srv.step()
        assert st["active_bytes"] <= budget
        saw_active = max(saw_active, st["active_sessions"])
        for t, s, t_sub, t_done in srv.poll():
            tickets.discard(t)
            assert t_done >= t_sub
        for j, s in sid.items():
            if j in results:
                continue
            info = srv.session_info(s)
            if info["state"] == SESSION_FINISHED:
                results[j] = srv.scene(s).read_blocks()
                assert info["frames_done"] == N_FRAMES and info["device_status"] == 0
                assert info["updated_voxels"] == alone_stats[j]["total_updated_voxels"]
                assert info["allocated_blocks"] == alone_stats[j]["allocated_blocks"]
                assert info["open_ms"] <= info["admit_ms"] <= info["finish_ms"]
                srv.release(s)
        it += 1
        assert it < 2000, "serving loop made no progress"
    srv.poll(wait_all=True)
    assert not tickets, "every submitted frame is reported done once"
    assert saw_waiting, "a session waited for memory"
    assert saw_active >= 2, "sessions shared steps"
    for j in range(len(ws)):
        a, b = alone[j], results[j]
        assert np.array_equal(a.keys, b.keys) and np.array_equal(a.w, b.w)
        assert np.array_equal(a.sdf, b.sdf)
    srv.close()


def test_server_rejects_bad_requests(data):
    from paper_1410_0925_gb300 import Server, TsdfError
    ws, seqs, depth = data
    srv = Server(1 << 30, max_active=2, max_queued_frames=1)
    with pytest.raises(TsdfError):
        srv.open(160, 120, voxel_size=0.02, mu=0.08, pool_blocks=1 << 22)   # over budget
    s = srv.open_workload(ws[0])
    srv.submit(s, depth[0][0], _intr(ws[0]), seqs[0].poses[0])
    with pytest.raises(TsdfError):
        srv.submit(s, depth[0][1], _intr(ws[0]), seqs[0].poses[1])          # queue full
    with pytest.raises(TsdfError):
        srv.release(s + 100)
    srv.step()
    with pytest.raises(TsdfError):
        srv.release(s)                                                      # still fusing
    srv.close_session(s)
    srv.poll(wait_all=True)
    assert srv.session_info(s)["state"] == 2
    srv.release(s)
    srv.close()
