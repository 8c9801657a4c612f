"""GPU parity of colour fusion (voxel clr / w_color, Section 3.1; updated with
the depth by the integration of Section 4.3): tsdf_integrate_rgb through the
C ABI against the oracle's or_integrate_rgb on the same seeded frames. Depth
is compared by the fusion parity rules; colours (integers decided in the
listing's float arithmetic on both sides) must be bit-exact on every voxel
whose depth decisions are unflagged, in blocks with an unambiguous history."""

import numpy as np
import pytest

import oracle
from parity import compare, oracle_intr, oracle_params
from synthdepth import make_sequence, workload_kinect, workload_tiny
from synthdepth.configs import STORAGE_F16, STORAGE_F32, STORAGE_I16

pytestmark = pytest.mark.gpu


def _intr(w):
    from paper_1410_0925_gb300 import make_intrinsics
    return make_intrinsics(w.fx, w.fy, w.cx, w.cy, w.width, w.height)


def _oracle_rgb(w, seq):
    p = oracle_params(w)
    o = oracle.Oracle(p)
    statuses = [o.integrate_rgb(seq.depth[i], seq.colour[i], oracle_intr(w), seq.poses[i])
                for i in range(seq.depth.shape[0])]
    return dict(res=o.read(), ghosts=o.ghosts(), params=p, statuses=statuses), o.read_colour()


def _gpu_rgb(w, seq, stream=None):
    import torch
    from paper_1410_0925_gb300 import Scene
    sc = Scene.from_workload(w, stream=stream)
    sc.enable_colour()
    depth = torch.from_numpy(np.ascontiguousarray(seq.depth)).cuda()
    col = torch.from_numpy(np.ascontiguousarray(seq.colour)).cuda()
    for i in range(depth.shape[0]):
        sc.integrate_rgb(depth[i], col[i], _intr(w), seq.poses[i])
    return sc, depth, col


def _compare_colour(blocks, gcol, orc, ocol):
    """Bit-exact colours on unflagged voxels of unambiguous common blocks."""
    res = orc["res"]
    gidx = {tuple(k): i for i, k in enumerate(blocks.keys.tolist())}
    exact = 0
    for b, k in enumerate(res["keys"].tolist()):
        if res["bflag"][b] or tuple(k) not in gidx:
            continue
        g = gidx[tuple(k)]
        m = res["vflag"][b] == 0
        assert np.array_equal(gcol[g][m], ocol[b][m]), f"colour differs in block {k}"
        exact += int(m.sum())
    return exact


@pytest.mark.parametrize("storage", [STORAGE_F32, STORAGE_I16, STORAGE_F16])
def test_colour_tiny_matches_oracle(storage):
    w = workload_tiny(storage=storage)
    seq = make_sequence(w, n_frames=8, colour=True)
    orc, ocol = _oracle_rgb(w, seq)
    sc, _, _ = _gpu_rgb(w, seq)
    blocks = sc.read_blocks()
    rep = compare(blocks, orc, seq, w, storage)
    assert rep["unresolved"] == 0
    gcol = sc.read_colour()
    assert gcol.shape == (len(blocks.keys), 512, 4)
    exact = _compare_colour(blocks, gcol, orc, ocol)
    assert exact > 0.95 * 512 * len(orc["res"]["keys"])
    assert (gcol[..., 3] == blocks.w).mean() > 0.999     # colour weight follows depth weight
    assert gcol[..., :3].max() > 0


def test_colour_kinect_full_resolution():
    w = workload_kinect()
    seq = make_sequence(w, n_frames=4, colour=True)
    orc, ocol = _oracle_rgb(w, seq)
    sc, _, _ = _gpu_rgb(w, seq)
    blocks = sc.read_blocks()
    rep = compare(blocks, orc, seq, w, STORAGE_F32, max_candidates=3000)
    assert rep["unresolved"] == 0
    exact = _compare_colour(blocks, sc.read_colour(), orc, ocol)
    assert exact > 0.95 * 512 * len(orc["res"]["keys"])   # 98.5 % measured


def test_colour_leaves_depth_alone_and_depth_frames_leave_colour():
    import torch
    from paper_1410_0925_gb300 import Scene
    w = workload_tiny()
    seq = make_sequence(w, n_frames=6, colour=True)
    sc, depth, col = _gpu_rgb(w, seq)
    plain = Scene.from_workload(w)
    for i in range(6):
        plain.integrate(depth[i], _intr(w), seq.poses[i])
    a, b = sc.read_blocks(), plain.read_blocks()
    assert np.array_equal(a.keys, b.keys) and np.array_equal(a.w, b.w)
    assert np.array_equal(a.sdf, b.sdf)
    before = sc.read_colour()
    # depth-only frames (pipelined sequence too) keep colours; their new
    # blocks start at colour 0
    more = make_sequence(workload_tiny(), n_frames=10)
    d2 = torch.from_numpy(np.ascontiguousarray(more.depth[6:])).cuda()
    sc.integrate(d2[0], _intr(w), more.poses[6])
    sc.integrate_frames(d2[1:], _intr(w), more.poses[7:])
    after_blocks = sc.read_blocks()
    after = sc.read_colour()
    old = {tuple(k): i for i, k in enumerate(a.keys.tolist())}
    n_new = 0
    for j, k in enumerate(after_blocks.keys.tolist()):
        if tuple(k) in old:
            assert np.array_equal(after[j], before[old[tuple(k)]])
        else:
            n_new += 1
            assert (after[j] == 0).all()
    assert n_new > 0


def test_colour_reset_load_graph_and_errors():
    import torch
    from paper_1410_0925_gb300 import Batch, Scene, TsdfError
    w = workload_tiny()
    seq = make_sequence(w, n_frames=4, colour=True)
    stream = torch.cuda.Stream()
    sc, depth, col = _gpu_rgb(w, seq, stream=stream)
    ref_blocks, ref_col = sc.read_blocks(), sc.read_colour()
    # reset, then the same frames again as one captured graph
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        sc.reset()
        for i in range(4):
            sc.integrate_rgb(depth[i], col[i], _intr(w), seq.poses[i])
    with torch.cuda.stream(stream):
        g.replay()
    stream.synchronize()
    assert np.array_equal(sc.read_colour(), ref_col)
    # blocks loaded into a colour scene read colour 0
    other = Scene.from_workload(w)
    other.enable_colour()
    other.load_blocks(ref_blocks)
    assert (other.read_colour() == 0).all()
    # errors
    plain = Scene.from_workload(w)
    with pytest.raises(TsdfError):
        plain.integrate_rgb(depth[0], col[0], _intr(w), seq.poses[0])   # colour not enabled
    with pytest.raises(TsdfError):
        plain.read_colour()
    with pytest.raises(ValueError):
        sc.integrate_rgb(depth[0], col[0, :, :, :3].contiguous(), _intr(w), seq.poses[0])
    batch = Batch(2)
    with pytest.raises(TsdfError):
        batch.integrate([(sc, depth[0], _intr(w), seq.poses[0])])
