"""GPU parity of swapping (Section 5): tsdf_swap_out / tsdf_swap_in through
the C ABI against the oracle's or_swap_out / or_swap_in on the same seeded
frames and the same call schedule. Device blocks and host copies are compared
separately, by the fusion parity rules, on the blocks whose swap decisions the
oracle did not flag; round trips must be bit-exact."""

import numpy as np
import pytest

import oracle
from parity import TOL, oracle_intr, oracle_params
from synthdepth import make_sequence, workload_kinect, workload_tiny
from synthdepth.configs import STORAGE_F32, STORAGE_I16

pytestmark = pytest.mark.gpu

BIG = 10 ** 9
# a view that sees nothing (every world point with z > -100 m is behind it)
AWAY = np.array([[-1.0, 0, 0, 0], [0, 1.0, 0, 0], [0, 0, -1.0, -100.0], [0, 0, 0, 1.0]])


def _intr(w):
    from paper_1410_0925_gb300 import make_intrinsics
    return make_intrinsics(w.fx, w.fy, w.cx, w.cy, w.width, w.height)


def _scene(w, storage, colour, capacity):
    from paper_1410_0925_gb300 import Scene
    sc = Scene.from_workload(w, storage=storage)
    if colour:
        sc.enable_colour()
    sc.enable_swapping(capacity)
    return sc


def _run(w, seq, order, capacity, margin, storage=STORAGE_F32, colour=False):
    """The same schedule on the GPU and in the oracle: per frame, the ops of
    `order` ("in", "int", "out") with that frame's view."""
    import torch
    sc = _scene(w, storage, colour, capacity)
    o = oracle.Oracle(oracle_params(w, storage, pool_blocks=w.pool_blocks))
    intr, ointr = _intr(w), oracle_intr(w)
    depth = torch.from_numpy(np.ascontiguousarray(seq.depth)).cuda()
    col = torch.from_numpy(np.ascontiguousarray(seq.colour)).cuda() if colour else None
    moved = []
    for t in range(seq.depth.shape[0]):
        P = seq.poses[t]
        for op in order:
            if op == "int":
                if colour:
                    sc.integrate_rgb(depth[t], col[t], intr, P)
                    o.integrate_rgb(seq.depth[t], seq.colour[t], ointr, P)
                else:
                    sc.integrate(depth[t], intr, P)
                    o.integrate(seq.depth[t], ointr, P)
            elif op == "in":
                sc.swap_in(intr, P, margin)
                n, _ = o.swap_in(w.width, w.height, ointr, P, margin, 0.0, capacity)
                moved.append(("in", sc.swap_stats()["last_in"], n))
            else:
                sc.swap_out(intr, P, margin)
                n = o.swap_out(w.width, w.height, ointr, P, margin, 0.0, capacity)
                moved.append(("out", sc.swap_stats()["last_out"], n))
    return sc, o, moved


def _compare_maps(gblocks, gcol, ores, ocol, ghosts, extra_ok, storage):
    """Block sets and voxels of one side (device or host)."""
    tol = TOL[storage]
    gk = [tuple(k) for k in gblocks.keys.tolist()]
    ok_ = [tuple(k) for k in ores["keys"].tolist()]
    unsure = {k for k, f in zip(ok_, ores["bflag"])
              if f & (oracle.BLOCK_MEMBERSHIP_AMBIGUOUS | oracle.BLOCK_SWAP_AMBIGUOUS)}
    missing = set(ok_) - set(gk) - unsure
    extra = set(gk) - set(ok_) - ghosts - extra_ok
    assert not missing, f"{len(missing)} oracle blocks missing on the GPU, e.g. {sorted(missing)[:3]}"
    assert not extra, f"{len(extra)} GPU blocks the oracle does not have, e.g. {sorted(extra)[:3]}"
    gidx = {k: i for i, k in enumerate(gk)}
    gvals = gblocks.sdf_values()
    strict = skipped = 0
    max_err = 0.0
    for b, k in enumerate(ok_):
        if k not in gidx:
            continue
        if int(ores["bflag"][b]) & ~oracle.BLOCK_SWAPPED:
            skipped += 512
            continue
        g = gidx[k]
        m = ores["vflag"][b] == 0
        bad = np.nonzero(m & (gblocks.w[g] != ores["w"][b]))[0]
        assert len(bad) == 0, (k, bad[0], gblocks.w[g][bad[0]], ores["w"][b][bad[0]])
        if m.any():
            e = float(np.abs(gvals[g] - ores["sdf"][b])[m].max())
            max_err = max(max_err, e)
            assert e <= tol, (k, e)
        if gcol is not None:
            assert np.array_equal(gcol[g][m], ocol[b][m]), f"colour differs in block {k}"
        strict += int(m.sum())
        skipped += int((~m).sum())
    return dict(blocks=len(gk), oracle_blocks=len(ok_), strict=strict, skipped=skipped,
                max_err=max_err)


def _compare_all(sc, o, storage, colour):
    res, hres = o.read(), o.read_host()
    ghosts = {tuple(k) for k in o.ghosts().tolist()}
    amb = {tuple(k) for k, f in zip(res["keys"].tolist(), res["bflag"])
           if f & oracle.BLOCK_SWAP_AMBIGUOUS}
    amb |= {tuple(k) for k, f in zip(hres["keys"].tolist(), hres["bflag"])
            if f & oracle.BLOCK_SWAP_AMBIGUOUS}
    dev = sc.read_blocks()
    dcol = sc.read_colour() if colour else None
    host, hcol = sc.read_host_blocks(colour=colour)
    d = _compare_maps(dev, dcol, res, o.read_colour() if colour else None, ghosts, amb, storage)
    h = _compare_maps(host, hcol, hres, hres["rgbw"] if colour else None, ghosts, amb, storage)
    return d, h, len(amb)


@pytest.fixture(scope="module")
def tiny():
    w = workload_tiny()
    return w, make_sequence(w, colour=True)


@pytest.mark.parametrize("order", [("int", "in", "out"), ("in", "int", "out")])
@pytest.mark.parametrize("storage", [STORAGE_F32, STORAGE_I16])
def test_swap_schedule_matches_oracle(tiny, order, storage):
    """Every frame: fuse, merge or bring back, move out what the view does
    not see (capacity 200 blocks, so calls are often full and the smallest
    keys win); or bring back first, then fuse."""
    w, seq = tiny
    sc, o, moved = _run(w, seq, order, capacity=200, margin=2.0, storage=storage,
                        colour=storage == STORAGE_F32)
    d, h, n_amb = _compare_all(sc, o, storage, storage == STORAGE_F32)
    print(order, storage, d, h, "swap-ambiguous", n_amb)
    assert sum(g for _, g, _ in moved) > 1000
    assert d["strict"] > 0.5 * 512 * d["oracle_blocks"]
    assert h["strict"] > 0 or h["oracle_blocks"] == 0
    assert n_amb <= 0.01 * (d["oracle_blocks"] + h["oracle_blocks"])
    if n_amb == 0 and len(o.ghosts()) == 0:
        assert [g for _, g, _ in moved] == [n for _, _, n in moved]
    assert all(g <= 200 for _, g, _ in moved)
    assert sc.stats_and_status()[1] == 0


def test_round_trip_is_bit_exact(tiny):
    """Everything out, everything back: the device map is bit for bit what it
    was, the pool is dense again, and fusion continues exactly as in a scene
    that never swapped."""
    import torch
    from paper_1410_0925_gb300 import Scene
    w, seq = tiny
    intr = _intr(w)
    depth = torch.from_numpy(np.ascontiguousarray(seq.depth)).cuda()
    col = torch.from_numpy(np.ascontiguousarray(seq.colour)).cuda()
    a = Scene.from_workload(w)
    a.enable_colour()
    # 4096 blocks per call: one call takes the whole map out, and the pool
    # keeps room for a full call while it comes back
    b = _scene(w, STORAGE_F32, True, 4096)
    for t in range(10):
        a.integrate_rgb(depth[t], col[t], intr, seq.poses[t])
        b.integrate_rgb(depth[t], col[t], intr, seq.poses[t])
    before = b.read_blocks()
    n = len(before.keys)
    assert n <= 4096
    b.swap_out(intr, AWAY)
    st = b.swap_stats()
    assert st["last_out"] == n and st["host_blocks"] == n and b.num_blocks() == 0
    host, _ = b.read_host_blocks()
    assert np.array_equal(host.keys, before.keys) and np.array_equal(host.sdf, before.sdf)
    assert np.array_equal(host.w, before.w)
    for P in seq.poses:
        b.swap_in(intr, P, 1e9)
    assert b.swap_stats()["host_blocks"] == 0
    after = b.read_blocks()
    assert np.array_equal(after.keys, before.keys)
    assert np.array_equal(after.sdf, before.sdf) and np.array_equal(after.w, before.w)
    assert np.array_equal(b.read_colour(), a.read_colour())
    ptr = b.lookup(after.keys)
    assert (ptr >= 0).all() and ptr.max() < n and len(set(ptr.tolist())) == n
    for t in range(10, 20):
        a.integrate_rgb(depth[t], col[t], intr, seq.poses[t])
        b.integrate_rgb(depth[t], col[t], intr, seq.poses[t])
    x, y = a.read_blocks(), b.read_blocks()
    assert np.array_equal(x.keys, y.keys) and np.array_equal(x.sdf, y.sdf)
    assert np.array_equal(x.w, y.w) and np.array_equal(a.read_colour(), b.read_colour())
    assert b.stats_and_status()[1] == 0


def test_partial_swap_out_compacts_the_pool(tiny):
    """A swap-out that frees blocks in the middle of the pool moves the tail
    into the holes: every device block keeps its data and its hash entry
    points at it."""
    import torch
    w, seq = tiny
    intr = _intr(w)
    sc = _scene(w, STORAGE_F32, False, w.pool_blocks)
    depth = torch.from_numpy(np.ascontiguousarray(seq.depth)).cuda()
    for t in range(12):
        sc.integrate(depth[t], intr, seq.poses[t])
    before = sc.read_blocks()
    sc.swap_out(intr, seq.poses[3])
    st = sc.swap_stats()
    assert 0 < st["last_out"] < len(before.keys)
    after = sc.read_blocks()
    host, _ = sc.read_host_blocks()
    # the two sides partition the map, with the data unchanged
    assert len(after.keys) + len(host.keys) == len(before.keys)
    idx = {tuple(k): i for i, k in enumerate(before.keys.tolist())}
    for side in (after, host):
        for i, k in enumerate(side.keys.tolist()):
            j = idx[tuple(k)]
            assert np.array_equal(side.sdf[i], before.sdf[j]) and np.array_equal(side.w[i], before.w[j])
    ptr = sc.lookup(after.keys)
    assert sorted(ptr.tolist()) == list(range(len(after.keys)))
    assert (sc.lookup(host.keys) < 0).all()
    # the swapped-out blocks are exactly the oracle's
    o = oracle.Oracle(oracle_params(w, pool_blocks=w.pool_blocks))
    for t in range(12):
        o.integrate(seq.depth[t], oracle_intr(w), seq.poses[t])
    o.swap_out(w.width, w.height, oracle_intr(w), seq.poses[3], 0.0, 0.0, w.pool_blocks)
    hres = o.read_host()
    amb = {tuple(k) for k, f in zip(hres["keys"].tolist(), hres["bflag"]) if f & 5}
    gk = {tuple(k) for k in host.keys.tolist()}
    okk = {tuple(k) for k in hres["keys"].tolist()}
    assert (gk ^ okk) <= amb | {tuple(k) for k in o.ghosts().tolist()}


def test_swap_calls_replay_in_a_graph(tiny):
    """Six steps (swap in, fuse, swap out; 100 blocks per call) captured in
    one CUDA graph after a reset equal the same calls made eagerly on a fresh
    scene, bit for bit, device blocks and host copies."""
    import torch
    from paper_1410_0925_gb300 import Scene
    w, seq = tiny
    intr = _intr(w)
    depth = torch.from_numpy(np.ascontiguousarray(seq.depth)).cuda()
    steps = [(2 * i, 2 * i + 9) for i in range(6)]  # (fused frame, swap-out view)

    def enqueue(sc):
        for t, v in steps:
            sc.swap_in(intr, seq.poses[t])
            sc.integrate(depth[t], intr, seq.poses[t])
            sc.swap_out(intr, seq.poses[v])

    stream = torch.cuda.Stream()
    eager = Scene.from_workload(w, stream=stream)
    eager.enable_swapping(100)
    torch.cuda.synchronize()
    enqueue(eager)
    graphed = Scene.from_workload(w, stream=stream)
    graphed.enable_swapping(100)
    enqueue(graphed)  # warm-up: work buffers are allocated outside the capture
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        graphed.reset()
        enqueue(graphed)
    with torch.cuda.stream(stream):
        g.replay()
    stream.synchronize()
    a, b = eager.read_blocks(), graphed.read_blocks()
    assert np.array_equal(a.keys, b.keys) and np.array_equal(a.sdf, b.sdf)
    assert np.array_equal(a.w, b.w)
    ha, hb = eager.read_host_blocks()[0], graphed.read_host_blocks()[0]
    assert len(ha.keys) > 0
    assert np.array_equal(ha.keys, hb.keys) and np.array_equal(ha.sdf, hb.sdf)
    assert np.array_equal(ha.w, hb.w)
    sa, sb = eager.swap_stats(), graphed.swap_stats()
    for k in ("host_blocks", "last_out", "last_in", "last_merged"):
        assert sa[k] == sb[k], k


def test_swap_errors(tiny):
    import torch
    from paper_1410_0925_gb300 import Batch, Scene, TsdfError
    w, seq = tiny
    intr = _intr(w)
    sc = Scene.from_workload(w)
    with pytest.raises(TsdfError):
        sc.swap_out(intr, seq.poses[0])
    with pytest.raises(TsdfError):
        sc.swap_stats()
    with pytest.raises(TsdfError):
        sc.enable_swapping(0)
    with pytest.raises(TsdfError):
        sc.enable_swapping(w.pool_blocks + 1)
    sc.enable_swapping(64)
    with pytest.raises(TsdfError):
        sc.enable_swapping(64)
    with pytest.raises(TsdfError):
        sc.enable_colour()
    with pytest.raises(TsdfError):
        sc.swap_out(intr, seq.poses[0], margin_px=-1.0)
    bad = np.array(seq.poses[0])
    bad[3, 3] = 2.0
    with pytest.raises(TsdfError):
        sc.swap_in(intr, bad)
    d = torch.from_numpy(np.ascontiguousarray(seq.depth[0])).cuda()
    # batched steps refuse swapping scenes
    with pytest.raises(TsdfError):
        Batch(2).integrate([(sc, d, intr, seq.poses[0])])
    # resume is refused while host copies exist; reset clears them
    sc.integrate(d, intr, seq.poses[0])
    blocks = sc.read_blocks()
    sc.swap_out(intr, AWAY)
    assert sc.swap_stats()["host_blocks"] > 0
    with pytest.raises(TsdfError):
        sc.load_blocks(blocks)
    sc.reset()
    assert sc.swap_stats()["host_blocks"] == 0 and sc.num_blocks() == 0
    sc.load_blocks(blocks)
    assert sc.num_blocks() == len(blocks.keys)


def test_kinect_swapping_loses_nothing():
    """Kinect 640x480, 60 noisy frames: bring back what the view sees (16 px
    margin), fuse, move out what it does not, 4096 blocks per call. The map
    (device blocks plus host copies) equals fusion without swapping bit for
    bit, as the oracle's swap-in-before-fusion identity requires, and every
    call respects the bound."""
    import torch
    from paper_1410_0925_gb300 import Scene
    w = workload_kinect(n_frames=60)
    seq = make_sequence(w)
    intr = _intr(w)
    depth = torch.from_numpy(np.ascontiguousarray(seq.depth)).cuda()
    a = Scene.from_workload(w)
    b = Scene.from_workload(w)
    b.enable_swapping(4096)
    outs = []
    for t in range(60):
        P = seq.poses[t]
        b.swap_in(intr, P, 16.0)
        a.integrate(depth[t], intr, P)
        b.integrate(depth[t], intr, P)
        b.swap_out(intr, P, 16.0)
        st = b.swap_stats()
        outs.append(st["last_out"])
        assert st["last_out"] <= 4096 and st["last_in"] <= 4096
    assert b.swap_stats()["total_merged"] == 0
    assert sum(outs) > 1000
    full = a.read_blocks()
    dev = b.read_blocks()
    host, _ = b.read_host_blocks()
    keys = np.concatenate([dev.keys, host.keys])
    order = np.lexsort(keys.T[::-1])
    assert np.array_equal(keys[order], full.keys)
    assert np.array_equal(np.concatenate([dev.sdf, host.sdf])[order], full.sdf)
    assert np.array_equal(np.concatenate([dev.w, host.w])[order], full.w)
    assert b.stats_and_status()[1] == 0


def test_engine_with_swapping():
    """The pipeline engine with swapping (bring in, fuse, move out around
    every fusion, 16 px margin, 4096 blocks a call) on 20 noisy Kinect
    frames: blocks do leave, tracking stays as accurate as without swapping
    (within 1 cm and the same poses up to a millimetre), and the map (device
    blocks plus host copies) covers the same blocks; where the poses agree bit
    for bit, the maps do too."""
    import torch
    from paper_1410_0925_gb300 import Engine
    w = workload_kinect(n_frames=20)
    seq = make_sequence(w)
    intr = _intr(w)
    depth = torch.from_numpy(np.ascontiguousarray(seq.depth)).cuda()
    a = Engine(w.scene_desc(), intr, seq.poses[0])
    b = Engine(w.scene_desc(), intr, seq.poses[0], swap_blocks=4096, swap_margin_px=16.0)
    same = True
    for t in range(20):
        pa, pb = a.process(depth[t]), b.process(depth[t])
        same = same and np.array_equal(pa, pb)
        assert np.linalg.norm((np.linalg.inv(pb) @ seq.poses[t])[:3, 3]) < 0.01
        assert np.linalg.norm(pa[:3, 3] - pb[:3, 3]) < 1e-3
    sa, sb = a.scene(), b.scene()
    st = sb.swap_stats()
    assert st["total_out"] > 0 and st["host_blocks"] > 0
    full = sa.read_blocks()
    dev = sb.read_blocks()
    host, _ = sb.read_host_blocks()
    keys = np.concatenate([dev.keys, host.keys])
    assert len(keys) == len({tuple(k) for k in keys.tolist()})
    order = np.lexsort(keys.T[::-1])
    if same:
        assert np.array_equal(keys[order], full.keys)
        assert np.array_equal(np.concatenate([dev.sdf, host.sdf])[order], full.sdf)
        assert np.array_equal(np.concatenate([dev.w, host.w])[order], full.w)
    else:
        assert abs(len(keys) - len(full.keys)) < 0.01 * len(full.keys)
    assert a.tracker_status() == 0 and b.tracker_status() == 0
