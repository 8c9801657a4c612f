"""Helpers shared by the GPU parity tests: run a sequence through the CUDA
library and through the FP64 oracle on the same inputs, and compare.

Comparison rules (FP32 GPU against FP64 oracle):
  * blocks: every oracle block that some segment meets robustly must be on
    the GPU; every GPU block must be an oracle block or a ghost (a block that
    a segment grazes within the margin); both sets are reported.
  * voxels of blocks with an unambiguous allocation frame, whose decisions
    were never within the margins: weights bit-exact, sdf within `tol`.
  * every other voxel (flagged decision, or block allocated in an ambiguous
    frame): the GPU state must equal, within `tol`, one of the states the
    oracle's single-voxel re-simulation admits (both outcomes of every
    flagged decision).
"""

from __future__ import annotations

import numpy as np

import oracle

TOL = {0: 1e-5, 1: 1.0 / 32767.0 + 1e-5, 2: 1e-3}

# Pixel-rounding margin of the GPU parity tests. The GPU's pixel coordinate
# x = fx X / Z + cx is FP32 from a double-float block origin: X and Z carry
# about 2.4e-7 m of rounding at a few metres, the approximate reciprocal 2^-22
# relative, the final fma half an ulp of a few hundred pixels, so |x_gpu -
# x_exact| < 1.5e-4 px. A margin of 2.5e-4 px (tighter than the oracle's
# default 1e-3) keeps every decision the GPU can take differently flagged
# and flags about 4 x 2.5e-4 of the voxel-frames (two coordinates, a window
# of 2 x margin each); the tests fail if a strictly checked voxel disagrees.
DELTA_PX = 2.5e-4


def f32(x) -> float:
    return float(np.float32(x))


def oracle_params(w, storage=None, pool_blocks=0, delta_px=DELTA_PX) -> oracle.OracleParams:
    return oracle.OracleParams(voxel_size=f32(w.voxel_size), mu=f32(w.mu),
                               max_weight=w.max_weight,
                               storage=w.storage if storage is None else storage,
                               pool_blocks=pool_blocks, delta_px=delta_px)


def oracle_intr(w):
    return tuple(f32(v) for v in (w.fx, w.fy, w.cx, w.cy))


def run_oracle(w, seq, storage=None, pool_blocks=0):
    p = oracle_params(w, storage, pool_blocks)
    o = oracle.Oracle(p)
    statuses = []
    for i in range(seq.depth.shape[0]):
        statuses.append(o.integrate(seq.depth[i], oracle_intr(w), seq.poses[i]))
    return dict(res=o.read(), ghosts=o.ghosts(), params=p, statuses=statuses)


def run_gpu(w, seq, storage=None, **scene_over):
    import torch
    from paper_1410_0925_gb300 import Scene, make_intrinsics
    desc = dict(w.scene_desc())
    if storage is not None:
        desc["storage"] = storage
    desc.update(scene_over)
    scene = Scene(**desc)
    intr = make_intrinsics(w.fx, w.fy, w.cx, w.cy, w.width, w.height)
    depth = torch.from_numpy(np.ascontiguousarray(seq.depth)).cuda()
    for i in range(depth.shape[0]):
        scene.integrate(depth[i], intr, seq.poses[i])
    stats, status = scene.stats_and_status()
    blocks = scene.read_blocks(check=False)
    return scene, blocks, stats, status


def compare(gpu_blocks, orc, seq, w, storage, tol=None, max_candidates=None,
            rng_seed=0) -> dict:
    """Compare as described above; every flagged voxel is checked against
    the re-simulation unless `max_candidates` limits it to a random sample.
    Reports the flagged fraction (flagged voxels over all voxels of the
    oracle blocks present on the GPU), the ghost blocks and the largest
    strict sdf error."""
    tol = TOL[storage] if tol is None else tol
    res, ghosts, p = orc["res"], orc["ghosts"], orc["params"]
    gvals = gpu_blocks.sdf_values()
    gk = [tuple(k) for k in gpu_blocks.keys.tolist()]
    ok_ = [tuple(k) for k in res["keys"].tolist()]
    gset, oset = set(gk), set(ok_)
    ghost_set = {tuple(k) for k in ghosts.tolist()}
    memb_amb = {k for k, f in zip(ok_, res["bflag"]) if f & oracle.BLOCK_MEMBERSHIP_AMBIGUOUS}
    missing = oset - gset - memb_amb
    extra = gset - oset - ghost_set
    assert not missing, f"{len(missing)} robust oracle blocks missing on the GPU, e.g. {sorted(missing)[:3]}"
    assert not extra, f"{len(extra)} GPU blocks the oracle never allocates, e.g. {sorted(extra)[:3]}"
    gidx = {k: i for i, k in enumerate(gk)}

    strict_vox = 0
    flagged = []  # (oracle block row, voxel index, gpu row)
    max_err = 0.0
    for b, k in enumerate(ok_):
        if k not in gidx:
            continue
        g = gidx[k]
        if res["bflag"][b] & oracle.BLOCK_HISTORY_AMBIGUOUS:
            flagged.extend((b, li, g) for li in range(512))
            continue
        m = res["vflag"][b] == 0
        wg, wo = gpu_blocks.w[g], res["w"][b]
        bad_w = np.nonzero(m & (wg != wo))[0]
        assert len(bad_w) == 0, (f"weight mismatch in block {k} voxel {bad_w[0]}: "
                                 f"gpu {wg[bad_w[0]]} oracle {wo[bad_w[0]]}")
        err = np.abs(gvals[g] - res["sdf"][b])[m]
        if err.size:
            e = float(err.max())
            max_err = max(max_err, e)
            assert e <= tol, f"sdf error {e} > {tol} in block {k}"
        strict_vox += int(m.sum())
        flagged.extend((b, li, g) for li in np.nonzero(~m)[0])

    # flagged voxels: the GPU state must be one the re-simulation admits
    rng = np.random.default_rng(rng_seed)
    order = rng.permutation(len(flagged))
    if max_candidates is not None:
        order = order[:max_candidates]
    hit_cache = {}
    n_cand = 0
    n_unresolved = 0
    intr = oracle_intr(w)
    for j in order:
        b, li, g = flagged[j]
        key = res["keys"][b]
        kt = tuple(key.tolist())
        if kt not in hit_cache:
            hit_cache[kt] = oracle.block_hit_frames(key, seq.depth, intr, seq.poses, p)
        vox = key * 8 + np.array([li % 8, (li // 8) % 8, li // 64])
        c = oracle.voxel_candidates(vox, seq.depth, intr, seq.poses, p, hit_cache[kt], max_out=256)
        if c is None:
            n_unresolved += 1
            continue
        cs, cw = c
        gs, gw = gvals[g, li], gpu_blocks.w[g, li]
        okc = [(cw[i] == gw and abs(cs[i] - gs) <= tol) for i in range(len(cs))]
        assert any(okc), (f"voxel {vox.tolist()} gpu ({gs}, {gw}) not among the oracle's "
                          f"admissible states {list(zip(cs.tolist(), cw.tolist()))}")
        n_cand += 1
    matched = len(oset & gset)
    return dict(gpu_blocks=len(gset), oracle_blocks=len(oset), ghosts=len(ghost_set),
                ghosts_on_gpu=len(gset & ghost_set), membership_ambiguous=len(memb_amb),
                strict_voxels=strict_vox, flagged_voxels=len(flagged),
                flagged_fraction=len(flagged) / max(512 * matched, 1),
                flagged_checked=n_cand, unresolved=n_unresolved, max_sdf_err=max_err,
                max_weight=int(gpu_blocks.w.max()) if len(gpu_blocks.w) else 0)


def flag_bound(n_frames: int, delta_px: float = DELTA_PX, slack: float = 2.0) -> float:
    """Upper bound of the flagged fraction expected from the margins: each
    voxel-frame falls within the pixel-rounding margin of x or y with
    probability about 4 delta_px (the other margins, eta = -mu and the image
    border, are far thinner in this workload); a voxel is flagged if any of
    its frames is, so at most n_frames times that, with `slack` for blocks
    whose whole history is ambiguous."""
    return slack * n_frames * 4.0 * delta_px


def check_sampled(blocks, w, depth, poses, storage, n_blocks=16, n_vox=24, seed=11) -> int:
    """Full-size check on sampled outputs: global invariants on every voxel
    (weights <= cap, sdf in [-1, 1], untouched voxels at their initial 1.0),
    and sampled voxels of sampled blocks against the oracle's single-voxel
    re-simulation over all frames (the GPU state must be one it admits).
    Returns the number of voxels checked."""
    vals = blocks.sdf_values()
    assert (blocks.w <= w.max_weight).all()
    assert (vals >= -1.0).all() and (vals <= 1.0).all()
    assert (vals[blocks.w == 0] == 1.0).all()
    p = oracle_params(w, storage)
    intr = oracle_intr(w)
    tol = TOL[storage]
    rng = np.random.default_rng(seed)
    rows = rng.choice(len(blocks.keys), min(n_blocks, len(blocks.keys)), replace=False)
    checked = 0
    for r in rows:
        key = blocks.keys[r].astype(np.int32)
        hits = oracle.block_hit_frames(key, depth, intr, poses, p)
        assert hits.any(), f"GPU block {key.tolist()} is met by no band segment"
        for li in rng.choice(512, n_vox, replace=False):
            vox = key * 8 + np.array([li % 8, (li // 8) % 8, li // 64])
            c = oracle.voxel_candidates(vox, depth, intr, poses, p, hits, max_out=256)
            if c is None:
                continue
            cs, cw = c
            gs, gw = vals[r, li], blocks.w[r, li]
            assert any(cw[i] == gw and abs(cs[i] - gs) <= tol for i in range(len(cs))), \
                (vox.tolist(), gs, gw, list(zip(cs.tolist(), cw.tolist())))
            checked += 1
    return checked


# ---------------------------------------------------------------------------
# raycast (Section 4.4)

# GPU point error allowed on an unflagged pixel: RAY_POS_VOXELS voxels times
# the oracle's per-pixel gain. An FP32 sample position is within ~3e-4
# voxels of the FP64 one (the ulp of coordinates up to ~1000 voxels, the ray
# direction's rounding over the ray's length; the distance along the ray is
# carried as a hi + lo pair); the gain bounds how the march's value-sized
# steps can scale such an error (see or_raycast).
RAY_POS_VOXELS = 1e-3


def storage_arrays(sdf_values, storage):
    """Oracle sdf values (real numbers) -> the raw storage array the CUDA
    scene loads, and the real numbers it then holds (identical for every
    form: int16 values are q / 32767, fp16 values are binary16)."""
    if storage == 1:
        q = np.rint(sdf_values * 32767.0).astype(np.int16)
        return q, q.astype(np.float64) / 32767.0
    if storage == 2:
        h = sdf_values.astype(np.float16)
        return h, h.astype(np.float64)
    f = sdf_values.astype(np.float32)
    return f, f.astype(np.float64)


def ray_params(w, z_near=0.2) -> oracle.RayParams:
    return oracle.RayParams(voxel_size=f32(w.voxel_size), mu=f32(w.mu), z_near=f32(z_near))


def compare_raycast(points, rng, orc, width, height, voxel_size, max_flagged=0.03):
    """GPU points (H, W, 4) and range (H, W, 2) against the oracle's raycast
    of the same volume: on every unflagged pixel the same hit / no hit, the
    same search range (to FP32 rounding of the corner depths) and the point
    within RAY_POS_VOXELS x gain. Returns a report dict."""
    n = width * height
    g = np.asarray(points, np.float64).reshape(n, 4)
    fl = orc["flags"]
    ok = fl == 0
    o_hit = orc["points"][:, 3] == 1.0
    g_hit = g[:, 3] == 1.0
    assert np.isin(g[:, 3], (0.0, 1.0)).all()
    assert (g[~g_hit, :3] == 0.0).all()
    bad_hit = ok & (o_hit != g_hit)
    assert not bad_hit.any(), f"{bad_hit.sum()} unflagged pixels disagree on hit / no hit"
    both = ok & o_hit
    err = np.abs(g[:, :3] - orc["points"][:, :3]).max(axis=1)
    tol = voxel_size * RAY_POS_VOXELS * orc["gain"]
    over = both & (err > tol)
    worst = float(err[both].max()) if both.any() else 0.0
    assert not over.any(), (f"{over.sum()} points beyond tolerance, e.g. error "
                            f"{err[over][:3]} m, gain {orc['gain'][over][:3]}")
    if rng is not None:
        r = np.asarray(rng, np.float64).reshape(n, 2)
        o = orc["range"].reshape(n, 2)
        rok = (orc["range_flags"].reshape(n) == 0)
        fin = np.isfinite(o[:, 0])
        assert np.array_equal(np.isfinite(r[rok, 0]), fin[rok])
        sel = rok & fin
        assert np.allclose(r[sel], o[sel], rtol=1e-6, atol=1e-7)
        assert (np.isposinf(r[rok & ~fin, 0]) & np.isneginf(r[rok & ~fin, 1])).all()
    flagged = float((~ok).mean())
    assert flagged <= max_flagged, f"flagged fraction {flagged}"
    q = np.quantile(err[both] / voxel_size, [0.5, 0.99, 1.0]) if both.any() else np.zeros(3)
    # the bound above is a worst case; nearly every point is within the
    # per-sample error itself
    assert q[1] <= RAY_POS_VOXELS, f"99th percentile point error {q[1]} voxels"
    return dict(pixels=n, hits=int(o_hit.sum()), gpu_hits=int(g_hit.sum()), flagged=flagged,
                worst_point_err_m=worst, max_gain=float(orc["gain"].max()),
                err_voxels_p50=float(q[0]), err_voxels_p99=float(q[1]), err_voxels_max=float(q[2]))


# ---------------------------------------------------------------------------
# depth tracker terms (Section 4.1)

# Error bounds of an FP32 evaluation: a world point (coordinates of a few
# metres) within ICP_P_ERR of the FP64 one; a normal from FP32 central
# differences within ICP_N_ERR (tests/test_gpu_icp.py checks it), so a row's
# rotation part P x N within ICP_P_MAX * ICP_N_ERR + ICP_P_ERR, its
# translation part within ICP_N_ERR, and a residual within ICP_P_ERR +
# max_dist * ICP_N_ERR. Summed over the inliers with Cauchy-Schwarz (sum |x|
# <= sqrt(n sum x^2)), plus 1e-5 of each term's magnitude for the FP32
# products and per-thread sums, plus the oracle's slack for flagged pixels.
ICP_P_ERR = 1e-6
ICP_N_ERR = 1e-4
ICP_P_MAX = 5.0


def _diag_index(a):
    """index of H[a][a] in the row-by-row upper triangle"""
    return sum(6 - i for i in range(a))


def compare_icp(gpu_sums, orc, max_dist=0.1):
    g = np.asarray(gpu_sums, np.float64)
    s, sl, sc = orc["sums"], orc["slack"], orc["scale"]
    n = max(s[28], 1.0)
    dJ = [ICP_P_MAX * ICP_N_ERR + ICP_P_ERR] * 3 + [ICP_N_ERR] * 3
    dr = ICP_P_ERR + max_dist * ICP_N_ERR
    rms = [np.sqrt(n * sc[_diag_index(a)]) for a in range(6)]   # bounds sum |J_a|
    rsum = np.sqrt(n * sc[27])                                   # bounds sum |r|
    tol = 1e-5 * sc + sl
    t = 0
    for a in range(6):
        for b in range(a, 6):
            tol[t] += dJ[a] * rms[b] + dJ[b] * rms[a] + n * dJ[a] * dJ[b]
            t += 1
    for a in range(6):
        tol[21 + a] += dr * rms[a] + dJ[a] * rsum + n * dr * dJ[a]
    tol[27] += 2 * dr * rsum + n * dr * dr
    tol[28] = sl[28]
    err = np.abs(g - s)
    bad = err > tol + 1e-12
    assert not bad.any(), f"terms {np.nonzero(bad)[0]} differ: {err[bad]} > {tol[bad]}"
    return dict(inliers=int(s[28]), gpu_inliers=int(g[28]), flagged=int(orc["flags"].sum()),
                max_err_over_tol=float(np.max(err / (tol + 1e-12))))
