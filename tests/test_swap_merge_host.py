"""The swap-in kernel's secondary integration, compiled for the host
(tsdf_swap_merge_voxels; no GPU needed), against the oracle's merge
(Section 5): int16 and colour bit for bit (both are integer arithmetic),
float within the FP32 rounding of the weighted mean, FP16 the nearest
binary16 of that mean; empty sides and the weight cap on every storage."""

import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module")
def lib():
    from paper_1410_0925_gb300 import build
    build.build()
    from paper_1410_0925_gb300.tsdf import load_library
    return load_library()


def _weights(rng, n):
    w = rng.integers(0, 101, n)
    w[rng.random(n) < 0.1] = 0
    w[rng.random(n) < 0.1] = 100
    return w.astype(np.uint8)


def _params(storage, max_w=100):
    return oracle.OracleParams(voxel_size=0.01, mu=0.04, max_weight=max_w, storage=storage)


@pytest.mark.parametrize("storage", [0, 1, 2])
def test_merge_matches_the_oracle(lib, storage):
    from paper_1410_0925_gb300 import swap_merge_voxels
    rng = np.random.default_rng(11 + storage)
    n = 6000
    wh, wd = _weights(rng, n), _weights(rng, n)
    if storage == 0:
        hs = rng.uniform(-1, 1, n).astype(np.float32)
        ds = rng.uniform(-1, 1, n).astype(np.float32)
        val = lambda a: a.astype(np.float64)  # noqa: E731
    elif storage == 1:
        hs = rng.integers(-32767, 32768, n).astype(np.int16)
        ds = rng.integers(-32767, 32768, n).astype(np.int16)
        val = lambda a: a.astype(np.float64) / 32767.0  # noqa: E731
    else:
        hs = rng.uniform(-1, 1, n).astype(np.float16)
        ds = rng.uniform(-1, 1, n).astype(np.float16)
        val = lambda a: a.astype(np.float64)  # noqa: E731
    for max_w in (100, 37):
        gs, gw, _ = swap_merge_voxels(storage, max_w, hs, wh, ds, wd)
        p = _params(storage, max_w)
        gv = val(gs)
        for i in range(n):
            f, w = oracle.swap_merge_voxel(p, val(hs[i:i + 1])[0], int(wh[i]),
                                           val(ds[i:i + 1])[0], int(wd[i]))
            assert gw[i] == w, (i, wh[i], wd[i], gw[i], w)
            if storage == 1:
                assert gs[i] == round(f * 32767), (i, gs[i], f * 32767)
            elif storage == 0:
                assert abs(gv[i] - f) <= 2.4e-7, (i, gv[i], f)
            else:
                # the FP32 mean rounded once more to binary16: within half an
                # ulp of the oracle's own nearest binary16, one ulp at most
                assert abs(gv[i] - f) <= 2.0 ** -11 * max(abs(f), 2.0 ** -14) * 2, (i, gv[i], f)
        # empty sides return the other side bit for bit
        e = wh == 0
        assert np.array_equal(gs[e].view(np.uint8), ds[e].view(np.uint8)) and np.array_equal(gw[e], wd[e])
        e = (wd == 0) & (wh > 0)
        assert np.array_equal(gs[e].view(np.uint8), hs[e].view(np.uint8)) and np.array_equal(gw[e], wh[e])


def test_colour_merge_is_bit_exact_over_every_channel_pair(lib):
    from paper_1410_0925_gb300 import swap_merge_voxels
    a, b = np.meshgrid(np.arange(256, dtype=np.uint32), np.arange(256, dtype=np.uint32))
    a, b = a.ravel(), b.ravel()
    n = len(a)
    zeros = np.zeros(n, np.float32)
    ones = np.ones(n, np.uint8)
    p = _params(0)
    for wh, wd in ((1, 1), (3, 7), (100, 100), (0, 5), (9, 0)):
        hw = (a | (b << 8) | (((a + b) % 256) << 16) | np.uint32(wh << 24)).astype(np.uint32)
        dw = (b | (a << 8) | (((a * 7) % 256) << 16) | np.uint32(wd << 24)).astype(np.uint32)
        _, _, got = swap_merge_voxels(0, 100, zeros, ones, zeros, ones, hw, dw)
        # the oracle on a sample of the pairs (every 97th) and on the corners
        idx = np.concatenate([np.arange(0, n, 97), [0, 255, n - 256, n - 1]])
        for i in idx:
            h = np.array([hw[i] >> (8 * c) & 255 for c in range(4)], np.uint8)
            d = np.array([dw[i] >> (8 * c) & 255 for c in range(4)], np.uint8)
            want = oracle.swap_merge_colour(p, h, d)
            have = np.array([got[i] >> (8 * c) & 255 for c in range(4)], np.uint8)
            assert np.array_equal(have, want), (wh, wd, h, d, have, want)
        # the closed form on every pair: (2 (w_h x + w_d y) + w) / (2 w), w = w_h + w_d
        if wh and wd:
            w = wh + wd
            r = (got & 255).astype(np.int64)
            assert np.array_equal(r, (2 * (wh * a.astype(np.int64) + wd * b) + w) // (2 * w))
            assert ((got >> 24) == min(w, 100)).all()


def test_merge_rejects_bad_arguments(lib):
    from paper_1410_0925_gb300 import TsdfError, swap_merge_voxels
    x = np.zeros(3, np.float32)
    w = np.zeros(3, np.uint8)
    with pytest.raises(TsdfError):
        swap_merge_voxels(3, 100, x, w, x, w)
    with pytest.raises(TsdfError):
        swap_merge_voxels(0, 0, x, w, x, w)
    with pytest.raises(TsdfError):
        swap_merge_voxels(0, 256, x, w, x, w)
