"""The readback entry point that allocates nothing.

tsdf_read_blocks_device_noalloc serves callers that cannot call cudaMalloc
when they read a scene back (real-time loops that must not take the
allocator's locks or its implicit device synchronisation, frameworks whose
caching pool owns the device memory): its sort scratch is a fixed array in
the library's device image. Here it is called through the C ABI, twice in a
row on the same scene, in every storage form, and must give exactly what
tsdf_read_blocks gives. This file is collected last on purpose.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _fused_scene(storage):
    import torch
    from paper_1410_0925_gb300 import Scene, make_intrinsics
    from synthdepth import make_sequence, workload_tiny
    w = workload_tiny(storage=storage)
    seq = make_sequence(w, n_frames=6)
    scene = Scene.from_workload(w)
    intr = make_intrinsics(w.fx, w.fy, w.cx, w.cy, w.width, w.height)
    depth = torch.from_numpy(seq.depth).cuda()
    for i in range(depth.shape[0]):
        scene.integrate(depth[i], intr, seq.poses[i])
    return scene


@pytest.mark.parametrize("storage", [0, 1, 2])
def test_noalloc_readback_equals_read_blocks_twice(storage):
    import torch
    from paper_1410_0925_gb300.tsdf import load_library
    lib = load_library()
    scene = _fused_scene(storage)
    ref = scene.read_blocks()
    n = len(ref.keys)
    assert n > 1000
    sdf_t = {0: torch.float32, 1: torch.int16, 2: torch.float16}[storage]
    for _ in range(2):
        keys = torch.full((n, 3), -7, dtype=torch.int16, device="cuda")
        sdf = torch.zeros((n, 512), dtype=sdf_t, device="cuda")
        w = torch.full((n, 512), 9, dtype=torch.uint8, device="cuda")
        written = ctypes.c_int64()
        rc = lib.tsdf_read_blocks_device_noalloc(
            ctypes.c_void_p(scene.handle), ctypes.c_void_p(keys.data_ptr()),
            ctypes.c_void_p(sdf.data_ptr()), ctypes.c_void_p(w.data_ptr()), n,
            ctypes.byref(written))
        assert rc == 0 and written.value == n
        assert np.array_equal(keys.cpu().numpy(), ref.keys)
        assert np.array_equal(w.cpu().numpy(), ref.w)
        assert np.array_equal(sdf.cpu().numpy().view(ref.sdf.dtype), ref.sdf)


def test_noalloc_readback_rejects_small_buffers_and_oversized_scenes():
    import torch
    from paper_1410_0925_gb300 import Blocks, Scene, TsdfError
    from paper_1410_0925_gb300.tsdf import READ_NOALLOC_MAX_BLOCKS
    scene = _fused_scene(0)
    n = scene.num_blocks()
    small = n - 1
    with pytest.raises(TsdfError):
        scene.read_blocks_device_noalloc(
            torch.zeros((small, 3), dtype=torch.int16, device="cuda"),
            torch.zeros((small, 512), dtype=torch.float32, device="cuda"),
            torch.zeros((small, 512), dtype=torch.uint8, device="cuda"))
    # a scene with more blocks than the fixed scratch holds is refused
    m = READ_NOALLOC_MAX_BLOCKS + 1
    big = Scene(voxel_size=0.01, mu=0.04, hash_buckets_log2=20, excess_entries=1 << 17,
                pool_blocks=1 << 19, storage=1)
    i = np.arange(m)
    keys = np.stack([i % 128 - 64, (i // 128) % 128 - 64, i // 16384 - 8], 1).astype(np.int16)
    big.load_blocks(Blocks(keys, np.full((m, 512), 32767, np.int16), np.zeros((m, 512), np.uint8)))
    assert big.num_blocks() == m
    # (no sdf or weight buffers: a refusal must come from the block count)
    with pytest.raises(TsdfError):
        big.read_blocks_device_noalloc(
            torch.zeros((m, 3), dtype=torch.int16, device="cuda"), None, None)


def test_noalloc_wrapper_checks_the_buffers():
    """The Python wrapper refuses buffers of the wrong shape, dtype or
    layout before the C function runs."""
    import torch
    from paper_1410_0925_gb300 import TsdfError
    scene = _fused_scene(0)
    n = scene.num_blocks()
    keys = torch.zeros((n, 3), dtype=torch.int16, device="cuda")
    good_sdf = torch.zeros((n, 512), dtype=torch.float32, device="cuda")
    good_w = torch.zeros((n, 512), dtype=torch.uint8, device="cuda")
    bad = [(keys, torch.zeros((n - 1, 512), dtype=torch.float32, device="cuda"), good_w),
           (keys, torch.zeros((n, 512), dtype=torch.int16, device="cuda"), good_w),
           (keys, good_sdf, torch.zeros((n, 256), dtype=torch.uint8, device="cuda")),
           (keys, torch.zeros((512, n), dtype=torch.float32, device="cuda").t(), good_w),
           (keys, good_sdf.cpu(), good_w)]
    for k, sdf, w in bad:
        with pytest.raises(TsdfError):
            scene.read_blocks_device_noalloc(k, sdf, w)
    assert scene.read_blocks_device_noalloc(keys, good_sdf, good_w) == n
