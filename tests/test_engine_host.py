"""Host-side checks of the pipeline engine and the tracker hierarchy that need
no GPU: configuration checks run before any device call, and the intrinsics
of a hierarchy level."""

import ctypes

import numpy as np
import pytest

from paper_1410_0925_gb300 import Icp, make_intrinsics
from paper_1410_0925_gb300.tsdf import (EngineConfig, SceneDesc, TSDF_ERR_INVALID_ARG,
                                        load_library)


def _cfg(**over):
    base = dict(levels=3, iterations=(4, 4, 6), max_dist=0.1, z_near=0.2, colour=0,
                width=640, height=480, swap_blocks=0, swap_margin=16.0)
    base.update(over)
    it = (ctypes.c_int32 * 4)(*(list(base["iterations"]) + [0] * (4 - len(base["iterations"]))))
    return EngineConfig(SceneDesc(0.005, 0.02, 100, 20, 2, 1 << 17, 1 << 18, 0),
                        make_intrinsics(525.0, 525.0, 319.5, 239.5, base["width"], base["height"]),
                        base["levels"], it, base["max_dist"], base["z_near"], base["colour"],
                        base["swap_blocks"], base["swap_margin"])


@pytest.mark.parametrize("over", [dict(levels=0), dict(levels=5), dict(max_dist=0.0),
                                  dict(max_dist=float("nan")), dict(z_near=0.0),
                                  dict(iterations=(101, 0, 0)), dict(iterations=(-1, 0, 0)),
                                  dict(levels=4, width=20, height=20),
                                  dict(swap_blocks=-1), dict(swap_blocks=(1 << 18) + 1),
                                  dict(swap_margin=-1.0), dict(swap_margin=float("inf"))])
def test_engine_rejects_bad_config_without_a_device(over):
    lib = load_library()
    cfg = _cfg(**over)
    h = ctypes.c_void_p()
    pose = np.eye(4)
    rc = lib.tsdf_engine_create(ctypes.byref(cfg), pose.ctypes.data_as(ctypes.c_void_p), None,
                                ctypes.byref(h))
    assert rc == TSDF_ERR_INVALID_ARG and not h.value


def test_engine_rejects_non_affine_initial_pose():
    lib = load_library()
    cfg = _cfg()
    bad = np.eye(4)
    bad[3, 0] = 1.0
    h = ctypes.c_void_p()
    assert lib.tsdf_engine_create(ctypes.byref(cfg), bad.ctypes.data_as(ctypes.c_void_p), None,
                                  ctypes.byref(h)) == TSDF_ERR_INVALID_ARG


def test_level_intrinsics_put_coarse_pixel_centres_on_block_centres():
    intr = make_intrinsics(525.0, 520.0, 319.5, 239.5, 640, 480)
    l2 = Icp.level_intrinsics(intr, 2)
    assert (l2.width, l2.height) == (160, 120)
    # coarse pixel u covers fine pixels 4u..4u+3, centred at 4u + 1.5
    u = np.arange(160, dtype=np.float64)
    assert np.allclose((u - l2.cx) / l2.fx, (4 * u + 1.5 - intr.cx) / intr.fx)
    assert Icp.level_intrinsics(intr, 0).fx == intr.fx
