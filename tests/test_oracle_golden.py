"""Oracle pinned to hand-derived cases of the report's definitions.

Each case in tests/golden/update_rule_cases.json was worked out by hand from
the integration listing (Section 4.3), the allocation band (Section 4.2) and
the voxel storage listing (Section 3.1); see the "why" field of each case.
"""

import json
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "update_rule_cases.json")
with open(GOLDEN) as f:
    SPEC = json.load(f)
SETUP = SPEC["setup"]


def _depth_image(spec):
    W, H = SETUP["width"], SETUP["height"]
    if isinstance(spec, dict):
        img = np.full((H, W), spec["default"], np.float32)
        for col, val in spec["columns"].items():
            img[:, int(col)] = val
        return img
    val = float("nan") if spec == "nan" else float(spec)
    return np.full((H, W), val, np.float32)


def _lookup(res, voxel):
    v = np.asarray(voxel)
    key = np.floor_divide(v, 8)
    local = v - 8 * key
    li = local[0] + 8 * local[1] + 64 * local[2]
    hit = np.nonzero((res["keys"] == key).all(axis=1))[0]
    if len(hit) == 0:
        return None
    b = hit[0]
    return res["sdf"][b, li], int(res["w"][b, li])


@pytest.mark.parametrize("case", SPEC["cases"], ids=[c["name"] for c in SPEC["cases"]])
def test_hand_derived_case(case):
    p = oracle.OracleParams(voxel_size=SETUP["voxel_size"], mu=SETUP["mu"],
                            max_weight=case["max_weight"], storage=case["storage"])
    o = oracle.Oracle(p)
    pose = np.asarray(case.get("pose", np.eye(4)), dtype=np.float64)
    intr = (SETUP["fx"], SETUP["fy"], SETUP["cx"], SETUP["cy"])
    for d in case["depths"]:
        o.integrate(_depth_image(d), intr, pose)
    res = o.read()
    for e in case["expect"]:
        got = _lookup(res, e["voxel"])
        if not e["allocated"]:
            assert got is None, f"{e['voxel']} should not be allocated"
            continue
        assert got is not None, f"{e['voxel']} should be allocated"
        sdf, w = got
        assert w == e["w"]
        assert math.isclose(sdf, e["sdf"], rel_tol=0, abs_tol=1e-12), (sdf, e["sdf"])


def test_fixed_point_identities():
    """Section 3.1: initial value 32767 is 1.0; conversion truncates."""
    assert oracle.i16_to_float(32767) == 1.0
    assert oracle.float_to_i16(1.0) == 32767
    assert oracle.float_to_i16(-1.0) == -32767
    assert oracle.float_to_i16(0.99999) == 32766          # 32766.67 -> 32766
    assert oracle.float_to_i16(-0.99999) == -32766        # toward zero
    assert oracle.float_to_i16(0.5 / 32767) == 0
    assert oracle.float_to_i16(-0.5 / 32767) == 0
    assert oracle.float_to_i16(0.5) == 16383              # 16383.5 -> 16383


def test_fixed_point_matches_numpy_cast():
    """trunc-toward-zero conversion equals numpy's float->int16 cast."""
    rng = np.random.default_rng(5)
    xs = np.concatenate([rng.uniform(-1, 1, 2000), np.linspace(-1, 1, 401)])
    want = (xs * 32767.0).astype(np.int16)
    got = np.array([oracle.float_to_i16(x) for x in xs], np.int16)
    assert np.array_equal(got, want)


def test_half_rounding_matches_numpy_float16():
    """FP16 storage rounding equals numpy's IEEE binary16 conversion,
    including ties, subnormals and values near 1."""
    rng = np.random.default_rng(6)
    xs = [0.0, 1.0, -1.0, 1.0 / 6.0, 2.0 ** -24, 2.0 ** -25, 3 * 2.0 ** -25,
          2.0 ** -14, 1 - 2.0 ** -12, 1 - 3 * 2.0 ** -12]
    xs += list(rng.uniform(-1, 1, 3000)) + list(rng.uniform(-1e-4, 1e-4, 1000))
    for x in xs:
        assert oracle.round_f16(x) == float(np.float16(x)), x
