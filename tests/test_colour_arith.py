"""The colour average's integer decision, checked over every input.

The oracle evaluates a channel's new value as the listing does, in float:
floor(fl(fl(N / D) + 1/2)) with N = w c + o and D = w + 1 (w the colour
weight, c the stored channel, o the observation, all 0..255). The CUDA
kernel computes the same integer as umulhi(2N + D, ceil(2^32 / (2D))). Both
must equal the exact floor((2N + D) / (2D)) for all 256^3 inputs; this test
enumerates them.
"""

import numpy as np


def test_float_average_equals_integer_rounding_for_every_input():
    c = np.arange(256, dtype=np.int64)[:, None]
    o = np.arange(256, dtype=np.int64)[None, :]
    for w in range(256):
        D = w + 1
        N = w * c + o                                        # exact integer
        exact = (2 * N + D) // (2 * D)
        x = N.astype(np.float32) / np.float32(D)              # IEEE single division
        fp = np.floor(x + np.float32(0.5)).astype(np.int64)   # single add, then floor
        assert np.array_equal(fp, exact), f"float rounding differs at w={w}"
        m = np.uint64(0xFFFFFFFF // (2 * D) + 1)              # ceil(2^32 / (2D))
        hi = ((2 * N + D).astype(np.uint64) * m) >> np.uint64(32)
        assert np.array_equal(hi.astype(np.int64), exact), f"umulhi differs at w={w}"
        assert exact.max() <= 255
