"""The pencil and slab passes sum x_HI in 2^-23 fixed point, rounding each cell's x_HI with one
fused multiply-add: v 2^23 + 2^23 (in [2^23, 2^24], where float spacing is 1) rounded once to
float32 has the bits of 2^23 plus round-half-even(v 2^23). Checked here in NumPy on float32
values of [0, 1], including every tie and the end points, against np.rint (round half even)."""
import numpy as np


def fixed23(v):
    exact = v.astype(np.float64) * 8388608.0 + 8388608.0       # exact in float64 (v has 24 bits)
    f = exact.astype(np.float32)                                # one rounding, as the FMA's
    return f.view(np.int32).astype(np.int64) - 0x4B000000


def test_fixed23_matches_round_half_even():
    rng = np.random.default_rng(5)
    v = np.concatenate([
        rng.random(200000, dtype=np.float32),
        np.float32([0.0, 1.0, 0.5, 2.0 ** -23, 2.0 ** -24, 3 * 2.0 ** -25, 1.0 - 2.0 ** -24]),
        (np.arange(0, 4096, dtype=np.float64) * 2.0 ** -24 + 2.0 ** -25).astype(np.float32),   # ties
    ]).astype(np.float32)
    v = v[(v >= 0) & (v <= 1)]
    ref = np.rint(v.astype(np.float64) * 8388608.0).astype(np.int64)
    np.testing.assert_array_equal(fixed23(v), ref)
