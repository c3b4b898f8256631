"""The arithmetic the scan's word-wide Gate test rests on (no GPU): for lanes
of W bits that all hold less than 2^(W-1), adding 2^(W-1) - t to every lane
of a 32-bit word sets a lane's top bit exactly when that lane holds t or more,
with no carry into the next lane.  The GPU parity tests check the kernel end
to end on both sides of the headroom limit; this checks the identity itself,
exhaustively where the space is small."""
import numpy as np
import pytest


def lanes(words, w):
    per = 32 // w
    mask = (1 << w) - 1
    return np.stack([(words >> (w * i)) & mask for i in range(per)], axis=-1)


def word_test(words, w, t):
    per = 32 // w
    ones = sum(1 << (w * i) for i in range(per))
    high = ones << (w - 1)
    add = (high - t * ones) & 0xFFFFFFFF
    return (words + np.uint64(add)) & 0xFFFFFFFF & high


@pytest.mark.parametrize("w", [4, 8, 16])
def test_top_bits_mark_exactly_the_lanes_at_or_above_t(w):
    rng = np.random.default_rng(w)
    half = 1 << (w - 1)
    if w == 4:  # every 4-bit-lane word with headroom in its low 16 bits, the rest random
        lo = np.arange(1 << 16, dtype=np.uint64)
        lo = lo[np.all(lanes(lo, 4)[:, :4] < half, axis=1)]
        hi = lanes(rng.integers(0, 1 << 16, lo.size).astype(np.uint64), 4)[:, :4] % half
        hi_w = sum(hi[:, i].astype(np.uint64) << np.uint64(4 * i) for i in range(4))
        words = lo | (hi_w << np.uint64(16))
    else:
        per = 32 // w
        vals = rng.integers(0, half, (50_000, per)).astype(np.uint64)
        vals[:1000] = half - 1  # lanes at the headroom limit
        vals[1000:2000] = 0
        words = sum(vals[:, i] << np.uint64(w * i) for i in range(per))
    l = lanes(words, w)
    ts = range(0, half + 1) if w < 16 else sorted(
        set(range(0, 66)) | set(range(half - 65, half + 1)) |
        set(int(x) for x in rng.integers(0, half + 1, 64)))
    for t in ts:
        got = word_test(words, w, t)
        top = lanes(got, w) >> (w - 1)  # the top bit of each lane of the sum
        assert np.array_equal(top, (l >= t).astype(top.dtype)), t


@pytest.mark.parametrize("w", [4, 8, 16])
def test_without_headroom_a_carry_can_cross_lanes(w):
    # a lane at 2^W - 1 overflows into its neighbour: why the kernel tests
    # each posting's own lane when the bound does not leave the top bit free
    per = 32 // w
    full = (1 << w) - 1
    words = np.array([full], dtype=np.uint64)
    got = word_test(words, w, 1)
    expect = np.array([[1] + [0] * (per - 1)])
    assert not np.array_equal(lanes(got, w) >> (w - 1), expect)
