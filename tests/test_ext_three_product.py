"""Host check of the fast extension's three-product limb sums in scale-and-round.

Each term y c (y, c < 2^50) is cut into 26-bit limbs; the weight-2^26 part is recovered as
sum (y0 + y1)(c0 + c1) - sum y0 c0 - sum y1 c1.  This replays the 64-bit sums at the operand extremes
and at random for 1 to 17 sources (scale-and-round extends from up to 17), checks that none wraps, that
the middle part equals sum (y0 c1 + y1 c0), and that the joined 128-bit value is the exact sum.
"""

import random

import pytest

M64 = (1 << 64) - 1
M26 = (1 << 26) - 1


def join(p00, mid, p11):
    lo = (p00 + ((mid << 26) & M64)) & M64
    hi = ((mid >> 38) + (1 if lo < p00 else 0)) & M64
    top = (p11 << 52) & M64
    lo2 = (lo + top) & M64
    hi = (hi + (p11 >> 12) + (1 if lo2 < top else 0)) & M64
    return (hi << 64) | lo2


@pytest.mark.parametrize("S", [1, 8, 9, 16, 17])
def test_three_product_sums_equal_the_exact_sum(S):
    rng = random.Random(S)
    cases = [([(1 << 50) - 1] * S, [(1 << 50) - 1] * S), ([0] * S, [0] * S)]
    cases += [([rng.randrange(1 << 50) for _ in range(S)], [rng.randrange(1 << 50) for _ in range(S)])
              for _ in range(300)]
    for ys, cs in cases:
        p00 = p11 = pm = cross = 0
        for y, c in zip(ys, cs):
            y0, y1, c0, c1 = y & M26, y >> 26, c & M26, c >> 26
            p00 += y0 * c0
            p11 += y1 * c1
            pm += (y0 + y1) * (c0 + c1)
            cross += y0 * c1 + y1 * c0
            assert max(p00, p11, pm) <= M64
        mid = (pm - p00 - p11) & M64
        assert mid == cross
        assert join(p00, mid, p11) == sum(y * c for y, c in zip(ys, cs))
