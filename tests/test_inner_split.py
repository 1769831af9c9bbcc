"""Host check of the key-switch inner product's split accumulation (every prime below 2^50).

The kernel cuts each digit a < 2^56 and key word b < 2^50 at bit 28 and accumulates
sum al bl, sum (al bh + ah bl), sum ah bh in 64-bit registers, then joins them into a 128-bit
(hi, lo).  This replays that arithmetic with 64-bit wrap-around at the operand extremes and checks
that no accumulator overflows and that the join equals the exact sum of products.
"""

import random

import pytest

M64 = (1 << 64) - 1
M28 = (1 << 28) - 1


def join28(sl, sm, sh):
    mlo, hlo = (sm << 28) & M64, (sh << 56) & M64
    r = (sl + mlo) & M64
    c = 1 if r < mlo else 0
    lo = (r + hlo) & M64
    c += 1 if lo < hlo else 0
    hi = ((sm >> 36) + (sh >> 8) + c) & M64
    return hi, lo


def split_sum(a, b):
    sl = sm = sh = 0
    for x, y in zip(a, b):
        al, ah = x & M28, x >> 28
        bl, bh = y & M28, y >> 28
        assert ah < 1 << 28 and bh < 1 << 22
        sl += al * bl
        sm += al * bh + ah * bl
        sh += ah * bh
        assert max(sl, sm, sh) <= M64     # the 64-bit accumulators never wrap
    return join28(sl, sm, sh)


@pytest.mark.parametrize("L", [1, 2, 8, 16])
def test_split_accumulation_equals_the_exact_sum(L):
    rng = random.Random(L)
    cases = [([(1 << 56) - 1] * L, [(1 << 50) - 1] * L), ([0] * L, [0] * L)]
    for _ in range(300):
        cases.append(([rng.randrange(1 << 56) for _ in range(L)], [rng.randrange(1 << 50) for _ in range(L)]))
    for a, b in cases:
        hi, lo = split_sum(a, b)
        z = sum(x * y for x, y in zip(a, b))
        assert (hi << 64) | lo == z
