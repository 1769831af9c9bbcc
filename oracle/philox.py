"""Philox4x64-10 and the samplers that draw the BFV randomness.

Philox4x64-10 is the counter-based generator of Salmon, Moraes, Dror and Shaw,
"Parallel random numbers: as easy as 1, 2, 3" (SC'11): ten rounds, each
multiplying words 0 and 2 by fixed 64-bit constants and mixing the high and
low halves with words 1 and 3 and the round key; the key is bumped by two
Weyl constants between rounds.  The paper under study is silent on its
randomness (it delegates to SEAL); this build's reading fixes:

    key     = (seed, purpose)
    counter = (block, poly, limb, kind)

* uniform residue mod q for (poly, limb, coefficient n):
  block = n >> 1, kind = 0; the two words w_lo = out[2(n&1)], w_hi =
  out[2(n&1)+1] give (w_hi * 2^64 + w_lo) mod q (bias < 2^-78);
* small samples for (poly, coefficient n): block = n >> 2, limb = 0, kind = 1,
  w = out[n & 3]; ternary = {0, 1, -1}[w mod 3]; centred binomial CBD(21) =
  popcount(w & (2^21-1)) - popcount((w >> 21) & (2^21-1)).
"""

MASK = (1 << 64) - 1
M0 = 0xD2E7470EE14C6C93
M1 = 0xCA5A826395121157
W0 = 0x9E3779B97F4A7C15
W1 = 0xBB67AE8584CAA73B

# purposes
SK, PK_A, PK_E, RLK_A, RLK_E, ENC_U, ENC_E1, ENC_E2 = 1, 2, 3, 4, 5, 6, 7, 8


def philox4x64(ctr, key, rounds=10):
    """One Philox4x64 block: four 64-bit words from a 4-word counter and 2-word key."""
    c0, c1, c2, c3 = ctr
    k0, k1 = key
    for r in range(rounds):
        if r:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0
        p1 = M1 * c2
        c0, c1, c2, c3 = ((p1 >> 64) ^ c1 ^ k0, p1 & MASK, (p0 >> 64) ^ c3 ^ k1, p0 & MASK)
    return [c0, c1, c2, c3]


def uniform_poly(seed, purpose, poly, limb, q, N):
    """N residues uniform mod q for (poly, limb)."""
    out = [0] * N
    for blk in range((N + 1) // 2):
        w = philox4x64((blk, poly, limb, 0), (seed, purpose))
        for h in range(2):
            n = 2 * blk + h
            if n < N:
                out[n] = ((w[2 * h + 1] << 64) | w[2 * h]) % q
    return out


def _small_words(seed, purpose, poly, N):
    out = [0] * N
    for blk in range((N + 3) // 4):
        w = philox4x64((blk, poly, 0, 1), (seed, purpose))
        for h in range(4):
            n = 4 * blk + h
            if n < N:
                out[n] = w[h]
    return out


def ternary_poly(seed, purpose, poly, N):
    """N coefficients in {-1, 0, 1}: word mod 3 mapped 0->0, 1->1, 2->-1."""
    return [(0, 1, -1)[w % 3] for w in _small_words(seed, purpose, poly, N)]


def cbd_poly(seed, purpose, poly, N, eta=21):
    """N centred-binomial samples with parameter eta (variance eta/2)."""
    m = (1 << eta) - 1
    return [bin(w & m).count("1") - bin((w >> eta) & m).count("1")
            for w in _small_words(seed, purpose, poly, N)]
