"""Pins for the oracle's number theory, parameter rule, generator and products.

Each test checks the oracle against something other than itself: sympy's
primality test and CRT, numpy's Philox bit generator and convolution, the
O(N^2) definition of the negacyclic product, or a closed form.
"""

import random

import numpy as np
import pytest
import sympy

from oracle import nt, philox as px
from oracle.params import Params, scan_primes
from oracle.poly import linear_product, negacyclic, negacyclic_schoolbook


# ------------------------------------------------------------ number theory
def test_is_prime_matches_sympy():
    rng = random.Random(1)
    cases = [0, 1, 2, 3, 4, 561, 1105, 1729, 2465, 2821, 6601, 8911,   # Carmichael
             3215031751, 2152302898747, 3474749660383, 341550071728321,  # strong pseudoprimes
             (1 << 61) - 1, (1 << 64) - 59, (1 << 50) - 27]
    cases += [rng.randrange(1 << 64) for _ in range(3000)]
    cases += [rng.randrange(1 << 50) | 1 for _ in range(3000)]
    for n in cases:
        assert nt.is_prime(n) == sympy.isprime(n), n


def test_crt_and_centered():
    rng = random.Random(2)
    mods = [1000003, 998244353, 1000000007]
    for _ in range(200):
        r = [rng.randrange(m) for m in mods]
        x = nt.crt(r, mods)
        y, M = sympy.ntheory.modular.crt(mods, r)
        assert x == int(y) and 0 <= x < int(M)
    M = 15
    assert [nt.centered(x, M) for x in range(M)] == [0, 1, 2, 3, 4, 5, 6, 7, -7, -6, -5, -4, -3, -2, -1]


def test_least_primitive_root():
    for p in (17, 257, 65537, 97, 7681, 12289):
        g = nt.least_primitive_root(p)
        assert sympy.ntheory.primitive_root(p) == g


@pytest.mark.parametrize("N,bits", [(8, 20), (16, 24), (4096, 50)])
def test_scan_primes_is_the_downward_scan(N, bits):
    ps = scan_primes(N, 6, bits)
    assert ps == sorted(ps, reverse=True) and len(set(ps)) == 6
    for q in ps:
        assert sympy.isprime(q) and q % (2 * N) == 1 and q < (1 << bits)
    # no prime of the form 2Nk+1 was skipped between 2^bits and the last one found
    if bits <= 24:
        allq = [q for q in range(ps[-1], 1 << bits) if q % (2 * N) == 1 and sympy.isprime(q)]
        assert sorted(allq, reverse=True) == ps


@pytest.mark.parametrize("cfg", [dict(N=4096, L=2, alpha=1), dict(N=16384, L=8, alpha=1),
                                 dict(N=32768, L=16, alpha=2), dict(N=8, L=3, alpha=1, t=17, prime_bits=40)])
def test_params_rule(cfg):
    prm = Params(**cfg)
    allp = prm.q + prm.p + prm.b
    assert len(set(allp)) == len(allp) and prm.t not in allp
    assert allp == scan_primes(prm.N, len(allp), prm.prime_bits, exclude=(prm.t,))
    assert prm.B > 2 * prm.t * prm.N * prm.Q
    assert nt.prod(prm.b[:-1]) <= 2 * prm.t * prm.N * prm.Q      # K is minimal
    assert prm.delta == prm.Q // prm.t
    # zeta is a primitive 2N-th root of unity mod t
    assert pow(prm.zeta, prm.N, prm.t) == prm.t - 1


def test_params_reject_bad_input():
    with pytest.raises(ValueError):
        Params(N=4096, L=2, alpha=1, t=65539)          # t != 1 mod 2N
    with pytest.raises(ValueError):
        Params(N=100, L=2, alpha=1)


# ------------------------------------------------------------ Philox4x64-10
@pytest.mark.parametrize("key", [(0, 0), (1, 6), (0xDEADBEEF, 2), ((1 << 64) - 1, (1 << 64) - 1)])
def test_philox_matches_numpy(key):
    rng = random.Random(3)
    for _ in range(20):
        ctr = [rng.randrange(1 << 64) for _ in range(3)] + [rng.randrange(1 << 63)]
        g = np.random.Philox(counter=np.array(ctr, dtype=np.uint64), key=np.array(key, dtype=np.uint64))
        got = [int(x) for x in g.random_raw(8)]
        # numpy advances the 256-bit counter before each block
        c1 = list(ctr)
        c1[0] = (c1[0] + 1) & px.MASK
        if c1[0] == 0:
            continue
        c2 = list(c1)
        c2[0] = (c2[0] + 1) & px.MASK
        if c2[0] == 0:
            continue
        assert got == px.philox4x64(c1, key) + px.philox4x64(c2, key)


def test_samplers_statistics():
    N = 1 << 14
    q = (1 << 50) - 27
    u = px.uniform_poly(9, px.PK_A, 0, 0, q, N)
    assert all(0 <= x < q for x in u)
    assert abs(np.mean(np.array(u, dtype=np.float64)) / q - 0.5) < 0.02
    tern = px.ternary_poly(9, px.SK, 0, N)
    counts = [tern.count(v) for v in (-1, 0, 1)]
    assert all(abs(c / N - 1 / 3) < 0.02 for c in counts)
    e = np.array(px.cbd_poly(9, px.PK_E, 0, N))
    assert e.min() >= -21 and e.max() <= 21
    assert abs(e.mean()) < 0.1 and abs(e.var() - 10.5) < 0.6
    # different purposes / polys / limbs give different streams
    assert px.uniform_poly(9, px.PK_A, 0, 1, q, 16) != px.uniform_poly(9, px.PK_A, 0, 0, q, 16)
    assert px.ternary_poly(9, px.SK, 1, 64) != px.ternary_poly(9, px.SK, 0, 64)


def test_sampler_word_layout():
    """Coefficient n takes words (2(n&1), 2(n&1)+1) of block n>>1 (uniform), word n&3 of block n>>2 (small)."""
    seed, q = 77, 1000003
    w = px.philox4x64((3, 5, 2, 0), (seed, px.RLK_A))
    u = px.uniform_poly(seed, px.RLK_A, 5, 2, q, 8)
    assert u[6] == ((w[1] << 64) | w[0]) % q and u[7] == ((w[3] << 64) | w[2]) % q
    w = px.philox4x64((1, 4, 0, 1), (seed, px.ENC_U))
    t = px.ternary_poly(seed, px.ENC_U, 4, 8)
    assert t[4:8] == [(0, 1, -1)[x % 3] for x in w]


# ------------------------------------------------------------ products in Z[X]/(X^N+1)
@pytest.mark.parametrize("N", [1, 2, 8, 16, 64])
def test_negacyclic_matches_schoolbook(N):
    rng = random.Random(N)
    for bits in (1, 20, 130):
        for _ in range(5):
            a = [rng.randrange(-(1 << bits), 1 << bits) for _ in range(N)]
            b = [rng.randrange(-(1 << bits), 1 << bits) for _ in range(N)]
            assert negacyclic(a, b) == negacyclic_schoolbook(a, b)
    z = [0] * N
    assert negacyclic(z, [1] * N) == z
    big = [rng.randrange(1 << 300) for _ in range(N)]
    assert negacyclic(z, big) == z and negacyclic(big, z) == z


def test_negacyclic_monomials():
    """X^i * X^j = X^(i+j) if i+j < N, else -X^(i+j-N)."""
    N = 16
    for i in range(N):
        for j in range(N):
            a = [0] * N
            b = [0] * N
            a[i] = 3
            b[j] = -5
            r = negacyclic(a, b)
            e = [0] * N
            if i + j < N:
                e[i + j] = -15
            else:
                e[i + j - N] = 15
            assert r == e


def test_linear_product_matches_numpy():
    rng = np.random.default_rng(4)
    for n, m in ((1, 1), (7, 3), (50, 50)):
        a = rng.integers(-1000, 1000, n)
        b = rng.integers(-1000, 1000, m)
        assert linear_product([int(x) for x in a], [int(x) for x in b]) == [int(x) for x in np.convolve(a, b)]
