"""Pins for the oracle's BFV: batching, keys, encryption and the exact multiply.

The checks are the defining properties of each step rather than retyped
formulas: slot evaluation by brute force, the ring isomorphism behind
batching, the key relations, decrypt(encrypt(m)) = m, homomorphic add and
multiply against plaintext arithmetic mod t, the nearest-integer property of
both roundings, and the three-component decryption of an unrelinearised
product.
"""

import random
from fractions import Fraction

import pytest

from oracle import bfv
from oracle import philox as px
from oracle.nt import centered, inv
from oracle.params import Params
from oracle.poly import negacyclic

TINY = dict(N=8, L=3, alpha=1, t=17, prime_bits=40)
SMALL = dict(N=64, L=3, alpha=1, t=257, prime_bits=50)


def _brute_eval(prm, m):
    t = prm.t
    return [sum(mk * pow(prm.zeta, (2 * j + 1) * k, t) for k, mk in enumerate(m)) % t
            for j in range(prm.N)]


@pytest.mark.parametrize("cfg", [TINY, dict(N=128, L=1, alpha=1, t=257, prime_bits=40)])
def test_decode_is_evaluation_at_odd_roots(cfg):
    prm = Params(**cfg)
    rng = random.Random(1)
    for _ in range(3):
        m = [rng.randrange(prm.t) for _ in range(prm.N)]
        assert bfv.decode_poly(prm, m) == _brute_eval(prm, m)
        y = [rng.randrange(prm.t) for _ in range(prm.N)]
        mm = bfv.encode_slots(prm, y)
        assert all(0 <= x < prm.t for x in mm)
        assert _brute_eval(prm, mm) == y


# the largest plaintext moduli the library accepts: primes t = 1 mod 2048 just below 2^31 and 2^32;
# at the second, (t - 1)^2 exceeds 2^63, so a product or a sum of products in int64 would wrap
LARGE_T = (2147473409, 4294957057)


def _brute_eval_table(prm, m):
    """y_j = sum_k m_k zeta^((2j+1)k) mod t with Python integers (no overflow), powers from a table."""
    t, N = prm.t, prm.N
    zp = [pow(prm.zeta, e, t) for e in range(2 * N)]
    return [sum(mk * zp[(2 * j + 1) * k % (2 * N)] for k, mk in enumerate(m)) % t for j in range(N)]


@pytest.mark.parametrize("t", LARGE_T)
def test_slot_transforms_are_exact_at_large_t(t):
    """Sec. 2.3 batching at the largest t below 2^32: decode against big-integer evaluation, encode as its
    inverse, with inputs near t - 1 where products are largest."""
    prm = Params(N=1024, L=1, alpha=1, t=t)
    assert pow(prm.zeta, 2 * prm.N, t) == 1 and pow(prm.zeta, prm.N, t) == t - 1
    rng = random.Random(t)
    m = [t - 1 - rng.randrange(16) for _ in range(prm.N)]
    assert bfv.decode_poly(prm, m) == _brute_eval_table(prm, m)
    y = [rng.randrange(t) for _ in range(prm.N)]
    mm = bfv.encode_slots(prm, y)
    assert all(0 <= x < t for x in mm)
    assert _brute_eval_table(prm, mm) == y
    # a plain int64 product-sum (no reduction per product) wraps here: the pin can tell the difference
    if (t - 1) ** 2 >= 1 << 63:
        import numpy as np
        with np.errstate(over="ignore"):
            a = np.array([t - 1] * 4, dtype=np.int64)
            assert int((a * a).sum() % t) != 4 * (t - 1) ** 2 % t


def test_parameter_rule_rejects_t_from_2_to_the_32():
    # 2^32 + 12 * 2^11 + 1 is a prime = 1 mod 2048: batching-friendly at N = 1024 but above the bound
    t = (1 << 32) + 12 * (1 << 11) + 1
    from oracle.nt import is_prime
    assert is_prime(t)
    with pytest.raises(ValueError):
        Params(N=1024, L=1, alpha=1, t=t)


@pytest.mark.parametrize("t", LARGE_T)
def test_multiply_decrypts_at_large_t(t):
    prm = Params(N=1024, L=3, alpha=1, t=t)
    keys = bfv.keygen(prm, 12)
    rng = random.Random(8)
    y1 = [rng.randrange(t) for _ in range(prm.N)]
    y2 = [rng.randrange(t) for _ in range(prm.N)]
    a = bfv.encrypt(prm, keys, y1, 2, 0)
    b = bfv.encrypt(prm, keys, y2, 2, 1)
    assert bfv.decrypt(prm, keys, a) == y1
    c = bfv.mul_relin(prm, keys, a, b)
    assert bfv.decrypt(prm, keys, c) == [x * y % t for x, y in zip(y1, y2)]
    assert bfv.noise_budget(prm, keys, c) > 0


@pytest.mark.parametrize("cfg", [TINY, SMALL, dict(N=4096, L=1, alpha=1)])
def test_batching_is_slotwise(cfg):
    """decode is a ring map: products in Z_t[X]/(X^N+1) are slot-wise products."""
    prm = Params(**cfg)
    rng = random.Random(2)
    y1 = [rng.randrange(prm.t) for _ in range(prm.N)]
    y2 = [rng.randrange(prm.t) for _ in range(prm.N)]
    m1, m2 = bfv.encode_slots(prm, y1), bfv.encode_slots(prm, y2)
    prodm = [x % prm.t for x in negacyclic(m1, m2)]
    assert bfv.decode_poly(prm, prodm) == [a * b % prm.t for a, b in zip(y1, y2)]
    assert bfv.decode_poly(prm, m1) == y1


def test_key_relations():
    prm = Params(**SMALL)
    keys = bfv.keygen(prm, 11)
    N, Q, P = prm.N, prm.Q, prm.P
    assert set(keys.s) <= {-1, 0, 1}
    e = px.cbd_poly(11, px.PK_E, 0, N)
    # pk0 + pk1 s = -e (mod Q)
    lhs = [(x + y) % Q for x, y in zip(keys.pk0, negacyclic(keys.pk1, keys.s))]
    assert lhs == [(-x) % Q for x in e]
    # b_j + a_j s = -e_j + P g_j s^2 (mod PQ), with g_j = 1 mod q_j, 0 mod q_i (i != j)
    s2 = negacyclic(keys.s, keys.s)
    for j, (bj, aj) in enumerate(keys.rlk):
        ej = px.cbd_poly(11, px.RLK_E, j, N)
        lhs = [(x + y) % (P * Q) for x, y in zip(bj, negacyclic(aj, keys.s))]
        for n in range(N):
            r = (lhs[n] + ej[n]) % (P * Q)            # = P g_j s^2
            assert r % P == 0
            for i, qi in enumerate(prm.q):
                want = (P * s2[n]) % qi if i == j else 0
                assert r % qi == want


@pytest.mark.parametrize("cfg", [TINY, SMALL, dict(N=4096, L=2, alpha=1)])
def test_encrypt_decrypt_roundtrip(cfg):
    prm = Params(**cfg)
    keys = bfv.keygen(prm, 5)
    rng = random.Random(3)
    for idx in range(2):
        y = [rng.randrange(prm.t) for _ in range(prm.N)]
        ct = bfv.encrypt(prm, keys, y, seed=9, idx=idx)
        assert all(0 <= x < prm.Q for x in ct[0] + ct[1])
        assert bfv.decrypt(prm, keys, ct) == y
        assert bfv.noise_budget(prm, keys, ct) > 10


def test_linear_homomorphisms():
    prm = Params(**SMALL)
    keys = bfv.keygen(prm, 5)
    rng = random.Random(4)
    t = prm.t
    y1 = [rng.randrange(t) for _ in range(prm.N)]
    y2 = [rng.randrange(t) for _ in range(prm.N)]
    w = [rng.randrange(t) for _ in range(prm.N)]
    a = bfv.encrypt(prm, keys, y1, 1, 0)
    b = bfv.encrypt(prm, keys, y2, 1, 1)
    dec = lambda c: bfv.decrypt(prm, keys, c)
    assert dec(bfv.add(prm, a, b)) == [(x + y) % t for x, y in zip(y1, y2)]
    assert dec(bfv.sub(prm, a, b)) == [(x - y) % t for x, y in zip(y1, y2)]
    assert dec(bfv.negate(prm, a)) == [(-x) % t for x in y1]
    assert dec(bfv.add_const(prm, a, 7)) == [(x + 7) % t for x in y1]
    assert dec(bfv.sub_const(prm, a, 7)) == [(x - 7) % t for x in y1]
    assert dec(bfv.const_sub(prm, 7, a)) == [(7 - x) % t for x in y1]
    assert dec(bfv.mul_scalar(prm, a, 3)) == [(3 * x) % t for x in y1]
    assert dec(bfv.mul_plain(prm, a, w)) == [(x * y) % t for x, y in zip(y1, w)]
    assert dec(bfv.trivial(prm, 5)) == [5] * prm.N


@pytest.mark.parametrize("cfg", [TINY, SMALL])
def test_multiply_and_relinearise(cfg):
    prm = Params(**cfg)
    keys = bfv.keygen(prm, 6)
    rng = random.Random(5)
    t, Q, P = prm.t, prm.Q, prm.P
    y1 = [rng.randrange(t) for _ in range(prm.N)]
    y2 = [rng.randrange(t) for _ in range(prm.N)]
    a = bfv.encrypt(prm, keys, y1, 2, 0)
    b = bfv.encrypt(prm, keys, y2, 2, 1)
    want = [x * y % t for x, y in zip(y1, y2)]

    d = bfv.tensor(prm, a, b)
    c3 = tuple(bfv.scale_round(prm, dk) for dk in d)
    # scale-and-round is the nearest integer to t d / Q (exact rationals)
    for dk, ck in zip(d, c3):
        for x, y in zip(dk, ck):
            r = round(Fraction(t * x, Q))
            assert abs(Fraction(t * x, Q) - r) < Fraction(1, 2)
            assert r % Q == y
    # three-component decryption of the unrelinearised product
    v = bfv.phase(prm, keys, c3)
    m3 = [bfv.round_div(t * x, Q) % t for x in v]
    assert bfv.decode_poly(prm, m3) == want

    w0, w1 = bfv.key_switch_parts(prm, keys, c3[2])
    for x in w0 + w1:
        y = bfv.mod_down(prm, [x])[0]
        r = centered(x, P)
        assert (P * y + r - x) % (P * Q) == 0 and abs(r) <= P // 2

    c = bfv.mul_relin(prm, keys, a, b)
    assert bfv.decrypt(prm, keys, c) == want
    assert bfv.noise_budget(prm, keys, c) < bfv.noise_budget(prm, keys, a)


def test_centred_lift_is_visible_and_quieter():
    """FV lifts to the symmetric range; lifting to [0, Q) gives other ciphertext
    bits (so the choice must be fixed) and more noise (so it is the worse one)."""
    prm = Params(**SMALL)
    keys = bfv.keygen(prm, 6)
    rng = random.Random(6)
    y1 = [rng.randrange(prm.t) for _ in range(prm.N)]
    y2 = [rng.randrange(prm.t) for _ in range(prm.N)]
    a = bfv.encrypt(prm, keys, y1, 3, 0)
    b = bfv.encrypt(prm, keys, y2, 3, 1)
    d0 = negacyclic(a[0], b[0])
    d1 = [x + y for x, y in zip(negacyclic(a[0], b[1]), negacyclic(a[1], b[0]))]
    d2 = negacyclic(a[1], b[1])
    other = bfv.relin(prm, keys, tuple(bfv.scale_round(prm, d) for d in (d0, d1, d2)))
    right = bfv.mul_relin(prm, keys, a, b)
    assert other != right
    assert bfv.noise_budget(prm, keys, right) > bfv.noise_budget(prm, keys, other) + 1


def test_noise_budget_decreases_along_a_squaring_chain():
    prm = Params(N=16, L=4, alpha=1, t=97, prime_bits=50)
    keys = bfv.keygen(prm, 8)
    y = [random.Random(7).randrange(prm.t) for _ in range(prm.N)]
    c = bfv.encrypt(prm, keys, y, 4, 0)
    budgets = [bfv.noise_budget(prm, keys, c)]
    for _ in range(4):
        c = bfv.mul_relin(prm, keys, c, c)
        y = [x * x % prm.t for x in y]
        budgets.append(bfv.noise_budget(prm, keys, c))
        assert bfv.decrypt(prm, keys, c) == y
    assert all(b1 < b0 for b0, b1 in zip(budgets, budgets[1:]))


def test_delta_and_inverse_constants():
    prm = Params(**SMALL)
    assert prm.delta * prm.t <= prm.Q < (prm.delta + 1) * prm.t
    assert inv(prm.N, prm.t) * prm.N % prm.t == 1
