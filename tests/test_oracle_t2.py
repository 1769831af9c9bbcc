"""Pins for the oracle's t = 2 mode (no batching): coefficient encryption,
the ring product of binary polynomials, the XOR-free gate equations and the
circuits built on them (Sec. 3.1, Sec. 4.3)."""

import itertools
import random

import pytest

from oracle import bfv, bridge, circuits
from oracle.bridge import AND, MUX, NAND, NOR, NOT, OR, XNOR, XOR
from oracle.params import Params
from tests.test_oracle_bridge import TRUTH, PlainEvaluator, _bits, _fib_oblivious, _val

T2 = dict(N=8, L=4, alpha=1, t=2, prime_bits=50)


@pytest.fixture(scope="module")
def t2():
    prm = Params(**T2)
    return prm, bfv.keygen(prm, 23)


def negacyclic_mod2(a, b):
    """Schoolbook product in Z_2[X]/(X^N + 1) (X^N = -1 = 1 mod 2)."""
    N = len(a)
    out = [0] * N
    for i in range(N):
        for j in range(N):
            out[(i + j) % N] ^= a[i] & b[j]
    return out


def test_params_without_batching(t2):
    prm, _ = t2
    assert not prm.batching and prm.zeta == 0
    assert prm.delta == (prm.Q - 1) // 2            # Q odd
    assert prm.K == prm.L + 1 and prm.B > 2 * prm.t * prm.N * prm.Q
    with pytest.raises(ValueError):
        Params(N=8, L=2, alpha=1, t=3)               # neither 2 nor 1 mod 16
    with pytest.raises(ValueError):
        bfv.encrypt(prm, None, [0] * prm.N, 1)


def test_coefficient_round_trip_and_ring_product(t2):
    prm, keys = t2
    rng = random.Random(3)
    for k in range(4):
        a = [rng.randrange(2) for _ in range(prm.N)]
        b = [rng.randrange(2) for _ in range(prm.N)]
        ca = bfv.encrypt_poly(prm, keys, a, 5, 2 * k)
        cb = bfv.encrypt_poly(prm, keys, b, 5, 2 * k + 1)
        assert bfv.decrypt_poly(prm, keys, ca) == a
        assert bfv.decrypt_poly(prm, keys, bfv.add(prm, ca, cb)) == [x ^ y for x, y in zip(a, b)]
        assert bfv.decrypt_poly(prm, keys, bfv.mul_relin(prm, keys, ca, cb)) == negacyclic_mod2(a, b)


T2_COUNTS = {AND: (0, 0, 1), OR: (1, 1, 1), XOR: (1, 0, 0), NAND: (0, 1, 1), NOR: (1, 2, 1),
             XNOR: (1, 1, 0), NOT: (0, 1, 0), MUX: (1, 1, 1)}


def test_gate_truth_tables_t2(t2):
    """Each bit in the constant coefficient (the product of constants is their product)."""
    prm, keys = t2
    for combo in itertools.product((0, 1), repeat=3):
        ct = [bfv.encrypt_poly(prm, keys, [v] + [0] * (prm.N - 1), 7, i) for i, v in enumerate(combo)]
        for g, f in TRUTH.items():
            ev = bridge.Evaluator(prm, keys)
            out = bfv.decrypt_poly(prm, keys, ev.gate(g, *ct))
            assert out == [f(*combo)] + [0] * (prm.N - 1), (bridge.GATE_NAMES[g], combo)
            assert ev.counts() == T2_COUNTS[g]


def test_circuits_t2_plain():
    rng = random.Random(14)
    m = 300
    a = [rng.randrange(256) for _ in range(m)]
    b = [rng.randrange(256) if k % 4 else a[k] for k in range(m)]
    ev = PlainEvaluator(2, m)
    assert _val(circuits.ripple_add(ev, _bits(a, 8), _bits(b, 8))) == [x + y for x, y in zip(a, b)]
    assert ev.n_mul == 15                                  # the products serve the carries
    ev = PlainEvaluator(2, m)
    assert circuits.equal(ev, _bits(a, 8), _bits(b, 8)) == [int(x == y) for x, y in zip(a, b)]
    assert ev.n_mul == 7                                   # XNOR is free, the AND tree is not
    ev = PlainEvaluator(2, m)
    assert circuits.less_than(ev, _bits(a, 8), _bits(b, 8)) == [int(x < y) for x, y in zip(a, b)]
    ev65537 = PlainEvaluator(65537, m)
    circuits.less_than(ev65537, _bits(a, 8), _bits(b, 8))
    assert ev.n_mul < ev65537.n_mul
    ev = PlainEvaluator(2, m)
    assert _val(circuits.multiply(ev, _bits(a, 8), _bits(b, 8))) == [x * y for x, y in zip(a, b)]


def test_fibonacci_bits_t2_plain():
    vals = list(range(256))
    n = len(vals)
    zero, one = [0] * n, [1] * n
    ev = PlainEvaluator(2, n)
    r = circuits.fibonacci_bits(ev, _bits(vals, 8), [zero] * 8, [zero] * 8, [one] + [zero] * 7, [zero] * 8, 10)
    assert _val(r) == [_fib_oblivious(v, 10, 8) % 256 for v in vals]
    assert ev.n_mul == 10 * (8 * 8 - 4 - 8)                # the 8 XNORs of each equality are free


def test_adder_encrypted_t2(t2):
    prm, keys = t2
    rng = random.Random(15)
    for trial in range(3):
        x, y = rng.randrange(16), rng.randrange(16)
        enc = lambda v, k: bfv.encrypt_poly(prm, keys, [v] + [0] * (prm.N - 1), 17 + trial, k)
        xb = [enc((x >> k) & 1, k) for k in range(4)]
        yb = [enc((y >> k) & 1, 4 + k) for k in range(4)]
        ev = bridge.Evaluator(prm, keys)
        s = circuits.ripple_add(ev, xb, yb)
        got = sum(bfv.decrypt_poly(prm, keys, c)[0] << k for k, c in enumerate(s))
        assert got == x + y
