"""Pins for the oracle's gates, bridge conversions and circuits.

Exhaustive truth tables (Sec. 3.1), all 2^s inputs of the Horner conversion
(Listing 5), Fermat's little theorem over all of Z_t (Eq. 2), the round trip
bits -> mod -> bits, and the multiply counts the paper states for pow and for
the SecureMod -> SecureUint conversion (Sec. 3.2.3).  Deep circuits are
checked through a plaintext evaluator with the same interface (the circuit
logic is what is pinned there; noise is not involved).
"""

import itertools
import random
import types

import pytest

from oracle import bfv, bridge, circuits
from oracle.bridge import AND, MUX, NAND, NOR, NOT, OR, PAPER, SELECT, XNOR, XOR
from oracle.params import Params

# N = 8 slots, t = 17 (= 1 mod 16); 4 x 50-bit primes leave room for depth 5
TINY = dict(N=8, L=4, alpha=1, t=17, prime_bits=50)


@pytest.fixture(scope="module")
def tiny():
    prm = Params(**TINY)
    keys = bfv.keygen(prm, 21)
    return prm, keys


class PlainEvaluator:
    """Slot vectors mod t with the oracle Evaluator's interface and counters."""

    def __init__(self, t, n):
        self.t, self.n = t, n
        self.prm = types.SimpleNamespace(t=t, N=n)
        self.n_add = self.n_sub = self.n_mul = 0

    def add(self, a, b):
        self.n_add += 1
        return [(x + y) % self.t for x, y in zip(a, b)]

    def sub(self, a, b):
        self.n_sub += 1
        return [(x - y) % self.t for x, y in zip(a, b)]

    def add_const(self, a, c):
        self.n_add += 1
        return [(x + c) % self.t for x in a]

    def sub_const(self, a, c):
        self.n_sub += 1
        return [(x - c) % self.t for x in a]

    def const_sub(self, c, a):
        self.n_sub += 1
        return [(c - x) % self.t for x in a]

    def mul(self, a, b):
        self.n_mul += 1
        return [(x * y) % self.t for x, y in zip(a, b)]

    def trivial(self, c):
        return [c % self.t] * self.n

    gate = bridge.Evaluator.gate
    bits_to_mod = bridge.Evaluator.bits_to_mod
    pow = bridge.Evaluator.pow
    equality = bridge.Evaluator.equality
    mod_to_bits = bridge.Evaluator.mod_to_bits
    sint_to_mod = bridge.Evaluator.sint_to_mod
    mod_to_sint = bridge.Evaluator.mod_to_sint


TRUTH = {AND: lambda x, y, z: x & y, OR: lambda x, y, z: x | y, XOR: lambda x, y, z: x ^ y,
         NAND: lambda x, y, z: 1 - (x & y), NOR: lambda x, y, z: 1 - (x | y),
         XNOR: lambda x, y, z: 1 - (x ^ y), NOT: lambda x, y, z: 1 - x,
         MUX: lambda x, y, z: y if x else z}
GATE_COUNTS = {AND: (0, 0, 1), OR: (1, 1, 1), XOR: (2, 1, 1), NAND: (0, 1, 1), NOR: (1, 2, 1),
               XNOR: (2, 2, 1), NOT: (0, 1, 0), MUX: (1, 1, 1)}


def test_gate_truth_tables_encrypted(tiny):
    prm, keys = tiny
    combos = list(itertools.product((0, 1), repeat=3))        # 8 slots = all (x, y, z)
    xs, ys, zs = ([c[i] for c in combos] for i in range(3))
    ct = [bfv.encrypt(prm, keys, v, 31, i) for i, v in enumerate((xs, ys, zs))]
    for g, f in TRUTH.items():
        ev = bridge.Evaluator(prm, keys)
        out = ev.gate(g, *ct)
        assert bfv.decrypt(prm, keys, out) == [f(*c) for c in combos], bridge.GATE_NAMES[g]
        assert ev.counts() == GATE_COUNTS[g]


@pytest.mark.parametrize("s", [1, 2, 3])
def test_bits_to_mod_all_inputs_encrypted(tiny, s):
    prm, keys = tiny
    vals = [v % (1 << s) for v in range(prm.N)]
    bits = [bfv.encrypt(prm, keys, [(v >> k) & 1 for v in vals], 41, k) for k in range(s)]
    ev = bridge.Evaluator(prm, keys)
    r = ev.bits_to_mod(bits)
    assert bfv.decrypt(prm, keys, r) == vals
    assert ev.counts() == (2 * (s - 1), 0, 0)


@pytest.mark.parametrize("s", [1, 4, 8, 12, 16])
def test_bits_to_mod_all_inputs_plain(s):
    t = 65537
    n = min(1 << s, 4096)
    vals = list(range(n)) if n == (1 << s) else random.Random(s).sample(range(1 << s), n)
    ev = PlainEvaluator(t, n)
    r = ev.bits_to_mod([[(v >> k) & 1 for v in vals] for k in range(s)])
    assert r == [v % t for v in vals]
    assert (ev.n_add, ev.n_sub, ev.n_mul) == (2 * (s - 1), 0, 0)


@pytest.mark.parametrize("e", [0, 1, 2, 3, 5, 7, 16, 17, 255, 256, 65536])
def test_pow_values_and_count(e):
    t = 65537
    xs = [0, 1, 2, 3, 12345, 65536]
    ev = PlainEvaluator(t, len(xs))
    assert ev.pow(xs, e) == [pow(x, e, t) for x in xs]
    if e >= 1:
        assert ev.n_mul == bridge.pow_mul_count(e) == (e.bit_length() - 1) + bin(e).count("1") - 1


def test_fermat_equality_exhaustive_plain():
    """(x - c)^(t-1) is 0 iff x == c, else 1, over all x in Z_t (t = 65537, t = 257, t = 17)."""
    for t in (17, 257, 65537):
        xs = list(range(t))
        for c in (0, 1, t // 2, t - 1):
            ev = PlainEvaluator(t, t)
            eq = ev.const_sub(1, ev.pow(ev.sub_const(xs, c), t - 1))
            assert eq == [int(x == c) for x in xs]


def test_fermat_equality_encrypted(tiny):
    prm, keys = tiny
    xs = [0, 3, 5, 16, 9, 5, 1, 0]
    x = bfv.encrypt(prm, keys, xs, 51, 0)
    for c in range(prm.t):
        ev = bridge.Evaluator(prm, keys)
        eq = ev.equality(x, c)
        assert bfv.decrypt(prm, keys, eq) == [int(v == c) for v in xs]
        assert ev.counts() == (0, 2, 4)


@pytest.mark.parametrize("mode", [PAPER, SELECT])
def test_mod_to_bits_roundtrip_encrypted(tiny, mode):
    prm, keys = tiny
    s = 5
    xs = [0, 3, 5, 16, 9, 12, 1, 7]
    x = bfv.encrypt(prm, keys, xs, 61, 0)
    ev = bridge.Evaluator(prm, keys)
    cands = range(prm.t)                      # every value of Z_17
    bits = ev.mod_to_bits(x, s, cands, mode)
    for k in range(s):
        assert bfv.decrypt(prm, keys, bits[k]) == [(v >> k) & 1 for v in xs]
    n_mul = ev.n_mul
    if mode == PAPER:
        assert n_mul == bridge.mod_to_bits_mul_count(len(cands), s, prm.t) == prm.t * (s + 4)
    else:
        assert n_mul == len(cands) * 4
    back = ev.bits_to_mod(bits)
    assert bfv.decrypt(prm, keys, back) == xs


def test_mod_to_bits_count_formula_at_65537():
    """t (s + floor(log2(t-1)) + w(t-1) - 1) with t - 1 = 2^16: s + 16 per candidate."""
    assert bridge.mod_to_bits_mul_count(65537, 8, 65537) == 65537 * 24
    assert bridge.mod_to_bits_mul_count(256, 8, 65537) == 256 * 24


# ------------------------------------------------------------ circuits (plaintext evaluator)
def _bits(vals, s):
    return [[(v >> k) & 1 for v in vals] for k in range(s)]


def _val(bits):
    return [sum(b[i] << k for k, b in enumerate(bits)) for i in range(len(bits[0]))]


def test_ripple_adder_plain():
    rng = random.Random(8)
    a = [rng.randrange(256) for _ in range(64)]
    b = [rng.randrange(256) for _ in range(64)]
    ev = PlainEvaluator(65537, 64)
    out = circuits.ripple_add(ev, _bits(a, 8), _bits(b, 8))
    assert len(out) == 9 and _val(out) == [x + y for x, y in zip(a, b)]
    assert ev.n_mul == 15


def test_comparator_plain():
    rng = random.Random(9)
    a = [rng.randrange(1 << 16) for _ in range(200)] + [5, 7, 7, 65535, 0]
    b = [rng.randrange(1 << 16) for _ in range(200)] + [7, 5, 7, 0, 65535]
    ev = PlainEvaluator(65537, len(a))
    lt = circuits.less_than(ev, _bits(a, 16), _bits(b, 16))
    assert lt == [int(x < y) for x, y in zip(a, b)]
    assert ev.n_mul == 57


def test_multiplier_plain():
    rng = random.Random(10)
    a = [rng.randrange(1 << 16) for _ in range(100)] + [65535, 0, 1]
    b = [rng.randrange(1 << 16) for _ in range(100)] + [65535, 7, 1]
    ev = PlainEvaluator(65537, len(a))
    prodb = circuits.multiply(ev, _bits(a, 16), _bits(b, 16))
    assert len(prodb) == 32 and _val(prodb) == [x * y for x, y in zip(a, b)]
    assert ev.n_mul == 256 + 30 + 14 * 31


def test_argmax3_plain():
    rng = random.Random(11)
    s = [[rng.randrange(1 << 12) for _ in range(300)] for _ in range(3)]
    s[0][:4] = [5, 5, 9, 1]
    s[1][:4] = [5, 9, 9, 1]
    s[2][:4] = [5, 2, 9, 1]
    ev = PlainEvaluator(65537, 300)
    idx = circuits.argmax3(ev, *(_bits(v, 12) for v in s))
    want = [max(range(3), key=lambda j: (s[j][i], -j)) for i in range(300)]
    assert [i0 + 2 * i1 for i0, i1 in zip(*idx)] == want


def test_adder_and_comparator_encrypted(tiny):
    prm, keys = tiny
    a = [0, 1, 2, 3, 3, 2, 1, 0]
    b = [0, 3, 1, 3, 2, 2, 0, 1]
    ab = [bfv.encrypt(prm, keys, v, 71, k) for k, v in enumerate(_bits(a, 2))]
    bb = [bfv.encrypt(prm, keys, v, 72, k) for k, v in enumerate(_bits(b, 2))]
    ev = bridge.Evaluator(prm, keys)
    s = circuits.ripple_add(ev, ab, bb)
    assert _val([bfv.decrypt(prm, keys, c) for c in s]) == [x + y for x, y in zip(a, b)]
    lt = circuits.less_than(ev, ab, bb)
    assert bfv.decrypt(prm, keys, lt) == [int(x < y) for x, y in zip(a, b)]


# ------------------------------------------------------------ signed conversions (Listings 6 and 9)
@pytest.mark.parametrize("s", [2, 4, 8, 16])
def test_sint_to_mod_all_values_plain(s):
    """Eq. 1: a negative s-bit value v maps to t - 2^s + (two's complement bits) = v mod t."""
    t = 65537
    vals = list(range(-(1 << (s - 1)), 1 << (s - 1)))
    if len(vals) > 4096:
        vals = random.Random(s).sample(vals, 4096) + [-(1 << (s - 1)), -1, 0, (1 << (s - 1)) - 1]
    ev = PlainEvaluator(t, len(vals))
    bits = [[((v + (1 << s)) >> k) & 1 for v in vals] for k in range(s)]
    r = ev.sint_to_mod(bits)
    assert r == [v % t for v in vals]
    # 2 multiplies and 2s + 1 additions or subtractions (Sec. 3.2.2)
    assert ev.n_mul == 2 and ev.n_add + ev.n_sub == 2 * s + 1


def test_sint_to_mod_encrypted(tiny):
    prm, keys = tiny
    s = 4                                         # t = 17 >= 2^4
    vals = list(range(-8, 8))
    ev = bridge.Evaluator(prm, keys)
    for half in (vals[:8], vals[8:]):
        bits = [bfv.encrypt(prm, keys, [((v + 16) >> k) & 1 for v in half], 81, k) for k in range(s)]
        r = ev.sint_to_mod(bits)
        assert bfv.decrypt(prm, keys, r) == [v % prm.t for v in half]


def test_mod_to_sint_listing_arithmetic_plain():
    """Listing 9 as printed, at t = 17, s = 5 (2^s >= t): values below 2^(s-1) come back as
    their bits; x = 16 (read as -1) comes back as the bits of (2^s - t + x) mod t = 14, because
    the listing's second conversion works mod t (Eq. 3 adds 2^s - t in bit-level arithmetic)."""
    t, s = 17, 5
    xs = list(range(t))
    ev = PlainEvaluator(t, t)
    out = ev.mod_to_sint(xs, s, range(t), range(t), SELECT)
    got = _val(out)
    assert got[:16] == list(range(16))
    assert got[16] == ((1 << s) - t + 16) % t == 14
    # two conversions (4 multiplies per candidate in the Fermat chain at t = 17), 2s for the multiplexer
    assert ev.n_mul == 2 * t * 4 + 2 * s


def test_mod_to_sint_encrypted_matches_plain(tiny):
    prm, keys = tiny
    s = 5
    xs = [0, 3, 15, 16, 9, 12, 1, 7]
    x = bfv.encrypt(prm, keys, xs, 91, 0)
    ev = bridge.Evaluator(prm, keys)
    bits = ev.mod_to_sint(x, s, range(prm.t), range(prm.t), SELECT)
    want = [v if v < 16 else ((1 << s) - prm.t + v) % prm.t for v in xs]
    assert _val([bfv.decrypt(prm, keys, b) for b in bits]) == want
    assert ev.n_mul == 2 * prm.t * 4 + 2 * s


@pytest.mark.parametrize("t,s", [(17, 5), (97, 7), (257, 9), (257, 10)])
def test_mod_to_sint_against_eq3(t, s):
    """Eq. 3 (bit-level: Y = X when X_{s-1} = 0, else the s-bit sum 2^s - t + X) is the two's
    complement of x - t for x >= 2^(s-1) and of x otherwise.  The listing agrees with it on every
    x whose shifted value 2^s - t + x stays below t, and on every non-negative x; elsewhere its
    mod-t addition wraps (the case the listing does not cover)."""
    xs = list(range(t))
    ev = PlainEvaluator(t, t)
    got = _val(ev.mod_to_sint(xs, s, range(t), range(t), SELECT))
    for x, g in zip(xs, got):
        eq3 = x if x < (1 << (s - 1)) else ((1 << s) - t + x) % (1 << s)
        if x < (1 << (s - 1)) or (1 << s) - t + x < t:
            assert g == eq3, x
            v = eq3 - (1 << s) if eq3 >> (s - 1) else eq3
            assert v % t == x                     # the signed value is congruent to x
        else:
            assert g == ((1 << s) - t + x) % t, x


# ------------------------------------------------------------ Fibonacci (Listings 1-4)
def _fib_plain(n_in):
    """Listing 1: the plain loop, run until i reaches the input."""
    i, a, b = 0, 0, 1
    while i != n_in:
        i += 1
        a, b = b, a
        a += b
    return a


def _fib_oblivious(n_in, max_iter, width):
    """Listing 2 with the counter i kept in `width` bits (it wraps like the encrypted one)."""
    i, a, b, r = 0, 0, 1, 0
    for _ in range(max_iter):
        r += (i == n_in) * a
        i = (i + 1) % (1 << width)
        a, b = b, a
        a += b
    return r


def test_fibonacci_listings_agree():
    assert [_fib_plain(k) for k in range(12)] == [0, 1, 1, 2, 3, 5, 8, 13, 21, 34, 55, 89]
    for k in range(10):
        assert _fib_oblivious(k, 10, 8) == _fib_plain(k)
    assert _fib_oblivious(12, 10, 8) == 0            # the accumulator never reaches the input


@pytest.mark.parametrize("width,max_iter", [(4, 10), (4, 20), (8, 10), (8, 16)])
def test_fibonacci_bit_level_and_bridged_plain(width, max_iter):
    """Every input value in its own slot: Listing 3 equals Listing 2 mod 2^width, Listing 4 mod t;
    multiply counts per iteration 8n - 4 (bit-level) and 3n - 1 (bridged)."""
    t = 65537
    vals = list(range(1 << width))
    n = len(vals)
    inp = _bits(vals, width)
    zero, one = [0] * n, [1] * n
    want = [_fib_oblivious(v, max_iter, width) for v in vals]

    ev = PlainEvaluator(t, n)
    r = circuits.fibonacci_bits(ev, inp, [zero] * width, [zero] * width, [one] + [zero] * (width - 1),
                                [zero] * width, max_iter)
    assert _val(r) == [w % (1 << width) for w in want]
    assert ev.n_mul == max_iter * (8 * width - 4)

    ev = PlainEvaluator(t, n)
    r = circuits.fibonacci_bridged(ev, inp, [zero] * width, zero, one, zero, max_iter)
    assert r == [w % t for w in want]
    assert ev.n_mul == max_iter * (3 * width - 1)


def test_equal_and_increment_plain():
    rng = random.Random(12)
    x = [rng.randrange(256) for _ in range(300)] + [0, 255, 17]
    y = [rng.randrange(256) if k % 3 else x[k] for k in range(300)] + [0, 255, 18]
    ev = PlainEvaluator(65537, len(x))
    assert circuits.equal(ev, _bits(x, 8), _bits(y, 8)) == [int(a == b) for a, b in zip(x, y)]
    assert ev.n_mul == 15
    ev = PlainEvaluator(65537, len(x))
    assert _val(circuits.increment(ev, _bits(x, 8))) == [(a + 1) % 256 for a in x]
    assert ev.n_mul == 7


def test_fibonacci_encrypted_small(tiny):
    """Both programs on encrypted 2-bit inputs (t = 17), one slot per input value."""
    prm, keys = tiny
    width, max_iter = 2, 3
    vals = [0, 1, 2, 3, 0, 1, 2, 3]
    enc = lambda v, k: bfv.encrypt(prm, keys, v, 141, k)
    z, o = [0] * prm.N, [1] * prm.N
    inp = [enc(p, k) for k, p in enumerate(_bits(vals, width))]
    zeros = [enc(z, 10 + k) for k in range(width)]
    ev = bridge.Evaluator(prm, keys)
    r = circuits.fibonacci_bridged(ev, inp, zeros, enc(z, 20), enc(o, 21), enc(z, 22), max_iter)
    assert bfv.decrypt(prm, keys, r) == [_fib_oblivious(v, max_iter, width) % prm.t for v in vals]
