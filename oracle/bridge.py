"""Homomorphic gates and the bridge between SecureUint and SecureMod.

Test infrastructure only.  Follows the paper directly:

* gate equations over encrypted bits (Sec. 3.1): AND = xy, NAND = 1 - xy,
  OR = x + y - xy, NOR = 1 - OR, XOR = x + y - 2xy, XNOR = 1 - XOR,
  NOT = 1 - x, MUX(x, y, z) = x(y - z) + z; one ciphertext multiply per gate
  except NOT; with t = 2 the XOR equation reduces to x + y (mod 2) and XOR and
  XNOR = 1 - (x + y) take no multiply (Sec. 3.1, Sec. 4.3);
* SecureUint -> SecureMod (Sec. 3.2.1, Listing 5): Horner, r = v[s-1];
  r += r + v[i] for i = s-2 .. 0; 2(s-1) additions, no multiplies;
* pow (Listing 7): square-and-multiply recursion, floor(log2 e) + w(e) - 1
  multiplies;
* SecureMod -> SecureUint (Sec. 3.2.3, Eq. 2 and Listing 8): for each
  candidate c, eq_c = 1 - (x - c)^(t-1), then SecureUint(c) * SecureBool(eq_c)
  and a per-bit sum over c;
* SecureInt -> SecureMod (Sec. 3.2.2, Eq. 1, Listing 6): a multiplexer on the
  sign bit between the Horner value and t - 2^s plus it (2 multiplies);
* SecureMod -> SecureInt (Sec. 3.2.4, Listing 9): two SecureMod -> SecureUint
  conversions (of x and of 2^s - t + x) and a per-bit multiplexer on the sign
  bit of the first; Listing 9 names the width `s`, read as Size, and Eq. 3 and
  the listing differ (a bit-level addition against a second conversion): the
  listing is followed.  Its multiplexer over s bits costs 2s multiplies where
  the paper's count says 2 (it counts the SecureInt product as one).

Readings (the paper is silent or loose here):
* constants are trivial ciphertexts (Delta [c]_t, 0);
* the candidate range is an argument (the paper's loop is i = 1 .. t-1);
* mode PAPER multiplies every bit of SecureUint(c) (a trivial ciphertext of
  that bit) with eq_c: s multiplies per candidate, the count the paper gives;
  mode SELECT adds eq_c into bit k only when bit k of c is 1 (no multiplies);
* sum(v) is per-bit ciphertext addition (the eq_c are one-hot);
* op counting: every ciphertext +/- (including +/- of a public constant) is
  one add or sub, every ciphertext x ciphertext product one mul.
"""

from . import bfv

AND, OR, XOR, NAND, NOR, XNOR, NOT, MUX = range(8)
GATE_NAMES = ("AND", "OR", "XOR", "NAND", "NOR", "XNOR", "NOT", "MUX")
PAPER, SELECT = 0, 1


class Evaluator:
    """Oracle evaluator with the paper's add / sub / mul accounting."""

    def __init__(self, prm, keys):
        self.prm = prm
        self.keys = keys
        self.n_add = 0
        self.n_sub = 0
        self.n_mul = 0

    # -- counted primitives
    def add(self, a, b):
        self.n_add += 1
        return bfv.add(self.prm, a, b)

    def sub(self, a, b):
        self.n_sub += 1
        return bfv.sub(self.prm, a, b)

    def add_const(self, a, c):
        self.n_add += 1
        return bfv.add_const(self.prm, a, c)

    def sub_const(self, a, c):
        self.n_sub += 1
        return bfv.sub_const(self.prm, a, c)

    def const_sub(self, c, a):
        self.n_sub += 1
        return bfv.const_sub(self.prm, c, a)

    def mul(self, a, b):
        self.n_mul += 1
        return bfv.mul_relin(self.prm, self.keys, a, b)

    def trivial(self, c):
        return bfv.trivial(self.prm, c)

    def counts(self):
        return (self.n_add, self.n_sub, self.n_mul)

    # -- Sec. 3.1 gate equations
    def gate(self, g, x, y=None, z=None):
        if g == NOT:
            return self.const_sub(1, x)
        if g == MUX:
            return self.add(self.mul(x, self.sub(y, z)), z)
        if self.prm.t == 2 and g in (XOR, XNOR):
            r = self.add(x, y)
            return r if g == XOR else self.const_sub(1, r)
        xy = self.mul(x, y)
        if g == AND:
            return xy
        if g == NAND:
            return self.const_sub(1, xy)
        if g in (OR, NOR):
            r = self.sub(self.add(x, y), xy)
            return r if g == OR else self.const_sub(1, r)
        if g in (XOR, XNOR):
            r = self.sub(self.add(x, y), self.add(xy, xy))
            return r if g == XOR else self.const_sub(1, r)
        raise ValueError(g)

    # -- Listing 5: SecureUint<s> -> SecureMod by Horner's scheme
    def bits_to_mod(self, v):
        i = len(v)
        i -= 1
        r = v[i]
        while i > 0:
            i -= 1
            r = self.add(r, self.add(r, v[i]))
        return r

    # -- Listing 7: square-and-multiply, product order as printed
    def pow(self, b, e):
        if e == 0:
            return self.trivial(1)
        if e == 1:
            return b
        r = self.pow(self.mul(b, b), e >> 1)
        if e & 1:
            r = self.mul(r, b)
        return r

    # -- Eq. 2 / Listing 8: SecureMod -> SecureUint<s>
    def equality(self, x, c):
        """eq_c = 1 - (x - c)^(t-1): an encryption of 1 where x == c, else 0."""
        return self.const_sub(1, self.pow(self.sub_const(x, c), self.prm.t - 1))

    def mod_to_bits(self, x, s, cands, mode=PAPER):
        bits = [None] * s
        for c in cands:
            eq = self.equality(x, c)
            for k in range(s):
                bit = (c >> k) & 1
                if mode == PAPER:
                    term = self.mul(self.trivial(bit), eq)
                elif bit:
                    term = eq
                else:
                    continue
                bits[k] = term if bits[k] is None else self.add(bits[k], term)
        return [b if b is not None else self.trivial(0) for b in bits]

    # -- Sec. 3.2.2, Eq. 1, Listing 6: SecureInt<s> -> SecureMod
    def sint_to_mod(self, v):
        """pos = Horner(v); neg = (t - 2^s) + pos; isNeg = v[s-1];
        result = isNeg * neg + (1 - isNeg) * pos (needs t >= 2^s)."""
        s = len(v)
        pos = self.bits_to_mod(v)
        neg = self.add_const(pos, (self.prm.t - (1 << s)) % self.prm.t)
        is_neg = v[s - 1]
        return self.add(self.mul(is_neg, neg), self.mul(self.const_sub(1, is_neg), pos))

    # -- Sec. 3.2.4, Eq. 3, Listing 9: SecureMod -> SecureInt<s>
    def mod_to_sint(self, x, s, cands_pos, cands_neg, mode=PAPER):
        """pos = to_SecureUint(x); neg = to_SecureUint((2^s - t) + x); isNeg = pos[s-1];
        result bit k = isNeg * neg[k] + (1 - isNeg) * pos[k] (needs 2^s >= t).
        The two candidate ranges of the conversions are arguments (the listing scans all of Z_t)."""
        t = self.prm.t
        pos = self.mod_to_bits(x, s, cands_pos, mode)
        neg = self.mod_to_bits(self.add_const(x, ((1 << s) - t) % t), s, cands_neg, mode)
        is_neg = pos[s - 1]
        not_neg = self.const_sub(1, is_neg)
        return [self.add(self.mul(is_neg, neg[k]), self.mul(not_neg, pos[k])) for k in range(s)]


def pow_mul_count(e):
    """floor(log2 e) + w(e) - 1 (Sec. 3.2.3)."""
    return e.bit_length() - 1 + bin(e).count("1") - 1


def mod_to_bits_mul_count(n_cands, s, t):
    """n_cands * (s + floor(log2(t-1)) + w(t-1) - 1) multiplies (Sec. 3.2.3, PAPER mode)."""
    return n_cands * (s + pow_mul_count(t - 1))
