"""Bit-level circuits built from the oracle's gates (test infrastructure only).

The paper builds comparison, addition and multiplication "using standard
combinational arithmetic circuit design" (Sec. 3.1) without giving netlists.
These are this build's netlists, written as plain gate expressions; bits are
little-endian lists of ciphertexts (bit 0 first).

* ripple-carry adder: p_i = a_i b_i, u_i = a_i XOR b_i, q_i = c_i u_i,
  s_i = u_i XOR c_i (= u_i + c_i - 2 q_i), c_{i+1} = p_i + q_i (the two terms
  are never both 1); c_0 = 0 is public, so bit 0 is a half adder; the carry
  out is kept (n + 1 output bits); XOR here is x + y - 2xy with the product
  shared with the carry logic, so an n-bit adder costs 2n - 1 multiplies;
* less-than comparator, balanced: a leaf is (lt, eq) = ((1 - a_i) b_i,
  1 - (a_i XOR b_i)); two blocks merge high over low as
  lt = lt_H + eq_H lt_L, eq = eq_H eq_L (eq only where a parent uses it);
  blocks split as low = bits [0, n//2), high = [n//2, n);
* shift-add multiplier: partial products a AND b_j, accumulated row by row
  with the ripple-carry adder (2n-bit product);
* argmax of three: i1 = [s0' < s2], i0 = [s0 < s1] AND NOT i1 where
  s0' = MUX([s0 < s1], s1, s0); ties keep the lower index.
"""

from .bridge import AND, MUX, NOT


def half_adder_shared(ev, x, y):
    """(x XOR y, x AND y) with one shared multiply."""
    p = ev.mul(x, y)
    u = ev.sub(ev.add(x, y), ev.add(p, p))
    return u, p


def ripple_add(ev, a, b):
    """len(a) <= len(b) = n bits (a zero-extended) -> n + 1 bits."""
    out = []
    c = None
    for i in range(len(b)):
        if i < len(a):
            u, p = half_adder_shared(ev, a[i], b[i])
        else:
            u, p = b[i], None             # a_i = 0: u = b_i, no generate term
        if c is None:
            out.append(u)
            c = p
            continue
        s, q = half_adder_shared(ev, u, c)
        out.append(s)
        c = q if p is None else ev.add(p, q)
    out.append(c)
    return out


def less_than(ev, a, b):
    """Encryption of [a < b] for little-endian bit vectors of equal length.

    A block's eq is formed only where a parent uses it (every high child, and
    a low child whose parent needs its own eq), so the low spine skips it.
    """
    def block(lo, hi, need_eq):
        if hi - lo == 1:
            lt = ev.mul(ev.const_sub(1, a[lo]), b[lo])
            eq = None
            if need_eq:
                u, _ = half_adder_shared(ev, a[lo], b[lo])
                eq = ev.const_sub(1, u)
            return lt, eq
        mid = lo + (hi - lo) // 2
        lt_l, eq_l = block(lo, mid, need_eq)
        lt_h, eq_h = block(mid, hi, True)
        lt = ev.add(lt_h, ev.mul(eq_h, lt_l))
        eq = ev.mul(eq_h, eq_l) if need_eq else None
        return lt, eq
    return block(0, len(a), False)[0]


def multiply(ev, a, b):
    """n x n -> 2n-bit shift-add product."""
    n = len(a)
    rows = [[ev.gate(AND, a[i], b[j]) for i in range(n)] for j in range(n)]
    acc = list(rows[0])                       # bits 0 .. n-1
    for j in range(1, n):
        summ = ripple_add(ev, acc[j:], rows[j])
        acc = acc[:j] + summ                  # bits 0 .. j+n
    return acc


def mux_bits(ev, sel, x, y):
    return [ev.gate(MUX, sel, xi, yi) for xi, yi in zip(x, y)]


def argmax3(ev, s0, s1, s2):
    lt01 = less_than(ev, s0, s1)
    best = mux_bits(ev, lt01, s1, s0)
    i1 = less_than(ev, best, s2)
    i0 = ev.gate(AND, lt01, ev.gate(NOT, i1))
    return [i0, i1]
