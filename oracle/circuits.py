"""Bit-level circuits built from the oracle's gates (test infrastructure only).

Sec. 3.1 leaves comparison, addition and multiplication to ordinary
combinational circuits over its gates and gives no netlists.  These are the
netlists chosen here, written as plain gate expressions; bits are
little-endian lists of ciphertexts (bit 0 first).

* ripple-carry adder: p_i = a_i b_i, u_i = a_i XOR b_i, q_i = c_i u_i,
  s_i = u_i XOR c_i (= u_i + c_i - 2 q_i), c_{i+1} = p_i + q_i (the two terms
  are never both 1); c_0 = 0 is public, so bit 0 is a half adder; the carry
  out is kept (n + 1 output bits); XOR here is x + y - 2xy with the product
  shared with the carry logic, so an n-bit adder costs 2n - 1 multiplies
  (with t = 2 the sums are x + y and the products serve the carries only);
* less-than comparator, balanced: a leaf is (lt, eq) = ((1 - a_i) b_i,
  1 - (a_i XOR b_i)); two blocks merge high over low as
  lt = lt_H + eq_H lt_L, eq = eq_H eq_L (eq only where a parent uses it);
  blocks split as low = bits [0, n//2), high = [n//2, n);
* shift-add multiplier: partial products a AND b_j, accumulated row by row
  with the ripple-carry adder (2n-bit product);
* argmax of three: i1 = [s0' < s2], i0 = [s0 < s1] AND NOT i1 where
  s0' = MUX([s0 < s1], s1, s0); ties keep the lower index;
* equality: e_k = XNOR(x_k, y_k), then a balanced AND tree (low half
  [0, n//2) times high half), 2n - 1 multiplies;
* increment by the public 1: bit 0 is NOT x_0 with carry x_0 (XOR and AND
  with a public 1 are exact rewrites, no multiply), then half adders; the
  carry out of the top bit is dropped (n-bit wraparound), n - 1 multiplies.

Fibonacci (Sec. 2.2 and 3.1, Listings 3 and 4): the data-oblivious loop
r += (i++ == in) * a; swap(a, b); a += b, max_iter times.  The initial
values i = 0, a = 0, b = 1, r = 0 are encrypted constants in E3; here they
are input ciphertexts.  The bit-level program keeps i, a, b, r as n-bit
SecureUint (r += e * a is an n-bit AND of e with a then an n-bit ripple add,
sums wrap mod 2^n); the bridged one keeps a, b, r as SecureMod, so the
SecureBool e is cast by Horner's scheme with one bit (the identity) and
r += e * a is one ciphertext multiply and one addition.
"""

from .bridge import AND, MUX, NOT, XNOR


def half_adder_shared(ev, x, y):
    """(x XOR y, x AND y) with one shared multiply (with t = 2 the sum is x + y alone)."""
    p = ev.mul(x, y)
    if ev.prm.t == 2:
        return ev.add(x, y), p
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
            eq = ev.gate(XNOR, a[lo], b[lo]) if need_eq else None
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


def equal(ev, x, y):
    """Encryption of [x == y] for little-endian bit vectors of equal length."""
    e = [ev.gate(XNOR, xi, yi) for xi, yi in zip(x, y)]

    def tree(lo, hi):
        if hi - lo == 1:
            return e[lo]
        mid = lo + (hi - lo) // 2
        return ev.mul(tree(lo, mid), tree(mid, hi))
    return tree(0, len(e))


def increment(ev, x):
    """x + 1 mod 2^n."""
    out = [ev.gate(NOT, x[0])]
    c = x[0]
    for k in range(1, len(x)):
        s, c = half_adder_shared(ev, x[k], c)
        out.append(s)
    return out


def fibonacci_bits(ev, inp, i, a, b, r, max_iter):
    """Listing 3: every variable an n-bit SecureUint (lists of bit ciphertexts)."""
    n = len(inp)
    for _ in range(max_iter):
        e = equal(ev, i, inp)
        i = increment(ev, i)
        r = ripple_add(ev, [ev.gate(AND, e, ak) for ak in a], r)[:n]
        a, b = ripple_add(ev, b, a)[:n], a
    return r


def fibonacci_bridged(ev, inp, i, a, b, r, max_iter):
    """Listing 4: in and i n-bit SecureUint; a, b, r SecureMod ciphertexts."""
    for _ in range(max_iter):
        e = equal(ev, i, inp)
        i = increment(ev, i)
        r = ev.add(r, ev.mul(ev.bits_to_mod([e]), a))
        a, b = ev.add(b, a), a
    return r
