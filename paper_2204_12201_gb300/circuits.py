"""Levelised bit-level circuits over the bfhe gate-level entry point.

Sec. 3.1 leaves comparison, addition and multiplication over its
homomorphic gates to ordinary combinational circuits and gives no netlists.  A circuit here is a DAG of two node
kinds: MUL (one relinearised ciphertext product) and LIN (a linear
combination with coefficients in -2..2 plus a multiple of the constant 1).
Every gate equation of Sec. 3.1 is one MUL and one LIN (NOT is a LIN).

Scheduling: a MUL sits one level above its deepest input; a LIN sits on the
level of its deepest input and, inside a level, on a sub-level above the
LINs it reads.  Level d runs as one bfhe_gate_level call holding all its
MULs (one batched multiply), then one call per LIN sub-level (a call may not
read a wire that another entry of the same call writes, and the LINs of a
level read its MULs).  Tables are uploaded once; the whole circuit can be
captured in a CUDA graph and replayed.

Netlists (the same structure the tests' oracle circuits follow):
* ripple-carry adder: p = a b, u = a + b - 2p, q = c u, s = u + c - 2q,
  c' = p + q; bit 0 is a half adder (c_0 = 0); carry out kept;
* less-than comparator: balanced blocks, leaf (lt, eq) = ((1 - a) b,
  1 - (a + b - 2ab)); merge lt = lt_H + eq_H lt_L, eq = eq_H eq_L, eq only
  where a parent uses it; low block = bits [0, n/2);
* shift-add multiplier: partial products a_i b_j, rows added by ripple
  adders (the first row is one bit shorter and zero-extended);
* argmax of three: i1 = [max(s0, s1) < s2], i0 = [s0 < s1] AND NOT i1;
* equality: XNOR per bit (1 - (x + y - 2xy)), then a balanced product tree
  (low half [0, n/2) times high half);
* increment by the public 1: bit 0 = NOT x_0, carry x_0, then half adders,
  top carry dropped;
* at t = 2 (no batching) XOR = x + y and XNOR = 1 - (x + y) are linear, so
  the half adders' sums and the equality's XNORs take no multiply.

Fibonacci (Listings 3 and 4): max_iter rounds of r += (i++ == in) * a;
swap(a, b); a += b, with the initial values as input wires.  Bit-level: a,
b, r are n-bit words (AND of e with a, ripple adds truncated to n bits);
bridged: a, b, r are single SecureMod wires, the SecureBool e is cast by
one-bit Horner (the wire itself), r += e * a is one MUL and one LIN.
"""

import torch

from . import bfhe

MUL, LIN = "mul", "lin"


def lin_code(cc, cx, cy, cz):
    for v in (cc, cx, cy, cz):
        assert -2 <= v <= 2
    return bfhe.OP_LIN | ((((cc + 2) * 5 + (cx + 2)) * 25 + (cy + 2) * 5 + (cz + 2)) << 8)


class Netlist:
    def __init__(self, t=65537):
        self.t = t             # plaintext modulus: at t = 2 XOR and XNOR are linear (Sec. 3.1)
        self.n_inputs = 0
        self.nodes = []        # (kind, args) ; node i is wire n_inputs + i (inputs are declared first)

    # wires -------------------------------------------------------------
    def inputs(self, k):
        assert not self.nodes, "declare inputs first"
        w = list(range(self.n_inputs, self.n_inputs + k))
        self.n_inputs += k
        return w

    def _add(self, kind, args):
        self.nodes.append((kind, args))
        return self.n_inputs + len(self.nodes) - 1

    def mul(self, x, y):
        return self._add(MUL, (x, y))

    def lin(self, terms, const=0):
        """sum coef * wire over at most three (wire, coef) terms, + const * 1."""
        assert 1 <= len(terms) <= 3
        return self._add(LIN, (tuple(terms), const))

    # gates (Sec. 3.1) --------------------------------------------------
    def AND(self, x, y):
        return self.mul(x, y)

    def NOT(self, x):
        return self.lin([(x, -1)], 1)

    def half_adder(self, x, y):
        """(x XOR y, x AND y) sharing one product (at t = 2 the sum does not use it)."""
        p = self.mul(x, y)
        if self.t == 2:
            return self.lin([(x, 1), (y, 1)]), p
        return self.lin([(x, 1), (y, 1), (p, -2)]), p

    def XOR(self, x, y):
        if self.t == 2:
            return self.lin([(x, 1), (y, 1)])
        return self.half_adder(x, y)[0]

    def MUX(self, s, x, y):
        d = self.lin([(x, 1), (y, -1)])
        p = self.mul(s, d)
        return self.lin([(p, 1), (y, 1)])

    # circuits ------------------------------------------------------------
    def ripple_add(self, a, b):
        out, c = [], None
        for i in range(len(b)):
            if i < len(a):
                u, p = self.half_adder(a[i], b[i])
            else:
                u, p = b[i], None
            if c is None:
                out.append(u)
                c = p
                continue
            s, q = self.half_adder(u, c)
            out.append(s)
            c = q if p is None else self.lin([(p, 1), (q, 1)])
        out.append(c)
        return out

    def less_than(self, a, b):
        def block(lo, hi, need_eq):
            if hi - lo == 1:
                na = self.NOT(a[lo])
                lt = self.mul(na, b[lo])
                eq = self.XNOR(a[lo], b[lo]) if need_eq else None
                return lt, eq
            mid = lo + (hi - lo) // 2
            lt_l, eq_l = block(lo, mid, need_eq)
            lt_h, eq_h = block(mid, hi, True)
            t = self.mul(eq_h, lt_l)
            lt = self.lin([(lt_h, 1), (t, 1)])
            eq = self.mul(eq_h, eq_l) if need_eq else None
            return lt, eq
        return block(0, len(a), False)[0]

    def multiply(self, a, b):
        n = len(a)
        rows = [[self.AND(a[i], b[j]) for i in range(n)] for j in range(n)]
        acc = list(rows[0])
        for j in range(1, n):
            acc = acc[:j] + self.ripple_add(acc[j:], rows[j])
        return acc

    def XNOR(self, x, y):
        if self.t == 2:
            return self.lin([(x, -1), (y, -1)], 1)
        p = self.mul(x, y)
        return self.lin([(x, -1), (y, -1), (p, 2)], 1)

    def equal(self, x, y):
        e = [self.XNOR(xi, yi) for xi, yi in zip(x, y)]

        def tree(lo, hi):
            if hi - lo == 1:
                return e[lo]
            mid = lo + (hi - lo) // 2
            return self.mul(tree(lo, mid), tree(mid, hi))
        return tree(0, len(e))

    def increment(self, x):
        out, c = [self.NOT(x[0])], x[0]
        for k in range(1, len(x)):
            sk, c = self.half_adder(x[k], c)
            out.append(sk)
        return out

    def fibonacci_bits(self, inp, i, a, b, r, max_iter):
        n = len(inp)
        for _ in range(max_iter):
            e = self.equal(i, inp)
            i = self.increment(i)
            r = self.ripple_add([self.AND(e, ak) for ak in a], r)[:n]
            a, b = self.ripple_add(b, a)[:n], a
        return r

    def fibonacci_bridged(self, inp, i, a, b, r, max_iter):
        for _ in range(max_iter):
            e = self.equal(i, inp)
            i = self.increment(i)
            r = self.lin([(r, 1), (self.mul(e, a), 1)])
            a, b = self.lin([(b, 1), (a, 1)]), a
        return r

    def argmax3(self, s0, s1, s2):
        lt01 = self.less_than(s0, s1)
        best = [self.MUX(lt01, x, y) for x, y in zip(s1, s0)]
        i1 = self.less_than(best, s2)
        i0 = self.AND(lt01, self.NOT(i1))
        return [i0, i1]

    # scheduling ------------------------------------------------------------
    @property
    def n_wires(self):
        return self.n_inputs + len(self.nodes)

    @property
    def n_mul(self):
        """Multiplicative gates: every Sec. 3.1 gate but NOT has exactly one multiply."""
        return sum(1 for k, _ in self.nodes if k == MUL)

    def schedule(self):
        """[(level, mul_entries, [lin entries per sub-level])] with entries as table rows."""
        level = [0] * self.n_wires
        sub = [0] * self.n_wires
        for i, (kind, args) in enumerate(self.nodes):
            w = self.n_inputs + i
            if kind == MUL:
                level[w] = 1 + max(level[args[0]], level[args[1]])
                sub[w] = -1
            else:
                ins = [x for x, _ in args[0]]
                lv = max(level[x] for x in ins)
                level[w] = lv
                sub[w] = 1 + max([sub[x] for x in ins if level[x] == lv and x >= self.n_inputs] + [-1])
        depth = max(level) if self.nodes else 0
        plan = []
        for d in range(depth + 1):
            muls, lins = [], {}
            for i, (kind, args) in enumerate(self.nodes):
                w = self.n_inputs + i
                if level[w] != d:
                    continue
                if kind == MUL:
                    muls.append([bfhe.OP_MUL, args[0], args[1], 0, w])
                else:
                    terms, const = args
                    ws = [x for x, _ in terms] + [0] * (3 - len(terms))
                    cs = [c for _, c in terms] + [0] * (3 - len(terms))
                    lins.setdefault(sub[w], []).append([lin_code(const, *cs), ws[0], ws[1], ws[2], w])
            subs = [lins[k] for k in sorted(lins)]
            if muls or subs:
                plan.append((d, muls, subs))
        return plan


class Compiled:
    """A netlist's level tables on the device, runnable eagerly or as a CUDA graph.

    per_op=True runs one gate per call instead (the same schedule order, one bfhe_gate_level call and so one
    multiply launch sequence per gate): the per-operation baseline the levelised batching is compared with."""

    def __init__(self, ctx, net, n, per_op=False):
        if net.t != ctx.t:
            raise ValueError("netlist built for t = %d, context has t = %d" % (net.t, ctx.t))
        self.ctx, self.net, self.n = ctx, net, n
        self.calls = []      # (table tensor, n_gates, n_mul)
        for _, muls, subs in net.schedule():
            if per_op:
                for row in muls:
                    self.calls.append(self._table([row], 1))
                for s in subs:
                    for row in s:
                        self.calls.append(self._table([row], 0))
                continue
            if muls:
                self.calls.append(self._table(muls, len(muls)))
            for s in subs:
                self.calls.append(self._table(s, 0))
        self.depth = sum(1 for _, muls, _ in net.schedule() if muls)
        self.wires = torch.zeros(net.n_wires, n, 2, ctx.L, ctx.N, dtype=torch.int64, device=ctx.device)
        self.graph = None

    def _table(self, rows, n_mul):
        t = torch.tensor(rows, dtype=torch.int32, device=self.ctx.device)
        return (t, len(rows), n_mul)

    def set_inputs(self, cts):
        """cts: [n_inputs][n][2][L][N]"""
        self.wires[: self.net.n_inputs].copy_(cts)

    def run(self):
        for t, ng, nm in self.calls:
            self.ctx.gate_level(self.wires, t, ng, nm)

    def capture(self):
        """Record run() as a CUDA graph (after one eager run sized the scratch)."""
        self.run()
        torch.cuda.synchronize(self.ctx.device)
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream(self.ctx.device)
        s.wait_stream(torch.cuda.current_stream(self.ctx.device))
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                self.run()
        torch.cuda.current_stream(self.ctx.device).wait_stream(s)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def out(self, wire_ids):
        return self.wires[list(wire_ids)]
