"""Host-side netlist logic: the levelised schedule and the product circuits'
arithmetic, checked on slot values mod t without a GPU.

A plaintext interpreter runs the level tables exactly as the device executes
them (each call reads the wires as they were before the call), so a
scheduling error (a LIN reading a MUL or LIN of its own call) or a wrong
coefficient shows up as a wrong value.  The oracle's circuits give the
expected values and multiply counts.
"""

import random

import pytest

from oracle import circuits as ocirc
from paper_2204_12201_gb300 import bfhe, circuits
from tests.test_oracle_bridge import PlainEvaluator, _bits, _fib_oblivious, _val

T = 65537


def decode_lin(code):
    v = code >> 8
    cz = v % 5 - 2
    cy = (v // 5) % 5 - 2
    cx = (v // 25) % 5 - 2
    cc = (v // 125) - 2
    return cc, cx, cy, cz


def run_plain(net, inputs, t=T):
    """inputs: [n_inputs][slots] -> wire values after every scheduled call."""
    n = len(inputs[0])
    wires = [list(v) for v in inputs] + [None] * len(net.nodes)
    for _, muls, subs in net.schedule():
        for rows in ([muls] if muls else []) + subs:
            before = list(wires)
            for op, x, y, z, w in rows:
                if op == bfhe.OP_MUL:
                    assert before[x] is not None and before[y] is not None
                    wires[w] = [(p * q) % t for p, q in zip(before[x], before[y])]
                else:
                    cc, cx, cy, cz = decode_lin(op)
                    vals = [[0] * n if c == 0 else before[u] for u, c in ((x, cx), (y, cy), (z, cz))]
                    assert all(v is not None for v in vals)
                    wires[w] = [(cc + cx * a + cy * b + cz * d) % t for a, b, d in zip(*vals)]
    return wires


def test_lin_code_round_trip():
    for cc in range(-2, 3):
        for cx in range(-2, 3):
            for cy in range(-2, 3):
                for cz in range(-2, 3):
                    code = circuits.lin_code(cc, cx, cy, cz)
                    assert code & 0xFF == bfhe.OP_LIN and decode_lin(code) == (cc, cx, cy, cz)


@pytest.mark.parametrize("t", [T, 2])
@pytest.mark.parametrize("width,max_iter", [(4, 10), (4, 20), (8, 10)])
def test_fibonacci_netlists_plain(width, max_iter, t):
    vals = list(range(1 << width))
    n = len(vals)
    zero, one = [0] * n, [1] * n
    want = [_fib_oblivious(v, max_iter, width) for v in vals]

    net = circuits.Netlist(t)
    inp, i0, a0, b0, r0 = (net.inputs(width) for _ in range(5))
    out = net.fibonacci_bits(inp, i0, a0, b0, r0, max_iter)
    ins = _bits(vals, width) + [zero] * (2 * width) + [one] + [zero] * (2 * width - 1)
    w = run_plain(net, ins, t)
    assert _val([w[k] for k in out]) == [v % (1 << width) for v in want]
    ev = PlainEvaluator(t, n)
    ocirc.fibonacci_bits(ev, _bits(vals, width), [zero] * width, [zero] * width,
                         [one] + [zero] * (width - 1), [zero] * width, max_iter)
    assert net.n_mul == ev.n_mul

    net = circuits.Netlist(t)
    inp, i0 = net.inputs(width), net.inputs(width)
    a0, b0, r0 = net.inputs(3)
    out = net.fibonacci_bridged(inp, i0, a0, b0, r0, max_iter)
    w = run_plain(net, _bits(vals, width) + [zero] * width + [zero, one, zero], t)
    assert w[out] == [v % t for v in want]
    ev = PlainEvaluator(t, n)
    ocirc.fibonacci_bridged(ev, _bits(vals, width), [zero] * width, zero, one, zero, max_iter)
    assert net.n_mul == ev.n_mul


@pytest.mark.parametrize("t", [T, 2])
def test_arith_netlists_plain(t):
    rng = random.Random(13)
    m = 200
    a = [rng.randrange(256) for _ in range(m)]
    b = [rng.randrange(256) if k % 4 else a[k] for k in range(m)]
    for build, ref, oref in (
            (lambda net, x, y: net.ripple_add(x, y), lambda p, q: p + q, ocirc.ripple_add),
            (lambda net, x, y: [net.less_than(x, y)], lambda p, q: int(p < q),
             lambda ev, x, y: [ocirc.less_than(ev, x, y)]),
            (lambda net, x, y: [net.equal(x, y)], lambda p, q: int(p == q),
             lambda ev, x, y: [ocirc.equal(ev, x, y)]),
            (lambda net, x, y: net.increment(x), lambda p, q: (p + 1) % 256,
             lambda ev, x, y: ocirc.increment(ev, x)),
            (lambda net, x, y: net.multiply(x, y), lambda p, q: p * q, ocirc.multiply)):
        net = circuits.Netlist(t)
        x, y = net.inputs(8), net.inputs(8)
        out = build(net, x, y)
        w = run_plain(net, _bits(a, 8) + _bits(b, 8), t)
        assert _val([w[k] for k in out]) == [ref(p, q) for p, q in zip(a, b)]
        ev = PlainEvaluator(t, m)
        oref(ev, _bits(a, 8), _bits(b, 8))
        assert net.n_mul == ev.n_mul
