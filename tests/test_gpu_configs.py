"""GPU: the small workloads at their full sizes, with sampled parity.

* N = 4096, 2 data primes: 64 independent ciphertext pairs through add and
  mul_relin, an 8-bit ripple-carry SecureUint adder on 64 batched operand
  pairs, then bits_to_mod on the 9-bit sums.  All 64 sums and products are
  decrypted against plaintext arithmetic; pairs 0 and 63 are recomputed by
  the oracle from the same seeded encryptions and compared bit for bit at
  every stage.
* N = 8192, 4 data primes: the 16-bit comparator and the 16 x 16 shift-add
  multiplier over 4096 slot-packed operand pairs, run as a captured CUDA
  graph.  The oracle recomputes sampled gates one by one from the input
  wires the device holds (every MUL is one relinearised product of two
  wires, every LIN an exact linear combination), and the multiply count is
  checked against the netlist.
* N = 32768, 16 data primes, 2 special primes: mod_to_bits in paper mode for
  c in 0..255 on x uniform in [0, 255], then bits_to_mod; the bits and the
  round trip decrypt to x, and the multiply count is 256 (8 + 16).
"""

import numpy as np
import pytest
import torch

from oracle import bfv, bridge
from oracle import circuits as ocirc
from oracle.params import Params
from paper_2204_12201_gb300 import inputs
from tests.gpu_util import assert_ct_equal, need_gpu, rns_to_ct

pytestmark = pytest.mark.gpu


def _ctx(cfg, seed):
    need_gpu()
    import __graft_entry__
    __graft_entry__.build()
    from paper_2204_12201_gb300 import bfhe
    ctx = bfhe.Context(**cfg)
    ctx.keygen(seed)
    return ctx


def test_small_workload_full_size():
    cfg = dict(N=4096, L=2, alpha=1)
    from paper_2204_12201_gb300 import circuits
    ctx = _ctx(cfg, 11)
    prm = Params(**cfg)
    N, t, n = prm.N, prm.t, 64
    A = inputs.slots(501, n, N)
    B = inputs.slots(502, n, N)
    a = ctx.encrypt(torch.from_numpy(A).cuda(), 501)
    b = ctx.encrypt(torch.from_numpy(B).cuda(), 502)
    s = ctx.add(a, b)
    p = ctx.mul_relin(a, b)
    assert np.array_equal(ctx.decrypt(s).cpu().numpy(), (A + B) % t)
    assert np.array_equal(ctx.decrypt(p).cpu().numpy(), (A * B) % t)

    X = inputs.slots(503, n, N, hi=256)
    Y = inputs.slots(504, n, N, hi=256)
    net = circuits.Netlist()
    x, y = net.inputs(8), net.inputs(8)
    out = net.ripple_add(x, y)
    planes = np.concatenate([inputs.bit_planes(X, 8), inputs.bit_planes(Y, 8)])      # [16][n][N]
    comp = circuits.Compiled(ctx, net, n)
    comp.set_inputs(ctx.encrypt(torch.from_numpy(planes.reshape(-1, N)).cuda(), 505)
                    .view(16, n, 2, prm.L, N))
    ctx.op_counts(reset=True)
    comp.run()
    assert ctx.op_counts()[2] == net.n_mul * n == 15 * n
    sum_bits = comp.out(out)
    m = ctx.bits_to_mod(sum_bits.contiguous())

    keys = bfv.keygen(prm, 11)
    for j in (0, n - 1):
        aj = bfv.encrypt(prm, keys, [int(v) for v in A[j]], 501, j)
        bj = bfv.encrypt(prm, keys, [int(v) for v in B[j]], 502, j)
        assert_ct_equal(prm, a[j:j + 1], [aj], "a[%d]" % j)
        assert_ct_equal(prm, s[j:j + 1], [bfv.add(prm, aj, bj)], "add[%d]" % j)
        assert_ct_equal(prm, p[j:j + 1], [bfv.mul_relin(prm, keys, aj, bj)], "mul_relin[%d]" % j)
        bits = [bfv.encrypt(prm, keys, [int(v) for v in planes[w, j]], 505, w * n + j) for w in range(16)]
        ev = bridge.Evaluator(prm, keys)
        want = ocirc.ripple_add(ev, bits[:8], bits[8:])
        for k, wk in enumerate(want):
            assert_ct_equal(prm, sum_bits[k, j:j + 1], [wk], "adder[%d] bit %d" % (j, k))
        assert_ct_equal(prm, m[j:j + 1], [ev.bits_to_mod(want)], "bits_to_mod[%d]" % j)
    ctx.close()


def _check_lin(prm, wires, node, w):
    """A LIN node against its definition, limb by limb."""
    terms, const = node
    g = wires[w, 0].cpu().numpy()
    acc = np.zeros_like(g)
    for u, c in terms:
        acc += c * wires[u, 0].cpu().numpy()
    q = np.array(prm.q, dtype=np.int64).reshape(1, -1, 1)
    acc[0, :, 0] += const * np.array([prm.delta % qi for qi in prm.q], dtype=np.int64)
    assert np.array_equal(acc % q, g), "LIN wire %d" % w


@pytest.mark.parametrize("name", ["lt16", "mul16"])
def test_bit_level_circuits_full_size(name):
    cfg = dict(N=8192, L=4, alpha=1)
    from paper_2204_12201_gb300 import circuits
    ctx = _ctx(cfg, 12)
    prm = Params(**cfg)
    N = prm.N
    net = circuits.Netlist()
    x, y = net.inputs(16), net.inputs(16)
    out = [net.less_than(x, y)] if name == "lt16" else net.multiply(x, y)
    X = np.zeros((1, N), dtype=np.int64)
    Y = np.zeros((1, N), dtype=np.int64)
    X[0, :4096] = inputs.slots(601, 1, 4096, hi=1 << 16)[0]
    Y[0, :4096] = inputs.slots(602, 1, 4096, hi=1 << 16)[0]
    planes = np.concatenate([inputs.bit_planes(X, 16), inputs.bit_planes(Y, 16)])
    comp = circuits.Compiled(ctx, net, 1)
    comp.set_inputs(ctx.encrypt(torch.from_numpy(planes.reshape(-1, N)).cuda(), 603).view(32, 1, 2, prm.L, N))
    comp.capture()
    comp.wires[net.n_inputs:].zero_()
    comp.replay()
    torch.cuda.synchronize()
    replayed = comp.wires.clone()
    ctx.op_counts(reset=True)
    comp.run()
    assert ctx.op_counts()[2] == net.n_mul == (57 if name == "lt16" else 256 + 30 + 14 * 31)
    assert torch.equal(comp.wires, replayed)
    del replayed
    assert len(out) == (1 if name == "lt16" else 32)
    keys = bfv.keygen(prm, 12)
    rng = np.random.default_rng(7)
    mul_nodes = [i for i, (k, _) in enumerate(net.nodes) if k == circuits.MUL]
    lin_nodes = [i for i, (k, _) in enumerate(net.nodes) if k == circuits.LIN]
    for i in [mul_nodes[-1], int(rng.choice(mul_nodes))]:
        w = net.n_inputs + i
        u, v = net.nodes[i][1]
        cu = rns_to_ct(prm, comp.wires[u, 0].cpu().numpy())
        cv = rns_to_ct(prm, comp.wires[v, 0].cpu().numpy())
        assert_ct_equal(prm, comp.wires[w], [bfv.mul_relin(prm, keys, cu, cv)], "MUL wire %d" % w)
    for i in [lin_nodes[-1]] + [int(v) for v in rng.choice(lin_nodes, 3)]:
        _check_lin(prm, comp.wires, net.nodes[i][1], net.n_inputs + i)
    ctx.close()


def test_bridge_workload_full_size():
    cfg = dict(N=32768, L=16, alpha=2)
    ctx = _ctx(cfg, 13)
    N = ctx.N
    xs = inputs.slots(701, 1, N, hi=256)
    x = ctx.encrypt(torch.from_numpy(xs).cuda(), 701)
    ctx.op_counts(reset=True)
    bits = ctx.mod_to_bits(x, 8, 0, 255, bridge.PAPER)
    assert ctx.op_counts()[2] == bridge.mod_to_bits_mul_count(256, 8, ctx.t) == 256 * 24
    for k in range(8):
        assert np.array_equal(ctx.decrypt(bits[k].contiguous()).cpu().numpy(), (xs >> k) & 1), "bit %d" % k
    back = ctx.bits_to_mod(bits)
    assert np.array_equal(ctx.decrypt(back).cpu().numpy(), xs)
    ctx.close()
