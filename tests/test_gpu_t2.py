"""GPU: the t = 2 mode (no batching) against the oracle, bit for bit.

Coefficient encryption, the product of binary polynomials, every gate with
the XOR-free equations, mod_to_bits (its Fermat chain is empty at t = 2) and
the bit-level Fibonacci netlist at N = 1024; the same program decrypted at
N = 32768 with 16 data primes, one instance per ciphertext.
"""

import numpy as np
import pytest
import torch

from oracle import bfv, bridge
from oracle import circuits as ocirc
from oracle.params import Params
from tests.gpu_util import assert_ct_equal, cts_to_device, need_gpu

pytestmark = pytest.mark.gpu

T2 = dict(N=1024, L=3, alpha=1, t=2)


@pytest.fixture(scope="module")
def t2():
    need_gpu()
    import __graft_entry__
    __graft_entry__.build()
    from paper_2204_12201_gb300 import bfhe
    prm = Params(**T2)
    ctx = bfhe.Context(**T2)
    ctx.keygen(9)
    yield prm, ctx, bfv.keygen(prm, 9), bfhe
    ctx.close()


def const_poly(prm, v):
    return [int(v)] + [0] * (prm.N - 1)


def test_slot_calls_are_refused(t2):
    prm, ctx, keys, bfhe = t2
    assert not ctx.batching
    with pytest.raises(bfhe.BfheError):
        ctx.encrypt(torch.zeros(1, prm.N, dtype=torch.int64, device="cuda"), 1)


def test_encrypt_poly_mul_relin(t2):
    prm, ctx, keys, _ = t2
    rng = np.random.default_rng(50)
    m = rng.integers(0, 2, size=(4, prm.N))
    got = ctx.encrypt_poly(torch.from_numpy(m).cuda(), 201)
    want = [bfv.encrypt_poly(prm, keys, [int(v) for v in m[i]], 201, i) for i in range(4)]
    assert_ct_equal(prm, got, want, "encrypt_poly")
    assert np.array_equal(ctx.decrypt_poly(got).cpu().numpy(), m)
    prod = ctx.mul_relin(got[:2], got[2:])
    assert_ct_equal(prm, prod, [bfv.mul_relin(prm, keys, want[i], want[2 + i]) for i in range(2)], "mul_relin")
    dec = ctx.decrypt_poly(prod).cpu().numpy()
    for i in range(2):
        assert [int(v) for v in dec[i]] == bfv.decrypt_poly(prm, keys, bfv.mul_relin(prm, keys, want[i],
                                                                                      want[2 + i]))


def test_gates_t2(t2):
    prm, ctx, keys, _ = t2
    combos = [(x, y, z) for x in (0, 1) for y in (0, 1) for z in (0, 1)]
    cts = [[bfv.encrypt_poly(prm, keys, const_poly(prm, c[i]), 211, 3 * j + i) for i in range(3)]
           for j, c in enumerate(combos)]
    dev = [cts_to_device(prm, [cts[j][i] for j in range(8)]) for i in range(3)]
    for g in range(8):
        ev = bridge.Evaluator(prm, keys)
        want = [ev.gate(g, *cts[j]) for j in range(8)]
        ctx.op_counts(reset=True)
        got = ctx.bit_gate(g, dev[0], dev[1], dev[2])
        assert_ct_equal(prm, got, want, "gate %s at t = 2" % bridge.GATE_NAMES[g])
        assert ctx.op_counts()[:3] == ev.counts()


def test_mod_to_bits_t2(t2):
    prm, ctx, keys, _ = t2
    x = [bfv.encrypt_poly(prm, keys, const_poly(prm, v), 221, v) for v in (0, 1)]
    for mode in (bridge.PAPER, bridge.SELECT):
        ev = bridge.Evaluator(prm, keys)
        want = [ev.mod_to_bits(c, 1, range(2), mode) for c in x]
        got = ctx.mod_to_bits(cts_to_device(prm, x), 1, 0, 1, mode)
        assert_ct_equal(prm, got[0], [w[0] for w in want], "mod_to_bits at t = 2")


def test_fibonacci_bits_t2_matches_oracle(t2):
    prm, ctx, keys, _ = t2
    from paper_2204_12201_gb300 import workloads
    width, max_iter = 2, 3
    job = workloads.FibonacciJob(ctx, "bits", width, max_iter, n=2)
    vals = torch.tensor([[2], [1]], dtype=torch.int64, device="cuda")
    job.set_inputs(vals, 231)
    coeffs = job.input_slots(vals).cpu().numpy()                  # [n_inputs][2][N]
    n_in = coeffs.shape[0]
    job.run()
    got = job.result()
    for b in range(2):
        cts = [bfv.encrypt_poly(prm, keys, [int(v) for v in coeffs[w, b]], 231, w * 2 + b) for w in range(n_in)]
        for w in (0, n_in - 1):
            assert_ct_equal(prm, job.circ.wires[w, b:b + 1], [cts[w]], "input wire %d" % w)
        ev = bridge.Evaluator(prm, keys)
        W = width
        want = ocirc.fibonacci_bits(ev, cts[:W], cts[W:2 * W], cts[2 * W:3 * W], cts[3 * W:4 * W],
                                    cts[4 * W:5 * W], max_iter)
        assert ev.n_mul == job.net.n_mul
        for k, wk in enumerate(want):
            assert_ct_equal(prm, got[k, b:b + 1], [wk], "fibonacci bit %d, instance %d" % (k, b))
    assert job.decrypt().cpu().numpy().ravel().tolist() == [1, 1]   # F(2), F(1)


def test_fibonacci_bits_t2_decrypts_at_n32768():
    need_gpu()
    from paper_2204_12201_gb300 import bfhe, workloads
    ctx = bfhe.Context(N=32768, L=16, alpha=1, t=2)
    ctx.keygen(10)
    vals = torch.arange(12, dtype=torch.int64, device="cuda").view(12, 1)
    job = workloads.FibonacciJob(ctx, "bits", 8, 10, n=12)
    job.set_inputs(vals, 241)
    job.run()
    fib = [0, 1, 1, 2, 3, 5, 8, 13, 21, 34]
    assert job.decrypt().cpu().numpy().ravel().tolist() == fib + [0, 0]
    ctx.close()
