"""GPU: the paper's example programs, Fibonacci bit-level (Listing 3) and
bridged (Listing 4), through the levelised circuit executor.

At N = 1024 the encrypted inputs made by the library's batched encrypt and
every output ciphertext are compared with the oracle bit for bit; at
N = 32768 with 16 data primes (the paper's ring degree) the decrypted results
of every slot are compared with the plain data-oblivious loop (Listing 2).
"""

import numpy as np
import pytest
import torch

from oracle import bfv, bridge
from oracle import circuits as ocirc
from oracle.params import Params
from tests.gpu_util import assert_ct_equal, need_gpu

pytestmark = pytest.mark.gpu

SMALL = dict(N=1024, L=3, alpha=1)
PAPER_N = dict(N=32768, L=16, alpha=1)


def fib_oblivious(v, max_iter, width):
    i, a, b, r = 0, 0, 1, 0
    for _ in range(max_iter):
        r += (i == v) * a
        i = (i + 1) % (1 << width)
        a, b = b, a
        a += b
    return r


def _ctx(cfg, seed):
    need_gpu()
    import __graft_entry__
    __graft_entry__.build()
    from paper_2204_12201_gb300 import bfhe
    ctx = bfhe.Context(**cfg)
    ctx.keygen(seed)
    return ctx


@pytest.mark.parametrize("kind,width,max_iter", [("bits", 2, 3), ("bridged", 3, 3)])
def test_fibonacci_matches_oracle(kind, width, max_iter):
    from paper_2204_12201_gb300 import workloads
    ctx = _ctx(SMALL, 5)
    prm = Params(**SMALL)
    keys = bfv.keygen(prm, 5)
    job = workloads.FibonacciJob(ctx, kind, width, max_iter, n=1)
    vals = torch.from_numpy(np.random.default_rng(40).integers(0, 1 << width, size=(1, prm.N))).cuda()
    job.set_inputs(vals, 151)
    slots = job.input_slots(vals).cpu().numpy()
    cts = [bfv.encrypt(prm, keys, [int(v) for v in slots[w, 0]], 151, w) for w in range(slots.shape[0])]
    for w, c in enumerate(cts):
        assert_ct_equal(prm, job.circ.wires[w], [c], "input wire %d" % w)
    ctx.op_counts(reset=True)
    job.run()
    assert ctx.op_counts()[2] == job.net.n_mul
    ev = bridge.Evaluator(prm, keys)
    W = width
    if kind == "bits":
        want = ocirc.fibonacci_bits(ev, cts[:W], cts[W:2 * W], cts[2 * W:3 * W], cts[3 * W:4 * W],
                                    cts[4 * W:5 * W], max_iter)
    else:
        want = [ocirc.fibonacci_bridged(ev, cts[:W], cts[W:2 * W], cts[2 * W], cts[2 * W + 1], cts[2 * W + 2],
                                        max_iter)]
    assert ev.n_mul == job.net.n_mul
    got = job.result()
    for k, w in enumerate(want):
        assert_ct_equal(prm, got[k], [w], "%s output %d" % (kind, k))
    ctx.close()


@pytest.mark.parametrize("kind,width,max_iter,hi", [("bridged", 8, 10, 12), ("bits", 4, 5, 8)])
def test_fibonacci_decrypts_at_the_papers_ring_degree(kind, width, max_iter, hi):
    from paper_2204_12201_gb300 import workloads
    ctx = _ctx(PAPER_N, 6)
    job = workloads.FibonacciJob(ctx, kind, width, max_iter, n=1)
    vals = np.random.default_rng(41).integers(0, hi, size=(1, ctx.N))
    job.set_inputs(torch.from_numpy(vals).cuda(), 161)
    job.run()
    got = job.decrypt().cpu().numpy()
    table = np.array([fib_oblivious(v, max_iter, width) for v in range(1 << width)])
    want = table[vals] % (ctx.t if kind == "bridged" else 1 << width)
    assert np.array_equal(got, want)
    ctx.close()
