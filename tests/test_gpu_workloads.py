"""GPU: NTT shapes (the autotuner's search space), levelised circuits and the
genotype-shaped job against the oracle, bit for bit.

The job is checked twice: at reduced size end to end against the oracle's
own pipeline (encrypt, plain multiplies, addition tree, mod_to_bits in paper
mode, argmax circuit), and at the benchmark's full size in the launch
configuration bench.py times, through properties the oracle can check there:
the first tag ciphertext, the decrypted SecureMod scores and the multiply
count of one step.
"""

import numpy as np
import pytest
import torch

from oracle import bfv, bridge
from oracle import circuits as ocirc
from oracle.params import Params
from tests.gpu_util import assert_ct_equal, ct_to_rns, cts_to_device, need_gpu

pytestmark = pytest.mark.gpu

SMALL = dict(N=1024, L=3, alpha=1)
C4 = dict(N=16384, L=8, alpha=1)


@pytest.fixture(scope="module")
def small():
    need_gpu()
    import __graft_entry__
    __graft_entry__.build()
    from paper_2204_12201_gb300 import bfhe
    prm = Params(**SMALL)
    ctx = bfhe.Context(**SMALL)
    ctx.keygen(3)
    keys = bfv.keygen(prm, 3)
    yield prm, ctx, keys
    ctx.close()


@pytest.mark.parametrize("N", [4096, 16384, 32768])
def test_every_ntt_shape_gives_the_same_transform(N):
    need_gpu()
    from paper_2204_12201_gb300 import autotune, bfhe
    logN = N.bit_length() - 1
    ctx = bfhe.Context(N=N, L=2, alpha=1)
    ctx.keygen(2)
    x = torch.randint(0, 1 << 40, (3, 2, N), dtype=torch.int64, device="cuda")
    x %= torch.tensor(ctx.primes[:2], dtype=torch.int64, device="cuda").view(1, 2, 1)
    cts = ctx.encrypt(torch.randint(0, 65537, (4, N), dtype=torch.int64, device="cuda"), 3)
    saved = [bfhe.ntt_config(logN, inv) for inv in (0, 1)]
    ref_f = ref_m = None
    try:
        for m, e in autotune.shapes(logN):
            for inv in (0, 1):
                bfhe.ntt_config(logN, inv, m, e)
            f = ctx.ntt(x.clone())
            b = ctx.ntt(f.clone(), inverse=True)
            # the multiply's transforms leave lazy words for the tensor and the inner product
            prod = ctx.mul_relin(cts[:2].contiguous(), cts[2:].contiguous())
            if ref_f is None:
                ref_f, ref_m = f, prod
            assert torch.equal(f, ref_f), (m, e)
            assert torch.equal(b, x), (m, e)
            assert torch.equal(prod, ref_m), (m, e)
    finally:
        for inv, (m, e) in enumerate(saved):
            bfhe.ntt_config(logN, inv, m, e)
    ctx.close()


@pytest.mark.parametrize("N,L", [(16384, 8), (32768, 4), (8192, 4)])
def test_large_in_place_batches_match_small_ones(N, L):
    """In-place transforms and multiplies over batches of many waves of CTAs give the same
    words as the same data processed a few limbs at a time."""
    need_gpu()
    from paper_2204_12201_gb300 import bfhe
    ctx = bfhe.Context(N=N, L=L, alpha=1)
    ctx.keygen(5)
    polys = (1 << 28) // (8 * N * L)                       # 256 MiB of limbs
    x = torch.randint(0, 1 << 40, (polys, L, N), dtype=torch.int64, device="cuda")
    x %= torch.tensor(ctx.primes[:L], dtype=torch.int64, device="cuda").view(1, L, 1)
    big = ctx.ntt(x.clone())
    small_ = torch.cat([ctx.ntt(x[i:i + 1].clone()) for i in range(polys)])
    assert torch.equal(big, small_)
    assert torch.equal(ctx.ntt(big, inverse=True), x)
    n = 48
    ys = torch.randint(0, 65537, (2 * n, N), dtype=torch.int64, device="cuda")
    ct = ctx.encrypt(ys, 9)
    a, b = ct[:n].contiguous(), ct[n:].contiguous()
    prod = ctx.mul_relin(a, b)
    one = torch.cat([ctx.mul_relin(a[i:i + 1], b[i:i + 1]) for i in range(n)])
    assert torch.equal(prod, one)
    sq = ctx.mul_relin(a, a)
    assert torch.equal(sq, torch.cat([ctx.mul_relin(a[i:i + 1], a[i:i + 1]) for i in range(n)]))
    ctx.close()


def test_circuits_match_the_oracle_eager_and_graph(small):
    prm, ctx, keys = small
    from paper_2204_12201_gb300 import circuits
    rng = np.random.default_rng(8)
    a_bits = rng.integers(0, 2, size=(3, prm.N))
    b_bits = rng.integers(0, 2, size=(3, prm.N))
    cts = [bfv.encrypt(prm, keys, [int(v) for v in row], 201, i) for i, row in enumerate(list(a_bits) + list(b_bits))]
    ev = bridge.Evaluator(prm, keys)
    want_add = ocirc.ripple_add(ev, cts[:3], cts[3:])
    want_lt = ocirc.less_than(ev, cts[:3], cts[3:])
    want_mul = ocirc.multiply(ev, cts[:2], cts[3:5])
    for build, want in ((lambda n, a, b: n.ripple_add(a, b), want_add),
                        (lambda n, a, b: [n.less_than(a, b)], [want_lt]),
                        (lambda n, a, b: n.multiply(a[:2], b[:2]), want_mul)):
        net = circuits.Netlist()
        a, b = net.inputs(3), net.inputs(3)
        out = build(net, a, b)
        comp = circuits.Compiled(ctx, net, 1)
        comp.set_inputs(cts_to_device(prm, cts)[:, None])
        comp.run()
        got = comp.out(out).clone()
        for k, w in enumerate(want):
            assert_ct_equal(prm, got[k], [w], "circuit output %d" % k)
        comp.wires[net.n_inputs:].zero_()
        comp.capture()
        comp.replay()
        torch.cuda.synchronize()
        assert torch.equal(comp.out(out), got)
        per_op = circuits.Compiled(ctx, net, 1, per_op=True)     # one gate per call, same results
        per_op.set_inputs(cts_to_device(prm, cts)[:, None])
        per_op.run()
        assert torch.equal(per_op.out(out), got) and per_op.depth == comp.depth


def test_genotype_job_matches_the_oracle_pipeline(small):
    """Reduced size: 4 x 200 slots, 1 tag, weights < 2, scores < 4 (s = 2 bits, candidates 0..3)."""
    prm, ctx, keys = small
    from paper_2204_12201_gb300 import workloads
    G, W = workloads.genotype_inputs(31, prm.N, n_ind=4, n_targets=200, n_tags=1, wmax=2)
    job = workloads.GenotypeJob(ctx, n_tags=1, s_bits=2)
    ctx.op_counts(reset=True)
    job.run(torch.from_numpy(G).cuda(), torch.from_numpy(W).cuda(), seed=77, keep=True)
    assert ctx.op_counts()[2] == job.muls_per_run()
    ev = bridge.Evaluator(prm, keys)
    g = bfv.encrypt(prm, keys, [int(v) for v in G[0]], 77, 0)
    assert_ct_equal(prm, job.last["enc"], [g], "tag ciphertext")
    scores = [bfv.mul_plain(prm, g, [int(v) for v in W[c][0]]) for c in range(3)]
    assert_ct_equal(prm, job.last["scores"], scores, "scores")
    bits = [ev.mod_to_bits(scores[c], 2, range(4), bridge.PAPER) for c in range(3)]
    for k in range(2):
        assert_ct_equal(prm, job.last["bits"][k], [bits[c][k] for c in range(3)], "bits %d" % k)
    idx = ocirc.argmax3(ev, *bits)
    assert_ct_equal(prm, job.last["idx"], idx, "argmax index bits")


def test_genotype_job_full_size_properties():
    """The benchmark's step at full size: first tag ciphertext against the oracle, decrypted
    SecureMod scores against plaintext dot products, multiplies per step against the formula."""
    need_gpu()
    import __graft_entry__
    __graft_entry__.build()
    from paper_2204_12201_gb300 import bfhe, workloads
    prm = Params(**C4)
    ctx = bfhe.Context(**C4)
    ctx.keygen(1)
    G, W = workloads.genotype_inputs(1004, prm.N)
    job = workloads.GenotypeJob(ctx)
    ctx.op_counts(reset=True)
    job.run(torch.from_numpy(G).cuda(), torch.from_numpy(W).cuda(), seed=10, keep=True)
    n_mul = ctx.op_counts()[2]
    assert n_mul == job.muls_per_run() == 3 * 4096 * (16 + 12) + job.circuit_muls
    scores = ctx.decrypt(job.last["scores"].contiguous()).cpu().numpy()
    want = (W * G[None]).sum(axis=1) % prm.t
    assert np.array_equal(scores, want) and want.max() < 4096
    keys = bfv.keygen(prm, 1)
    g0 = bfv.encrypt(prm, keys, [int(v) for v in G[0]], 10, 0)
    assert np.array_equal(job.last["enc"][0].cpu().numpy(), ct_to_rns(prm, g0))
    ctx.close()


def test_benchmark_launch_configuration_sampled_against_the_oracle():
    """The bench's squaring launches at N = 16384, L = 8: one mul_relin call squares 468 ciphertexts
    (156 candidates x 3 chains, the tile mod_to_bits forms inside the step), with the context's
    default (fast) base extension; the first and the last outputs are recomputed by the oracle."""
    need_gpu()
    import __graft_entry__
    __graft_entry__.build()
    from paper_2204_12201_gb300 import bfhe, inputs
    prm = Params(**C4)
    ctx = bfhe.Context(**C4)
    ctx.keygen(1)
    assert ctx.fast_extension
    n = 468
    y = inputs.slots(901, n, prm.N, hi=prm.t)
    x = ctx.encrypt(torch.from_numpy(y).cuda(), 902)
    sq = ctx.mul_relin(x, x)
    keys = bfv.keygen(prm, 1)
    for i in (0, n - 1):
        xi = bfv.encrypt(prm, keys, [int(v) for v in y[i]], 902, i)
        assert_ct_equal(prm, sq[i:i + 1], [bfv.mul_relin(prm, keys, xi, xi)], "squaring %d of %d" % (i, n))
    assert np.array_equal(ctx.decrypt(sq).cpu().numpy(), (y * y) % prm.t)
    ctx.close()
