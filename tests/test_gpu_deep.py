"""GPU: deep circuits at insecure, test-only moduli with more data primes.

The paper's deep bit-level programs and the genotype job's bridge exceed the noise budget of the
workloads' own moduli (8 x 50-bit Q at N = 16384; a depth-36 bit-level program at N = 32768 with 16
primes); parity there is bit-exactness, not decryption.  Here the same circuits run with larger Q
(17 to 32 data primes run the library's runtime-size base-extension and inner-product kernels) and must
decrypt to the plaintext results:

* parity of keys, mul_relin and the squaring path against the oracle at N = 1024 with 20 and 32 data primes;
* the genotype job (mul_plain, addition tree, SecureMod -> SecureUint<7> over c in 0..127 in paper mode,
  the levelised 3-way argmax) at N = 16384 with 20 data primes: decrypted class indices equal the plain
  argmax of the plain scores for all 16,000 packed slots;
* the 8-bit bit-level Fibonacci of Listing 3, 10 iterations (multiplicative depth 36), at N = 32768 with
  28 data primes: every slot decrypts to the plain loop's result.
"""

import numpy as np
import pytest
import torch

from oracle import bfv
from oracle.params import Params
from paper_2204_12201_gb300 import inputs
from tests.gpu_util import assert_ct_equal, cts_to_device, need_gpu, poly_to_rns

pytestmark = pytest.mark.gpu


def _ctx(cfg, seed):
    need_gpu()
    import __graft_entry__
    __graft_entry__.build()
    from paper_2204_12201_gb300 import bfhe
    ctx = bfhe.Context(**cfg)
    ctx.keygen(seed)
    return ctx


@pytest.mark.parametrize("cfg", [dict(N=1024, L=20, alpha=2), dict(N=1024, L=32, alpha=1)])
def test_runtime_size_kernels_match_the_oracle(cfg):
    ctx = _ctx(cfg, 7)
    prm = Params(**cfg)
    keys = bfv.keygen(prm, 7)
    assert ctx.primes == prm.q + prm.p + prm.b and ctx.K == prm.K == prm.L + 1
    assert not ctx.fast_extension
    sk, _, rlk = ctx.export_keys()
    qp = prm.q + prm.p
    assert sk.cpu().numpy().tolist() == keys.s
    want = np.array([[poly_to_rns(bj, qp), poly_to_rns(aj, qp)] for bj, aj in keys.rlk])
    assert np.array_equal(rlk.cpu().numpy(), want)
    y = inputs.slots(91, 4, prm.N, hi=prm.t)
    a = [bfv.encrypt(prm, keys, [int(v) for v in y[i]], 92, i) for i in range(2)]
    b = [bfv.encrypt(prm, keys, [int(v) for v in y[2 + i]], 92, 2 + i) for i in range(2)]
    da, db = cts_to_device(prm, a), cts_to_device(prm, b)
    got = ctx.mul_relin(da, db)
    assert_ct_equal(prm, got, [bfv.mul_relin(prm, keys, a[i], b[i]) for i in range(2)], "mul_relin")
    sq = ctx.mul_relin(da, da)
    assert_ct_equal(prm, sq, [bfv.mul_relin(prm, keys, a[i], a[i]) for i in range(2)], "square")
    assert np.array_equal(ctx.decrypt(got).cpu().numpy(), (y[:2] * y[2:]) % prm.t)
    assert np.array_equal(ctx.decrypt(da).cpu().numpy(), y[:2])
    ctx.close()


def test_genotype_full_depth_decrypts_with_a_larger_modulus():
    from paper_2204_12201_gb300 import workloads
    cfg = dict(N=16384, L=20, alpha=1)
    ctx = _ctx(cfg, 8)
    n_tags, s = 4, 7
    G, W = workloads.genotype_inputs(1104, ctx.N, n_tags=n_tags, wmax=16)
    job = workloads.GenotypeJob(ctx, n_tags=n_tags, s_bits=s)
    idx = job.run(torch.from_numpy(G).cuda(), torch.from_numpy(W).cuda(), seed=12, keep=True).cpu().numpy()
    scores = (W * G[None]).sum(axis=1) % ctx.t                        # [3][N], below 2^7 here
    assert scores.max() < (1 << s)
    assert np.array_equal(ctx.decrypt(job.last["scores"].contiguous()).cpu().numpy(), scores)
    best = np.zeros(ctx.N, dtype=np.int64)                           # ties to the lower index
    best[scores[1] > scores[0]] = 1
    best[scores[2] > np.maximum(scores[0], scores[1])] = 2
    assert np.array_equal(idx[0] + 2 * idx[1], best)
    ctx.close()


def test_bit_level_fibonacci_depth_36_decrypts_with_a_larger_modulus():
    from paper_2204_12201_gb300 import workloads
    cfg = dict(N=32768, L=28, alpha=1)
    ctx = _ctx(cfg, 9)
    job = workloads.FibonacciJob(ctx, "bits", 8, 10, n=1)
    assert job.circ.depth == 36
    vals = np.random.default_rng(43).integers(0, 12, size=(1, ctx.N))
    job.set_inputs(torch.from_numpy(vals).cuda(), 171)
    job.run()
    got = job.decrypt().cpu().numpy()
    fib = [0, 1]
    while len(fib) < 10:
        fib.append(fib[-1] + fib[-2])
    table = np.array(fib + [0, 0])                                    # inputs 10, 11 never match in 10 rounds
    assert np.array_equal(got, table[vals] % 256)
    ctx.close()
