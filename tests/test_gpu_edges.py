"""GPU: empty batches, argument errors and the tiled paths.

* every batched entry point accepts n = 0 and leaves its output untouched;
* argument errors come back as error codes (raised by the binding), the
  context stays usable afterwards;
* with a scratch budget of 1 MiB the multiplies run in tiles of three
  ciphertexts (ragged last tile) and mod_to_bits runs one candidate per
  group; every result equals the untiled one word for word, and one of each
  is checked against the oracle.
"""

import numpy as np
import pytest
import torch

from oracle import bfv, bridge
from oracle.params import Params
from paper_2204_12201_gb300 import inputs
from tests.gpu_util import assert_ct_equal, need_gpu

pytestmark = pytest.mark.gpu

LOW_T = dict(N=1024, L=2, alpha=1, t=12289)


@pytest.fixture(scope="module")
def env():
    need_gpu()
    import __graft_entry__
    __graft_entry__.build()
    from paper_2204_12201_gb300 import bfhe
    ctx = bfhe.Context(**LOW_T)
    ctx.keygen(3)
    prm = Params(**LOW_T)
    yield ctx, prm, bfv.keygen(prm, 3), bfhe
    ctx.close()


def _cts(ctx, n, seed, hi=None):
    hi = ctx.t if hi is None else hi
    vals = inputs.slots(seed, n, ctx.N, hi=hi)
    return ctx.encrypt(torch.from_numpy(vals).cuda(), seed), vals


def test_empty_batches(env):
    ctx, prm, keys, bfhe = env
    e = ctx.empty_ct(0)
    sentinel = torch.full((1, 2, ctx.L, ctx.N), 7, dtype=torch.int64, device="cuda")
    assert ctx.encrypt(torch.empty(0, ctx.N, dtype=torch.int64, device="cuda"), 1).shape[0] == 0
    assert ctx.decrypt(e).shape[0] == 0
    for fn in (ctx.add, ctx.sub, ctx.mul_relin):
        fn(e, e, out=e)
    ctx.add_const(e, 1, out=e)
    ctx.mul_scalar(e, 3, out=e)
    ctx.bit_gate(bridge.AND, e, e, out=e)
    ctx.pow(e, 5, out=e)
    assert ctx.mod_to_bits(e, 2, 0, 3).shape[1] == 0
    assert ctx.mod_to_sint(e, 14, (0, 1), (0, 1)).shape[1] == 0
    assert ctx.sint_to_mod(torch.empty(3, 0, 2, ctx.L, ctx.N, dtype=torch.int64, device="cuda")).shape[0] == 0
    torch.cuda.synchronize()
    assert bool((sentinel == 7).all())


def test_argument_errors_leave_the_context_usable(env):
    ctx, prm, keys, bfhe = env
    a, _ = _cts(ctx, 2, 11)
    with pytest.raises(bfhe.BfheError):
        ctx.mul_relin(a, a.clone(), out=a)                      # out aliases an input
    with pytest.raises(ValueError):
        ctx.mul_relin(a, a[:1].clone())                         # the binding checks batch sizes first
    with pytest.raises(bfhe.BfheError):
        ctx.bit_gate(9, a, a)
    with pytest.raises(bfhe.BfheError):
        ctx.mod_to_bits(a, 2, 0, ctx.t)                         # candidate outside Z_t
    with pytest.raises(bfhe.BfheError):
        ctx.mod_to_bits(a, 2, 0, 3, mode=5)
    with pytest.raises(bfhe.BfheError):
        ctx.mod_to_bits(a, 0, 0, 3)
    with pytest.raises(bfhe.BfheError):
        ctx.sint_to_mod(torch.zeros(14, 2, 2, ctx.L, ctx.N, dtype=torch.int64, device="cuda"))   # 2^14 > t
    with pytest.raises(bfhe.BfheError):
        ctx.mod_to_sint(a, 13, (0, 1), (0, 1))                  # 2^13 < t
    with pytest.raises(bfhe.BfheError):
        ctx.add_const(a, ctx.t)                                 # constant must be < t
    fresh = bfhe.Context(**LOW_T)
    with pytest.raises(bfhe.BfheError):
        fresh.encrypt(torch.zeros(1, ctx.N, dtype=torch.int64, device="cuda"), 1)   # before keygen
    fresh.close()
    y = ctx.mul_relin(a, a)
    assert np.array_equal(ctx.decrypt(y).cpu().numpy(), (ctx.decrypt(a).cpu().numpy() ** 2) % ctx.t)


def test_zero_ciphertext_decrypts_to_zero(env):
    ctx, *_ = env
    z = torch.zeros(2, 2, ctx.L, ctx.N, dtype=torch.int64, device="cuda")
    assert not ctx.decrypt(z).any()
    assert not ctx.mul_relin(z, z.clone()).any()


def test_tiled_paths_equal_untiled(env):
    ctx, prm, keys, bfhe = env
    a, av = _cts(ctx, 7, 21)
    b, bv = _cts(ctx, 7, 22)
    x, xv = _cts(ctx, 1, 23, hi=4)
    bits = torch.stack([ctx.encrypt(torch.from_numpy((bv[:2] >> k) & 1).cuda(), 30 + k) for k in range(13)])

    def run_all():
        return [ctx.mul_relin(a, b), ctx.mul_relin(a, a), ctx.pow(a[:3].contiguous(), 12288),
                ctx.bit_gate(bridge.MUX, a, b, a),
                ctx.mod_to_bits(x, 2, 0, 3, bridge.PAPER), ctx.mod_to_bits(x, 2, 0, 3, bridge.SELECT),
                ctx.sint_to_mod(bits), ctx.mod_to_sint(x, 14, (0, 3), (4095, 4098), bridge.SELECT)]

    ref = run_all()
    old = bfhe.scratch_budget()
    try:
        bfhe.set_scratch_budget(1 << 20)
        tiled = run_all()
    finally:
        bfhe.set_scratch_budget(old)
    for k, (u, v) in enumerate(zip(ref, tiled)):
        assert torch.equal(u, v), k
    ca = bfv.encrypt(prm, keys, [int(v) for v in av[6]], 21, 6)
    cb = bfv.encrypt(prm, keys, [int(v) for v in bv[6]], 22, 6)
    assert_ct_equal(prm, tiled[0][6:7], [bfv.mul_relin(prm, keys, ca, cb)], "tiled mul_relin, last tile")
    cx = bfv.encrypt(prm, keys, [int(v) for v in xv[0]], 23, 0)
    want = bridge.Evaluator(prm, keys).mod_to_bits(cx, 2, range(4), bridge.PAPER)
    for k in range(2):
        assert_ct_equal(prm, tiled[4][k], [want[k]], "tiled mod_to_bits bit %d" % k)
    assert np.array_equal(ctx.decrypt(tiled[0]).cpu().numpy(), (av * bv) % ctx.t)


def test_out_of_range_inputs_are_flagged(env):
    """Kernels raise a context flag on a plaintext value >= t or a ciphertext residue >= q_i
    (values within the lazy ranges, so the arithmetic stays in bounds); bfhe_check reports and clears."""
    ctx, prm, keys, bfhe = env
    ctx.check()                                                   # nothing pending
    good = torch.from_numpy(inputs.slots(41, 2, ctx.N, hi=ctx.t)).cuda()
    a = ctx.encrypt(good, 41)
    ctx.check()
    bad = good.clone()
    bad[1, 5] = ctx.t
    ctx.encrypt(bad, 42)
    with pytest.raises(bfhe.BfheError) as ei:
        ctx.check()
    assert ei.value.flags == 1
    ctx.check()                                                   # cleared
    coeffs = torch.zeros(1, ctx.N, dtype=torch.int64, device="cuda")
    coeffs[0, 3] = ctx.t + 1
    ctx.encrypt_poly(coeffs, 43)
    with pytest.raises(bfhe.BfheError) as ei:
        ctx.check()
    assert ei.value.flags == 1
    ctx.mul_plain(a, bad)
    with pytest.raises(bfhe.BfheError) as ei:
        ctx.check()
    assert ei.value.flags == 1
    r = a.clone()
    r[0, 0, 0, 7] = ctx.primes[0]                                 # residue == q_0
    ctx.mul_relin(r, a)
    with pytest.raises(bfhe.BfheError) as ei:
        ctx.check()
    assert ei.value.flags == 2
    ctx.decrypt(r)
    with pytest.raises(bfhe.BfheError) as ei:
        ctx.check()
    assert ei.value.flags == 2
    y = ctx.mul_relin(a, a)
    ctx.check()
    assert np.array_equal(ctx.decrypt(y).cpu().numpy(), (good.cpu().numpy() ** 2) % ctx.t)
