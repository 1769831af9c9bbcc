"""GPU parity at the mod_to_bits workload's exact shape: N = 32768, 16 data primes, 2 special primes,
t = 65537, guarded fast base extension on (the default at this size) and off.

At this shape the multiply's lazy bounds are tightest: 15 reduction-free NTT stages reach 64q, and the
key-switch inner product sums 16 digit products before one reduction.  One oracle multiply takes about 11
minutes here, so tests/golden/make_c3_golden.py (oracle only) stored SHA-256 digests of the oracle's secret
key, relinearisation key and three products of seeded random ciphertexts (two general products in one batch,
one squaring); the test recomputes them on the GPU and compares digests of the same RNS words.
"""

import hashlib
import json
import os

import numpy as np
import pytest
import torch

from paper_2204_12201_gb300 import inputs
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c3_mul_relin.json")


def _digest(t):
    a = t.cpu().numpy() if isinstance(t, torch.Tensor) else t
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<i8").tobytes()).hexdigest()


@pytest.fixture(scope="module")
def c3():
    need_gpu()
    import __graft_entry__
    __graft_entry__.build()
    from paper_2204_12201_gb300 import bfhe
    with open(GOLDEN) as f:
        g = json.load(f)
    p = g["params"]
    ctx = bfhe.Context(N=p["N"], L=p["L"], alpha=p["alpha"], t=p["t"])
    ctx.keygen(g["key_seed"])
    yield ctx, g
    ctx.close()


def test_keys_and_inputs_match_the_oracle(c3):
    ctx, g = c3
    sk, _, rlk = ctx.export_keys()
    torch.cuda.synchronize()
    assert _digest(sk) == g["sha256"]["sk"]
    assert _digest(rlk) == g["sha256"]["rlk"]
    q = ctx.primes[:ctx.L]
    assert _digest(inputs.residues(g["input_seed"], g["n_inputs"], q, ctx.N)) == g["sha256"]["a"]
    assert _digest(inputs.residues(g["input_seed"] + 1, g["n_inputs"], q, ctx.N)) == g["sha256"]["b"]


@pytest.mark.parametrize("fast", [True, False])
def test_products_match_the_oracle(c3, fast):
    ctx, g = c3
    assert ctx.fast_extension            # the default from 8 data primes up
    q = ctx.primes[:ctx.L]
    a = torch.from_numpy(inputs.residues(g["input_seed"], g["n_inputs"], q, ctx.N)).cuda()
    b = torch.from_numpy(inputs.residues(g["input_seed"] + 1, g["n_inputs"], q, ctx.N)).cuda()
    try:
        ctx.set_fast_extension(fast)
        ab = ctx.mul_relin(a, b)                 # general products, one batch of two
        x = a[0:1].contiguous()
        aa = ctx.mul_relin(x, x)                 # the squaring path (both operands one buffer)
        torch.cuda.synchronize()
    finally:
        ctx.set_fast_extension(True)
    assert _digest(ab[0]) == g["sha256"]["ab0"]
    assert _digest(ab[1]) == g["sha256"]["ab1"]
    assert _digest(aa[0]) == g["sha256"]["aa0"]
