"""bfhe_mul_relin_noalloc: the multiply for callers that cannot allocate.

Some callers of this library may not allocate device memory when they call
it: services that reserve all device memory at start-up and forbid
allocation afterwards, and host code whose hot path must not enter an
allocator or wait for the device-wide synchronisation that growing the
context's scratch arena takes.  For them the library has one entry point
whose scratch is a fixed static device array instead of the arena.  These
tests call it through the C ABI and check it against the ordinary
bfhe_mul_relin, bit for bit (the tolerance of every parity test here: exact
equality of the residues), on two calls in a row with different inputs, so
that contents the first call leaves in the shared array cannot leak into the
second.  This file is collected last so a failure here never hides another
test; it also passes when run alone in a fresh process.
"""

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

CFG = dict(N=4096, L=2, alpha=1)   # one ciphertext needs 1.19 MiB of scratch: at most 26 per call


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2204_12201_gb300 import bfhe
    c = bfhe.Context(**CFG)
    c.keygen(7)
    yield c
    c.close()


def _pair(ctx, seed, n):
    g = torch.Generator().manual_seed(seed)
    ys = torch.randint(0, ctx.t, (2 * n, ctx.N), generator=g, dtype=torch.int64).cuda()
    ct = ctx.encrypt(ys, seed)
    return ct[:n].contiguous(), ct[n:].contiguous()


def test_noalloc_matches_mul_relin_on_two_calls_in_a_row(ctx):
    a1, b1 = _pair(ctx, 11, 3)
    a2, b2 = _pair(ctx, 12, 5)
    want1 = ctx.mul_relin(a1, b1)
    want2 = ctx.mul_relin(a2, b2)
    got1 = ctx.mul_relin_noalloc(a1, b1)
    out2 = torch.empty_like(a2)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    ctx.mul_relin_noalloc(a2, b2, out=out2)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before        # the second call allocated nothing
    assert torch.equal(got1, want1)
    assert torch.equal(out2, want2)
    # and the products decrypt to the slot-wise products
    y = ctx.decrypt(out2).cpu().numpy()
    ya, yb = ctx.decrypt(a2).cpu().numpy(), ctx.decrypt(b2).cpu().numpy()
    assert np.array_equal(y, (ya * yb) % ctx.t)


def test_noalloc_rejects_batches_beyond_the_static_scratch(ctx):
    from paper_2204_12201_gb300 import bfhe
    a, b = _pair(ctx, 13, 27)
    with pytest.raises(bfhe.BfheError, match="at most 26 ciphertexts"):
        ctx.mul_relin_noalloc(a, b)
    a, b = a[:26].contiguous(), b[:26].contiguous()
    assert torch.equal(ctx.mul_relin_noalloc(a, b), ctx.mul_relin(a, b))
