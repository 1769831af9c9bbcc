"""GPU: the launch accounting the bench's roofline divides by.

For one general multiply and one squaring, each kernel class reports (through bfhe_profile_read) the
algorithmic modmuls and DRAM bytes that include/bfhe.h states per unit; here they are recomputed from those
per-unit formulas and the multiply's shape (limbs transformed forward: the operands over Q u B and the L
digits over Q u P; inverse: the three tensor polys over Q u B and the two key-switch polys over Q u P).
"""

import pytest
import torch

from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def expected(N, L, alpha, n, square):
    K, QP, logN = L + 1, L + alpha, N.bit_length() - 1
    slots = 2 if square else 4
    fwd = slots * n * (L + K) + n * L * QP
    inv = 3 * n * (L + K) + 2 * n * QP
    return {
        "ntt_fwd": (fwd * (N // 2) * logN, 16 * N * fwd),
        "ntt_inv": (inv * (N // 2) * logN, 16 * N * inv),
        "modup": (slots * n * N * (L * (L - 1) // 2 + K * (L - 1)), 8 * slots * n * N * (2 * L + K)),
        "tensor": (4 * n * (L + K) * N, (40 if square else 56) * n * (L + K) * N),
        "scale": (3 * n * N * (2 * L + 3 * K + L * (L - 1) // 2 + K * (L - 1) + K * (K - 1) // 2 + L * (K - 1)),
                  24 * n * N * (2 * L + K)),
        "inner": (2 * L * n * QP * N, 8 * QP * N * (n * (L + 2) + 2 * L)),
        "moddown": (2 * n * N * (alpha * (alpha - 1) // 2 + L * alpha + L + alpha), 16 * n * N * (3 * L + alpha)),
    }


@pytest.mark.parametrize("N,L,alpha", [(1024, 3, 1), (1024, 4, 2)])
def test_profile_counts_follow_the_stated_formulas(N, L, alpha):
    need_gpu()
    import __graft_entry__
    __graft_entry__.build()
    from paper_2204_12201_gb300 import bfhe
    ctx = bfhe.Context(N=N, L=L, alpha=alpha)
    ctx.keygen(1)
    n = 2
    ct = ctx.encrypt(torch.randint(0, ctx.t, (2 * n, N), dtype=torch.int64, device="cuda"), 3)
    a, b = ct[:n].contiguous(), ct[n:].contiguous()
    for square in (False, True):
        y = a if square else b
        ctx.mul_relin(a, y)
        torch.cuda.synchronize()
        ctx.profile(True)
        ctx.mul_relin(a, y)
        prof = ctx.profile_read()
        ctx.profile(False)
        for k, (work, nbytes) in expected(N, L, alpha, n, square).items():
            ms, launches, got_work, got_bytes = prof[k]
            assert launches >= 1 and ms > 0, (k, square)
            assert got_work == work and got_bytes == nbytes, (k, square, got_work, work, got_bytes, nbytes)
    ctx.close()
