"""Small, self-contained launches for profiling one kernel family under ncu.

python -m paper_2204_12201_gb300.profile_cases ntt --N 16384 --L 8 --polys 256
    forward + inverse NTT over polys x L limbs (256 x 8 x 16384 words = 256 MiB,
    above the 129 MB L2), three rounds; capture with -s 2 -c 2 to skip the first round.
python -m paper_2204_12201_gb300.profile_cases mul --N 16384 --L 8 --n 32
    three batched mul_relin calls of n ciphertext pairs.

The measured rounds run inside the NVTX range "bfhe_cases", so that ncu can
skip the set-up (keygen, encryption) with --nvtx --nvtx-include "bfhe_cases/".
"""

import argparse
import contextlib
import sys


@contextlib.contextmanager
def _range(torch, name):
    """An NVTX push/pop range around the measured rounds (a no-op where NVTX is missing)."""
    try:
        torch.cuda.nvtx.range_push(name)
        pushed = True
    except RuntimeError:
        pushed = False
    try:
        yield
    finally:
        if pushed:
            torch.cuda.nvtx.range_pop()


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["ntt", "mul"])
    ap.add_argument("--N", type=int, default=16384)
    ap.add_argument("--L", type=int, default=8)
    ap.add_argument("--alpha", type=int, default=1)
    ap.add_argument("--polys", type=int, default=256)
    ap.add_argument("--n", type=int, default=32)
    ap.add_argument("--rounds", type=int, default=3)
    a = ap.parse_args(argv)
    import torch

    from . import bfhe
    ctx = bfhe.Context(N=a.N, L=a.L, alpha=a.alpha)
    if a.case == "ntt":
        x = torch.randint(0, 1 << 40, (a.polys, a.L, a.N), dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        with _range(torch, "bfhe_cases"):
            for _ in range(a.rounds):
                ctx.ntt(x)
                ctx.ntt(x, inverse=True)
    else:
        ctx.keygen(1)
        g = torch.Generator().manual_seed(3)
        ys = torch.randint(0, 65537, (2 * a.n, a.N), generator=g, dtype=torch.int64).cuda()
        ct = ctx.encrypt(ys, 5)
        x, y = ct[: a.n].contiguous(), ct[a.n:].contiguous()
        out = torch.empty_like(x)
        torch.cuda.synchronize()
        with _range(torch, "bfhe_cases"):
            for _ in range(a.rounds):
                ctx.mul_relin(x, y, out=out)
    torch.cuda.synchronize()
    ctx.close()
    print("ok")
    return 0


if __name__ == "__main__":
    sys.exit(main())
