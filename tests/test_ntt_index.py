"""Host check of the NTT kernels' shared-memory index arithmetic.

The padded layout stores word j at j + (j >> 4).  Each pass of a block of
2^LOG_M words gives thread tid the words base + (e << W_LO), e < 2^LOG_E.
The kernels compute the padded address as phys(base) plus a compile-time
offset per e, which is exact only if no carry crosses bit 4 when e << W_LO
is added to base.  This walks every shape the library instantiates (forward
and inverse passes, every thread) and checks the identity and that the
addresses of a pass are a permutation within the padded buffer.
"""

import pytest


def phys(j):
    return j + (j >> 4)


def fwd_wlo(log_m, log_e, p):
    hi = log_m - 1 - p * log_e
    return max(hi - log_e + 1, 0)


def inv_wlo(log_m, log_e, p):
    lo = p * log_e
    hi = min(lo + log_e - 1, log_m - 1)
    return lo if hi - lo + 1 == log_e else log_m - log_e


@pytest.mark.parametrize("log_m", [10, 11, 12, 13, 14])
@pytest.mark.parametrize("log_e", [3, 4, 5])
def test_padded_offsets_are_compile_time(log_m, log_e):
    E = 1 << log_e
    threads = 1 << (log_m - log_e)
    npass = (log_m + log_e - 1) // log_e
    for wlo_of in (fwd_wlo, inv_wlo):
        for p in range(npass):
            w = wlo_of(log_m, log_e, p)
            seen = set()
            for tid in range(threads):
                base = (tid & ((1 << w) - 1)) | ((tid >> w) << (w + log_e))
                for e in range(E):
                    j = base + (e << w)
                    assert j < (1 << log_m)
                    off = (e << w) + ((e << w) >> 4)
                    assert phys(j) == phys(base) + off, (log_m, log_e, p, tid, e)
                    seen.add(j)
            assert len(seen) == 1 << log_m
