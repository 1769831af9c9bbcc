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


def regrouped_table(log_n, log_e):
    """Where the host puts the forward twiddles for the last pass: position -> standard entry index.
    Stage b < log_e covers [N >> (b+1), N >> b); thread tg's g-th entry there (standard
    (N >> (b+1)) + tg B + g, B = E >> (b+1)) moves to (N >> (b+1)) + g (N / E) + tg."""
    N, E = 1 << log_n, 1 << log_e
    T = N >> log_e
    pos = list(range(N))
    for b in range(log_e):
        lo, B = N >> (b + 1), E >> (b + 1)
        for r in range(lo):
            pos[lo + (r % B) * T + r // B] = lo + r
    return pos


SHAPES = [(log_n, log_m, log_e) for log_n in range(10, 16) for log_m in (log_n - 1, log_n)
          for log_e in (3, 4, 5) if 10 <= log_m <= 14 and not (log_m == 14 and log_e < 4)]


@pytest.mark.parametrize("log_n,log_m,log_e", SHAPES)
def test_forward_last_pass_reads_its_twiddles_from_the_regrouped_table(log_n, log_m, log_e):
    """The last forward pass (W_LO = 0) loads entry (N >> (b+1)) + g (N / E) + tg of the regrouped table,
    tg = (half M + base) / E; that entry must hold the standard twiddle (jb >> (b+1)) + g,
    jb = N + half M + base, stay inside the limb's N entries, and a warp's lanes must read consecutive
    entries."""
    N, E, M = 1 << log_n, 1 << log_e, 1 << log_m
    T = N >> log_e
    table = regrouped_table(log_n, log_e)
    assert sorted(table) == list(range(N))
    npass = (log_m + log_e - 1) // log_e
    hi = log_m - 1 - (npass - 1) * log_e
    assert fwd_wlo(log_m, log_e, npass - 1) == 0 and 0 <= hi < log_e
    for half in range(N // M):
        for tid in range(M >> log_e):
            base = tid << log_e
            tg = ((half << log_m) + base) >> log_e
            jb = N + (half << log_m) + base
            for b in range(hi + 1):
                for g in range(E >> (b + 1)):
                    p = (N >> (b + 1)) + g * T + tg
                    assert 0 < p < N
                    assert table[p] == (jb >> (b + 1)) + g, (half, tid, b, g)
                    if tid % 32:   # the previous lane of the warp reads the entry before
                        tg_prev = ((half << log_m) + ((tid - 1) << log_e)) >> log_e
                        assert p == (N >> (b + 1)) + g * T + tg_prev + 1
