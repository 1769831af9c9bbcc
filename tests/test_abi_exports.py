"""The C-ABI library loads and exports every function include/bfhe.h declares
(no GPU needed: nothing is called but the loader)."""

import ctypes
import os
import re

from paper_2204_12201_gb300 import build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "bfhe.h")


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bfhe_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    path = build.lib_path()
    if not os.path.exists(path):
        build.build()
    lib = ctypes.CDLL(path)
    names = declared()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_abi():
    from paper_2204_12201_gb300 import bfhe
    src = open(bfhe.__file__).read()
    missing = [n for n in declared() if '"%s"' % n not in src]
    assert not missing, missing


def _lib():
    from paper_2204_12201_gb300 import bfhe
    path = build.lib_path()
    if not os.path.exists(path):
        build.build()
    return bfhe.load(), bfhe


def test_context_parameters_are_validated_on_the_host():
    """Every rejected parameter set returns BFHE_EINVAL before any CUDA call (runs without a GPU)."""
    lib, bfhe = _lib()
    bad = [dict(N=1000), dict(N=512), dict(N=65536), dict(L=0), dict(L=33), dict(alpha=0), dict(alpha=3),
           dict(prime_bits=29), dict(prime_bits=59), dict(t=65536), dict(t=17), dict(t=3), dict(t=1),
           dict(t=(1 << 32) + 15)]
    for over in bad:
        kw = dict(N=4096, L=2, alpha=1, prime_bits=50, t=65537)
        kw.update(over)
        prm = bfhe._Params(kw["N"], kw["L"], kw["alpha"], kw["prime_bits"], kw["t"])
        out = ctypes.c_void_p(0)
        rc = lib.bfhe_ctx_create(ctypes.byref(prm), 0, ctypes.byref(out))
        assert rc == -1, over
        assert out.value is None, over
        assert lib.bfhe_last_error().decode()


def test_scratch_budget_setting():
    lib, bfhe = _lib()
    old = bfhe.scratch_budget()
    try:
        with __import__("pytest").raises(bfhe.BfheError):
            bfhe.set_scratch_budget(1000)
        bfhe.set_scratch_budget(64 << 20)
        assert bfhe.scratch_budget() == 64 << 20
    finally:
        bfhe.set_scratch_budget(old)
    assert bfhe.scratch_budget() == old == 16 << 30


def test_error_strings():
    lib, _ = _lib()
    for rc in (0, -1, -2, -3, -4, -5):
        assert lib.bfhe_strerror(rc)


def test_library_parameter_rule_matches_the_oracle():
    """The library's moduli (host-side rule) equal the oracle's for every shape the tests and the
    workloads use, including t = 2 and 55-bit primes (no GPU involved)."""
    from oracle.params import Params
    _, bfhe = _lib()
    cases = [(1024, 2, 1, 12289, 50), (1024, 3, 1, 65537, 50), (1024, 4, 2, 65537, 50), (1024, 16, 2, 65537, 50),
             (1024, 2, 1, 65537, 55), (1024, 3, 1, 2, 50), (4096, 2, 1, 65537, 50), (8192, 4, 1, 65537, 50),
             (16384, 8, 1, 65537, 50), (32768, 16, 2, 65537, 50), (32768, 16, 1, 2, 50), (32768, 4, 2, 65537, 50),
             (1024, 3, 1, 4294957057, 50), (1024, 20, 2, 65537, 50), (1024, 32, 1, 65537, 50),
             (16384, 20, 1, 65537, 50), (32768, 28, 1, 65537, 50)]
    for N, L, alpha, t, bits in cases:
        primes, K = bfhe.param_primes(N, L, alpha, t, bits)
        prm = Params(N=N, L=L, alpha=alpha, t=t, prime_bits=bits)
        assert primes == prm.q + prm.p + prm.b, (N, L, alpha, t, bits)
        assert K == prm.K == L + 1


def test_autotuner_search_space_is_what_the_library_accepts():
    """Every NTT shape the autotuner tries is accepted by bfhe_ntt_config (host only), shapes outside it are
    rejected, and the current configuration is restored afterwards."""
    import pytest
    lib, bfhe = _lib()
    from paper_2204_12201_gb300 import autotune
    for logN in range(10, 16):
        saved = [bfhe.ntt_config(logN, inv) for inv in (0, 1)]
        try:
            tried = set(autotune.shapes(logN))
            assert tried, logN
            for m, e in tried:
                for inv in (0, 1):
                    assert bfhe.ntt_config(logN, inv, m, e) == (m, e)
            for m in range(8, 17):
                for e in range(2, 7):
                    if (m, e) in tried:
                        continue
                    with pytest.raises(bfhe.BfheError):
                        bfhe.ntt_config(logN, 0, m, e)
        finally:
            for inv, (m, e) in enumerate(saved):
                bfhe.ntt_config(logN, inv, m, e)
        assert [bfhe.ntt_config(logN, inv) for inv in (0, 1)] == saved
