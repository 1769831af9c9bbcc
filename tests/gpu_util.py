"""Helpers shared by the GPU parity tests (conversion between the oracle's
polynomials over Z_Q and the library's RNS layout)."""

import numpy as np
import pytest
import torch


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def ct_to_rns(prm, ct):
    """Oracle ciphertext (lists over Z_Q) -> int64 [len(ct)][L][N] residues."""
    return np.array([[[x % q for x in comp] for q in prm.q] for comp in ct], dtype=np.int64)


def poly_to_rns(poly, primes):
    return np.array([[x % q for x in poly] for q in primes], dtype=np.int64)


def cts_to_device(prm, cts):
    return torch.from_numpy(np.stack([ct_to_rns(prm, c) for c in cts])).cuda()


def assert_ct_equal(prm, got, want_cts, what=""):
    """got: tensor [n][2][L][N] from the GPU; want_cts: list of oracle ciphertexts."""
    g = got.cpu().numpy()
    assert g.shape[0] == len(want_cts)
    for i, w in enumerate(want_cts):
        wr = ct_to_rns(prm, w)
        if not np.array_equal(g[i], wr):
            bad = np.argwhere(g[i] != wr)
            raise AssertionError("%s: ciphertext %d differs at %d words, first %s" % (what, i, len(bad), bad[:4].tolist()))


def rns_to_ct(prm, arr):
    """int64 [2][L][N] residues from the device -> oracle ciphertext (two lists over Z_Q)."""
    from oracle import bfv
    a = np.asarray(arr)
    return tuple(bfv.from_rns([[int(v) for v in a[c, i]] for i in range(prm.L)], prm.q) for c in range(a.shape[0]))
