"""Seeded synthetic inputs shared by the tests, the bench and the oracle leg.

Holds no FHE arithmetic: only numpy draws of plaintext data with the shapes
and distributions of the workloads (slot vectors mod t, bit vectors,
genotype-shaped data).  Every generator takes an explicit seed.
"""

import numpy as np


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def slots(seed, n, N, lo=0, hi=65537):
    """n slot vectors of N values uniform in [lo, hi)."""
    return rng(seed).integers(lo, hi, size=(n, N), dtype=np.int64)


def bit_planes(values, s):
    """Little-endian bit planes [s][...] of non-negative integer arrays."""
    v = np.asarray(values, dtype=np.int64)
    return np.stack([(v >> k) & 1 for k in range(s)])


def genotypes(seed, n_ind, n_targets, n_tags):
    """Tag genotypes in {0, 1, 2} with P = (0.5, 0.35, 0.15): [n_tags][n_ind * n_targets]."""
    g = rng(seed).choice(3, size=(n_tags, n_ind * n_targets), p=[0.5, 0.35, 0.15])
    return g.astype(np.int64)


def weights(seed, n_classes, n_tags, n_targets, n_ind):
    """6-bit weights per (class, tag, target), repeated over the individuals of a slot row:
    [n_classes][n_tags][n_ind * n_targets]."""
    w = rng(seed).integers(0, 64, size=(n_classes, n_tags, n_targets), dtype=np.int64)
    return np.repeat(w[:, :, None, :], n_ind, axis=2).reshape(n_classes, n_tags, n_ind * n_targets)


def residues(seed, n, primes, N, comps=2):
    """n ciphertext-shaped arrays [n][comps][len(primes)][N] of residues uniform in [0, q_i) per limb (random
    ciphertexts: valid multiply inputs that decrypt to nothing in particular)."""
    g = rng(seed)
    out = np.empty((n, comps, len(primes), N), dtype=np.int64)
    for c in range(n):
        for k in range(comps):
            for i, q in enumerate(primes):
                out[c, k, i] = g.integers(0, q, size=N, dtype=np.int64)
    return out
