"""GB300 library for the bridged BFV arithmetic of Chielle et al. (ICCAD'22).

Modules:
- `bfhe`: the Python binding of the CUDA library's C ABI (include/bfhe.h).
  `Context` covers keys, encryption (slots, or coefficients at t = 2),
  linear ops, mul_relin, the Sec. 3.1 gates and gate levels, the bridge
  (bits_to_mod, mod_to_bits, sint_to_mod, mod_to_sint, pow), range checks
  and measurement hooks.
- `circuits`: levelised netlists (adder, comparator, multiplier, argmax,
  equality, increment, the Fibonacci programs of Listings 3 and 4),
  run eagerly or replayed as CUDA graphs.
- `workloads`: the genotype-shaped bridged job and the Fibonacci job.
- `serving`: the continuous-batching request loop.
- `autotune`: the NTT block-shape tuner.
- `inputs`: the seeded synthetic input generators (no FHE arithmetic).
- `build`: builds the library in-tree with nvcc for sm_103a.

Nothing here computes on the CPU: without the built library every call
raises.
"""
