"""GB300 library for the bridged BFV arithmetic of Chielle et al. (ICCAD'22).

`bfhe` is the Python binding of the CUDA library's C ABI (include/bfhe.h);
`circuits` builds levelised gate tables for bit-level circuits; `inputs`
holds the seeded synthetic input generators (no FHE arithmetic).
"""
