"""Plain CPU oracle for bridged BFV arithmetic (Chielle et al., ICCAD'22).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) may import, call or link anything in this package; only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.

The oracle is written for a reader checking it against the paper by eye:
Python arbitrary-precision integers, every polynomial held as a list of N
coefficients over Z_Q (not RNS residues), exact negacyclic products by
Kronecker substitution, and each function citing the passage it follows.

Modules
-------
nt        number theory (Miller-Rabin, modular inverse, primitive roots, CRT)
params    the parameter rule (prime scan, auxiliary base size, Delta)
philox    Philox4x64-10 counter-based generator and the samplers built on it
poly      exact negacyclic products over Z (Kronecker) and a schoolbook pin
bfv       textbook FV: encode/decode, keygen, encrypt, decrypt, linear ops,
          exact multiply (tensor + scale-and-round), relinearisation, noise
bridge    homomorphic gates (Sec. 3.1), Listing 5 (bits to SecureMod),
          Listing 7 (pow), Listing 8 / Eq. 2 (SecureMod to bits), op counts
circuits  ripple-carry adder, comparator, shift-add multiplier and argmax
          built from the oracle's gates

Parity status: every function here is pinned by a ``-m "not gpu"`` test
(tests/test_oracle_*.py) against brute force, closed forms, a library routine
or a homomorphic identity; none is "parity unpinned".
"""
