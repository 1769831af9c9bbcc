"""Writes c3_mul_relin.json: SHA-256 digests of the oracle's keys and multiply outputs at the mod_to_bits
workload's parameters (N = 32768, 16 data primes, 2 special primes, t = 65537).

Only the oracle computes here (oracle/ and the seeded generators of paper_2204_12201_gb300/inputs.py).  One
oracle multiply at these parameters takes about 11 minutes on one core, so the three multiplies run in
spawned processes in parallel:  python tests/golden/make_c3_golden.py
Digests are taken over the little-endian int64 words of the RNS layout the library uses: ciphertexts
[2][L][N] over the data primes, the relinearisation key [L][2][L + alpha][N] over Q u P in coefficient form.
"""

import hashlib
import json
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

CFG = dict(N=32768, L=16, alpha=2, t=65537)
KEY_SEED = 1
INPUT_SEED = 3232
N_IN = 2            # inputs a[0..1], b[0..1]
# (name, left operand, right operand): two general products and one squaring
PRODUCTS = [("ab0", ("a", 0), ("b", 0)), ("ab1", ("a", 1), ("b", 1)), ("aa0", ("a", 0), ("a", 0))]


def digest(arr):
    import numpy as np
    return hashlib.sha256(np.ascontiguousarray(arr, dtype="<i8").tobytes()).hexdigest()


def _setup():
    from oracle import bfv
    from oracle.params import Params
    from paper_2204_12201_gb300 import inputs
    prm = Params(**CFG)
    keys = bfv.keygen(prm, KEY_SEED)
    a = inputs.residues(INPUT_SEED, N_IN, prm.q, prm.N)
    b = inputs.residues(INPUT_SEED + 1, N_IN, prm.q, prm.N)
    return prm, keys, {"a": a, "b": b}


def _product(job):
    import numpy as np
    from oracle import bfv
    name, (xa, ia), (xb, ib) = job
    prm, keys, ins = _setup()
    ct = lambda arr: tuple(bfv.from_rns([[int(v) for v in arr[c, i]] for i in range(prm.L)], prm.q)
                           for c in range(2))
    out = bfv.mul_relin(prm, keys, ct(ins[xa][ia]), ct(ins[xb][ib]))
    return name, digest(np.array([bfv.to_rns(p, prm.q) for p in out], dtype=np.int64))


def main():
    import numpy as np
    from oracle import bfv
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(PRODUCTS)) as pool:
        res = pool.map_async(_product, PRODUCTS)
        prm, keys, ins = _setup()
        qp = prm.q + prm.p
        rlk = np.array([[bfv.to_rns(bj, qp), bfv.to_rns(aj, qp)] for bj, aj in keys.rlk], dtype=np.int64)
        out = {"params": CFG, "key_seed": KEY_SEED, "input_seed": INPUT_SEED, "n_inputs": N_IN,
               "inputs": "paper_2204_12201_gb300.inputs.residues(input_seed, n_inputs, data primes, N) for a, "
                         "input_seed + 1 for b",
               "products": {name: [xa, ia, xb, ib] for name, (xa, ia), (xb, ib) in PRODUCTS},
               "sha256": {"a": digest(ins["a"]), "b": digest(ins["b"]), "sk": digest(np.array(keys.s)),
                          "rlk": digest(rlk)}}
        for name, h in res.get():
            out["sha256"][name] = h
    with open(os.path.join(HERE, "c3_mul_relin.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out["sha256"], indent=1))


if __name__ == "__main__":
    main()
