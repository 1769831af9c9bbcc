"""Autotuner for the NTT block shapes and the multiply's tile.

For each ring degree the library can run a limb's transform as one CTA of 2^logN words or as two CTAs of
half a limb each (the outer stage fused into the first pass forward, exchanged through a thread-block
cluster inverse), with 2^3, 2^4 or 2^5 words per thread.  The multiply launches the forward transform with
lazy outputs and the inverse without its twist, so the tuner times the multiply itself: (1) a batched
mul_relin at a representative number of data primes for every pair of forward and inverse shapes, (2) with
the best pair, the tile (most ciphertexts per multiply launch sequence) over a larger batch.  It times with
CUDA events (best of a few repetitions), installs the winners with bfhe_ntt_config and bfhe_set_mul_tile,
and caches them per GPU name in a JSON file.  Outputs do not depend on shapes or tiles (canonical residues
in a fixed order, checked by the tests), so tuning never changes results.
"""

import json
import os

from . import bfhe

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "autotune.json")
# ring degree -> (data primes, special primes, batch of the shape search): the workloads' parameters
# (at N = 16384 the batch is the genotype step's multiply tile: its squarings launch about 470 ciphertexts at a
# time, in tiles of 128)
REPRESENTATIVE = {1024: (2, 1, 64), 2048: (2, 1, 64), 4096: (2, 1, 64), 8192: (4, 1, 64), 16384: (8, 1, 128),
                  32768: (16, 2, 8)}
TILES = (4, 8, 16, 32, 64, 128, 0)   # 0: as many as the scratch budget holds


def shapes(logN):
    out = []
    for m in (logN - 1, logN):
        if 10 <= m <= 14:
            for e in (3, 4, 5):
                if m == 14 and e < 4:
                    continue
                out.append((m, e))
    return out


def _best_ms(torch, fn, reps=3):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn()
    best = None
    for _ in range(reps):
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return best


def tune_ring(N, verbose=False):
    """Search one ring degree; returns {"fwd", "inv", "tile", "ms"} and installs the result."""
    import torch
    logN = N.bit_length() - 1
    L, alpha, B = REPRESENTATIVE[N]
    ctx = bfhe.Context(N=N, L=L, alpha=alpha)
    ctx.keygen(1)
    g = torch.Generator().manual_seed(1)
    a = ctx.encrypt(torch.randint(0, ctx.t, (4 * B, N), generator=g, dtype=torch.int64).cuda(), 1)
    b = ctx.encrypt(torch.randint(0, ctx.t, (4 * B, N), generator=g, dtype=torch.int64).cuda(), 2)
    o = torch.empty_like(a)
    x, y, z = a[:B], b[:B], o[:B]
    bfhe.set_mul_tile(logN, 0)
    timings = {}
    for fm, fe in shapes(logN):
        bfhe.ntt_config(logN, 0, fm, fe)
        for im, ie in shapes(logN):
            bfhe.ntt_config(logN, 1, im, ie)
            timings["%d,%d/%d,%d" % (fm, fe, im, ie)] = _best_ms(torch, lambda: ctx.mul_relin(x, y, out=z), reps=5)
    best = min(timings, key=timings.get)
    fwd, inv = ([int(v) for v in part.split(",")] for part in best.split("/"))
    bfhe.ntt_config(logN, 0, *fwd)
    bfhe.ntt_config(logN, 1, *inv)
    tiles = {}
    for t in TILES:
        if t and t > 4 * B:
            continue
        bfhe.set_mul_tile(logN, t)
        tiles[str(t)] = _best_ms(torch, lambda: ctx.mul_relin(a, b, out=o))
    tile = int(min(tiles, key=tiles.get))
    bfhe.set_mul_tile(logN, tile)
    ctx.close()
    res = {"fwd": fwd, "inv": inv, "tile": tile, "batch": B, "L": L, "ms_pairs": timings, "ms_tiles": tiles}
    if verbose:
        print(N, fwd, inv, tile)
    return res


def tune(ring_degrees=(4096, 8192, 16384, 32768), use_cache=True, verbose=False):
    """Pick and install the fastest shapes and tile per ring degree; returns {N: result}."""
    import torch
    name = torch.cuda.get_device_name()
    table = {}
    if use_cache and os.path.exists(CACHE):
        with open(CACHE) as f:
            table = json.load(f).get(name, {})
    for N in ring_degrees:
        key = str(N)
        if key not in table:
            table[key] = tune_ring(N, verbose)
        r = table[key]
        logN = N.bit_length() - 1
        bfhe.ntt_config(logN, 0, *r["fwd"])
        bfhe.ntt_config(logN, 1, *r["inv"])
        bfhe.set_mul_tile(logN, r["tile"])
    if use_cache:
        allc = {}
        if os.path.exists(CACHE):
            with open(CACHE) as f:
                allc = json.load(f)
        allc[name] = table
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        with open(CACHE, "w") as f:
            json.dump(allc, f, indent=1)
    return {int(k): v for k, v in table.items() if int(k) in ring_degrees}


if __name__ == "__main__":
    print(json.dumps(tune(use_cache=False, verbose=True), indent=1))
