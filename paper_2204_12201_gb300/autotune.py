"""NTT shape autotuner.

For each ring degree and direction the library can run a limb's transform
as one CTA of 2^logN words or as two CTAs of half a limb each (the outer
stage fused into the first pass forward, exchanged through a thread-block
cluster inverse), with 2^3, 2^4 or 2^5 words per thread.  The tuner times
every valid shape on the device with CUDA events (a batch of limbs larger
than L2, best of a few repetitions), installs the fastest with
bfhe_ntt_config and caches the choice per GPU name in a JSON file.  The
transform's output does not depend on the shape (canonical residues in a
fixed order), so tuning never changes results.
"""

import json
import os

from . import bfhe

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "ntt_shapes.json")


def shapes(logN):
    out = []
    for m in (logN - 1, logN):
        if 10 <= m <= 14:
            for e in (3, 4, 5):
                if m == 14 and e < 4:
                    continue
                out.append((m, e))
    return out


def time_shape(ctx, x, inverse, reps=5):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.ntt(x, inverse=inverse)
    best = None
    for _ in range(reps):
        e0.record()
        ctx.ntt(x, inverse=inverse)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return best


def tune(ring_degrees=(4096, 8192, 16384, 32768), limbs_bytes=256 << 20, use_cache=True, verbose=False):
    """Pick and install the fastest shape per (ring degree, direction); returns the table."""
    import torch
    name = torch.cuda.get_device_name()
    table = {}
    if use_cache and os.path.exists(CACHE):
        with open(CACHE) as f:
            table = json.load(f).get(name, {})
    for N in ring_degrees:
        logN = N.bit_length() - 1
        for inverse in (0, 1):
            key = "%d/%s" % (N, "inv" if inverse else "fwd")
            if key not in table:
                ctx = bfhe.Context(N=N, L=1, alpha=1)
                limbs = max(1, limbs_bytes // (8 * N))
                x = torch.randint(0, 1 << 40, (limbs, 1, N), dtype=torch.int64, device="cuda")
                timings = {}
                for m, e in shapes(logN):
                    bfhe.ntt_config(logN, inverse, m, e)
                    timings["%d,%d" % (m, e)] = time_shape(ctx, x, inverse)
                best = min(timings, key=timings.get)
                table[key] = {"shape": [int(v) for v in best.split(",")], "ms": timings}
                ctx.close()
                if verbose:
                    print(key, best, timings)
            m, e = table[key]["shape"]
            bfhe.ntt_config(logN, inverse, m, e)
    if use_cache:
        allc = {}
        if os.path.exists(CACHE):
            with open(CACHE) as f:
                allc = json.load(f)
        allc[name] = table
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        with open(CACHE, "w") as f:
            json.dump(allc, f, indent=1)
    return table


if __name__ == "__main__":
    print(json.dumps(tune(use_cache=False, verbose=True), indent=1))
