"""Continuous-batching request loop for bridged-FHE jobs.

Two kinds of request, each on one ring degree N:
* chain: n ciphertexts (slot vectors encrypted on admission) go through `depth` successive squarings (the
  multiply chain every Fermat equality test of the bridge is made of, Listing 7);
* bridge: one SecureMod -> SecureUint<s> conversion (Eq. 2, Listing 8, select mode) of n ciphertexts whose
  slots hold values below 2^s: the n 2^s differences x - c (c = 0 .. 2^s - 1) are the request's chains of
  squarings, batched with every other request's chains; when they reach x^(t-1), 1 - d_c is summed into the
  s bits.

The server keeps one context per ring degree with its keys resident and runs iteration-level (continuous)
batching: at every step each ring degree with work does ONE batched mul_relin over the current ciphertexts
of all its active requests, on its own CUDA stream so the three ring degrees overlap on the device; a request
leaves the batch when its chains are done and a newly arrived one joins at the next step.

Admission, first come first served, is by device memory: a request is admitted while the memory the process
holds on the device stays within the budget after it joins.  That memory is the contexts' resident tables
and keys, their scratch arenas (which grow to the largest batched multiply and never shrink: the arena of the
request's ring is projected to the batch it joins), the buffers of all active requests (current and next
ciphertexts, and a bridge request's input, difference and bit buffers), and the blocks the tensor allocator
keeps cached.  The baseline serves one request at a time with per-op launches (one multiply call per
ciphertext per level).

Scheduling is host-side logic over a small backend interface, so the policy is testable without a GPU
(tests/test_serving.py drives it with a fake backend).
"""

import dataclasses
import time

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    N: int
    depth: int                         # chain: squarings; bridge: set on admission (squarings to x^(t-1))
    n: int
    arrival: float                     # seconds after the stream starts
    seed: int
    kind: str = "chain"                # "chain" or "bridge"
    s: int = 0                         # bridge: output bits (candidates c = 0 .. 2^s - 1)
    cur: object = None                 # device ciphertexts [units][2][L][N]
    x: object = None                   # bridge: the encrypted input [n][2][L][N]
    level: int = 0
    t_admit: float = None
    t_done: float = None
    done_event: object = None
    result: object = None

    def units(self):
        """Ciphertexts the request puts into every batched multiply step."""
        return self.n << self.s if self.kind == "bridge" else self.n


def poisson_stream(seed, n_req, rate, ring_degrees=(4096, 8192, 16384), depth=(1, 16), cts=(1, 64), bridge=0.0,
                   bits=(2, 4)):
    """n_req requests with exponential inter-arrival times (mean 1/rate); a fraction `bridge` of them are
    bridge conversions of `bits` output bits (their n drawn from the lower quarter of `cts`)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for i in range(n_req):
        t += rng.exponential(1.0 / rate)
        N = int(rng.choice(ring_degrees))
        d = int(rng.integers(depth[0], depth[1] + 1))
        n = int(rng.integers(cts[0], cts[1] + 1))
        if bridge > 0 and rng.random() < bridge:
            sb = int(rng.integers(bits[0], bits[1] + 1))
            out.append(Request(rid=i, N=N, depth=0, n=max(1, n // 4), arrival=t, seed=10_000 + i, kind="bridge",
                               s=sb))
        else:
            out.append(Request(rid=i, N=N, depth=d, n=n, arrival=t, seed=10_000 + i))
    return out


class GpuBackend:
    """Contexts per ring degree (keys resident), one CUDA stream each."""

    PARAMS = {4096: dict(L=2, alpha=1), 8192: dict(L=4, alpha=1), 16384: dict(L=8, alpha=1)}

    def __init__(self, ring_degrees=(4096, 8192, 16384), key_seed=1, device=0):
        import torch

        from . import bfhe
        self.torch = torch
        self.ctx, self.stream = {}, {}
        for N in ring_degrees:
            c = bfhe.Context(N=N, device=device, **self.PARAMS[N])
            c.keygen(key_seed)
            self.ctx[N] = c
            self.stream[N] = torch.cuda.Stream(device)
        torch.cuda.synchronize(device)

    def ct_bytes(self, N):
        return 2 * self.ctx[N].L * N * 8

    def mul_scratch_bytes(self, N, n):
        """Arena one batched multiply of n ciphertexts needs: the library tiles a batch whose scratch exceeds
        its scratch budget, so the arena stops growing at the largest whole tile under that budget."""
        from . import bfhe
        c = self.ctx[N]
        per = c.mul_scratch_bytes(1)
        cap = max(per, bfhe.scratch_budget() // per * per)
        return min(n * per, cap)

    def resident_bytes(self):
        """Tables and keys of every context (held for the server's lifetime)."""
        tot = 0
        for c in self.ctx.values():
            d = c.device_bytes()
            tot += d["tables"] + d["keys"] + d["other"]
        return tot

    def arena_bytes(self, N):
        return self.ctx[N].device_bytes()["scratch"]

    def cache_bytes(self):
        """Device memory the tensor allocator holds in freed, cached blocks."""
        return self.torch.cuda.memory_reserved() - self.torch.cuda.memory_allocated()

    def fermat_depth(self, N):
        """Squarings of Listing 7 for x^(t-1) when t - 1 is a power of two (t = 65537: 16)."""
        e = self.ctx[N].t - 1
        assert e & (e - 1) == 0, "bridge requests need t - 1 to be a power of two"
        return e.bit_length() - 1

    def slots(self, req):
        g = np.random.Generator(np.random.PCG64(req.seed))
        hi = (1 << req.s) if req.kind == "bridge" else 65537
        return g.integers(0, hi, size=(req.n, req.N), dtype=np.int64)

    def encrypt(self, req):
        torch = self.torch
        with torch.cuda.stream(self.stream[req.N]):
            s = torch.from_numpy(self.slots(req)).to("cuda", non_blocking=False)
            return self.ctx[req.N].encrypt(s, req.seed)

    def chains(self, N, x, C):
        """The differences x - c for c = 0 .. C - 1, laid out [C][n]."""
        torch = self.torch
        with torch.cuda.stream(self.stream[N]):
            return torch.cat([self.ctx[N].sub_const(x, c) for c in range(C)])

    def finish(self, N, d, n, s):
        """bits[k] = sum over candidates c with bit k set of 1 - d_c (d_c = (x - c)^(t-1)): [s][n]."""
        torch = self.torch
        ctx = self.ctx[N]
        with torch.cuda.stream(self.stream[N]):
            eq = ctx.const_sub(1, d)
            bits = []
            for k in range(s):
                acc = None
                for c in range(1 << s):
                    if (c >> k) & 1:
                        t = eq[c * n:(c + 1) * n]
                        acc = t.clone() if acc is None else ctx.add(acc, t, out=acc)
                bits.append(acc)
            return torch.stack(bits)

    def square(self, N, x):
        torch = self.torch
        with torch.cuda.stream(self.stream[N]):
            return self.ctx[N].mul_relin(x, x)

    def cat(self, N, xs):
        torch = self.torch
        with torch.cuda.stream(self.stream[N]):
            return torch.cat(xs) if len(xs) > 1 else xs[0]

    def event(self, N):
        torch = self.torch
        e = torch.cuda.Event()
        e.record(self.stream[N])
        return e

    def synchronize(self):
        self.torch.cuda.synchronize()

    def close(self):
        for c in self.ctx.values():
            c.close()


class Server:
    def __init__(self, backend, mem_budget_bytes):
        self.b = backend
        self.budget = mem_budget_bytes
        self.used = 0          # bytes of the active requests' buffers
        self.steps = 0
        self.muls = 0
        self.max_batch = {}
        self.peak = 0          # largest device memory the admission check projected

    def need(self, req):
        """Device bytes a request's buffers take while it is active: current and next ciphertexts of its
        chains, and for a bridge its input, the candidates' terms 1 - d_c and its bits."""
        ct = self.b.ct_bytes(req.N)
        extra = (req.n + (req.n << req.s) + req.s * req.n) * ct if req.kind == "bridge" else 0
        return 2 * req.units() * ct + extra

    def _footprint(self, active_units, extra_req=None):
        """Projected device memory: resident tables and keys, the allocator's cache, the active buffers and the
        arenas grown to the batches (including extra_req's ring with it joined)."""
        tot = self.b.resident_bytes() + self.b.cache_bytes() + self.used
        rings = set(active_units) | ({extra_req.N} if extra_req is not None else set())
        for N in rings:
            units = active_units.get(N, 0) + (extra_req.units() if extra_req is not None and extra_req.N == N else 0)
            tot += max(self.b.arena_bytes(N), self.b.mul_scratch_bytes(N, units) if units else 0)
        if extra_req is not None:
            tot += self.need(extra_req)
        return tot

    def fits(self, req, active):
        units = {N: sum(r.units() for r in act) for N, act in active.items() if act}
        f = self._footprint(units, req)
        if f <= self.budget:
            self.peak = max(self.peak, f)
            return True
        return False

    def start(self, r):
        if r.kind == "bridge":
            r.depth = self.b.fermat_depth(r.N)
            r.x = self.b.encrypt(r)
            r.cur = self.b.chains(r.N, r.x, 1 << r.s)
        else:
            r.cur = self.b.encrypt(r)

    def run(self, requests, clock=time.perf_counter, sleep=time.sleep):
        """Serve the stream in wall-clock time; returns the requests with t_admit / t_done set."""
        pending = sorted(requests, key=lambda r: r.arrival)
        for r in pending:
            if not self.fits(r, {}):
                raise ValueError("request %d alone exceeds the memory budget" % r.rid)
        self.peak = 0
        active = {}            # N -> [Request]
        inflight = {}          # N -> [event of previous steps]
        finished = []
        t0 = clock()
        while pending or any(active.values()):
            now = clock() - t0
            # admit arrived requests first come first served while device memory allows
            while pending and pending[0].arrival <= now and self.fits(pending[0], active):
                r = pending.pop(0)
                self.used += self.need(r)
                r.t_admit = now
                self.start(r)
                active.setdefault(r.N, []).append(r)
            progressed = False
            for N, act in active.items():
                if not act:
                    continue
                # keep at most two steps in flight per ring degree
                q = inflight.setdefault(N, [])
                while len(q) >= 2:
                    q.pop(0).synchronize()
                x = self.b.cat(N, [r.cur for r in act])
                y = self.b.square(N, x)
                self.steps += 1
                self.muls += x.shape[0]
                self.max_batch[N] = max(self.max_batch.get(N, 0), x.shape[0])
                off = 0
                still = []
                for r in act:
                    u = r.units()
                    r.cur = y[off:off + u]
                    off += u
                    r.level += 1
                    if r.level >= r.depth:
                        r.result = self.b.finish(N, r.cur, r.n, r.s) if r.kind == "bridge" else r.cur
                        r.done_event = self.b.event(N)
                        finished.append(r)
                    else:
                        still.append(r)
                active[N] = still
                q.append(self.b.event(N))
                progressed = True
            # completions: poll events, release memory
            for r in finished:
                if r.t_done is None and r.done_event is not None and r.done_event.query():
                    r.t_done = clock() - t0
                    self.used -= self.need(r)
            if not progressed and pending:
                wait = pending[0].arrival - (clock() - t0)
                if wait > 0:
                    sleep(max(0.0, min(wait, 0.002)))
                elif not self.fits(pending[0], active):
                    # memory-bound: wait for a completion
                    for r in finished:
                        if r.t_done is None:
                            r.done_event.synchronize()
                            r.t_done = clock() - t0
                            self.used -= self.need(r)
                            break
        self.b.synchronize()
        for r in finished:
            if r.t_done is None:
                r.t_done = clock() - t0
                self.used -= self.need(r)
        return finished


def serve_sequential(backend, requests, clock=time.perf_counter, sleep=time.sleep):
    """Baseline: one request at a time in arrival order, one multiply call per ciphertext per level."""
    t0 = clock()
    out = []
    for r in sorted(requests, key=lambda r: r.arrival):
        while clock() - t0 < r.arrival:
            sleep(max(0.0, min(0.002, r.arrival - (clock() - t0))))
        r.t_admit = clock() - t0
        x = backend.encrypt(r)
        if r.kind == "bridge":
            r.depth = backend.fermat_depth(r.N)
            x = backend.chains(r.N, x, 1 << r.s)
        cts = [x[i:i + 1] for i in range(x.shape[0])]
        for _ in range(r.depth):
            cts = [backend.square(r.N, c) for c in cts]
        y = backend.cat(r.N, cts)
        r.result = backend.finish(r.N, y, r.n, r.s) if r.kind == "bridge" else y
        backend.event(r.N).synchronize()
        r.t_done = clock() - t0
        out.append(r)
    return out


def summarize(reqs):
    lat = np.array([r.t_done - r.arrival for r in reqs])
    muls = sum(r.units() * r.depth for r in reqs)
    span = max(r.t_done for r in reqs) - min(r.arrival for r in reqs)
    return {"requests": len(reqs), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "mul_relin_per_s": muls / span, "requests_per_s": len(reqs) / span,
            "makespan_s": span}


def demo(n_req=40, rate=20.0, seed=5, budget_gb=64.0, bridge=0.25):
    """Mixed stream (a fraction `bridge` of bridge conversions) through both servers; returns their summaries."""
    import copy
    b = GpuBackend()
    reqs = poisson_stream(seed, n_req, rate, bridge=bridge)
    warm = poisson_stream(seed + 1, 3, 1000.0, bridge=0.5)
    Server(b, int(budget_gb * 2**30)).run(warm)
    srv = Server(b, int(budget_gb * 2**30))
    cont = summarize(srv.run(copy.deepcopy(reqs)))
    cont.update(steps=srv.steps, max_batch={str(k): v for k, v in srv.max_batch.items()},
                peak_projected_gb=round(srv.peak / 2**30, 2), bridge_requests=sum(r.kind == "bridge" for r in reqs))
    seq = summarize(serve_sequential(b, copy.deepcopy(reqs)))
    b.close()
    return {"continuous": cont, "sequential_per_op": seq, "rate_per_s": rate, "n_requests": n_req}


if __name__ == "__main__":
    import json
    print(json.dumps(demo()))
