"""Continuous-batching request loop for bridged-FHE jobs.

A request carries n ciphertexts (slot vectors encrypted on admission) under
one ring degree N and asks for `depth` successive squarings (the multiply
chain every Fermat equality test of the bridge is made of, Listing 7).  The
server keeps one context per ring degree with its keys resident, admits
arrived requests first-come-first-served while their buffers fit a device
memory budget, and runs iteration-level (continuous) batching: at every step
each ring degree with work does ONE batched mul_relin over the current
ciphertexts of all its active requests, on its own CUDA stream so the three
ring degrees overlap on the device; a request leaves the batch when its
chain is done and a newly arrived one joins at the next step.  The baseline
serves one request at a time with per-op launches (one multiply call per
ciphertext per level).

Scheduling is host-side logic over a small backend interface (encrypt,
square, decrypt, memory accounting), so the policy is testable without a
GPU (tests/test_serving.py drives it with a fake backend).
"""

import dataclasses
import time

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    N: int
    depth: int
    n: int
    arrival: float                     # seconds after the stream starts
    seed: int
    cur: object = None                 # device ciphertexts [n][2][L][N]
    level: int = 0
    t_admit: float = None
    t_done: float = None
    done_event: object = None
    result: object = None


def poisson_stream(seed, n_req, rate, ring_degrees=(4096, 8192, 16384), depth=(1, 16), cts=(1, 64)):
    """n_req requests with exponential inter-arrival times (mean 1/rate)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for i in range(n_req):
        t += rng.exponential(1.0 / rate)
        out.append(Request(rid=i, N=int(rng.choice(ring_degrees)), depth=int(rng.integers(depth[0], depth[1] + 1)),
                           n=int(rng.integers(cts[0], cts[1] + 1)), arrival=t, seed=10_000 + i))
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
        c = self.ctx[N]
        L, K, QP = c.L, c.K, c.L + c.alpha
        return n * (4 * (L + K) + 3 * L + L * QP + 2 * QP) * N * 8

    def slots(self, req):
        g = np.random.Generator(np.random.PCG64(req.seed))
        return g.integers(0, 65537, size=(req.n, req.N), dtype=np.int64)

    def encrypt(self, req):
        torch = self.torch
        with torch.cuda.stream(self.stream[req.N]):
            s = torch.from_numpy(self.slots(req)).to("cuda", non_blocking=False)
            return self.ctx[req.N].encrypt(s, req.seed)

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
        self.used = 0
        self.steps = 0
        self.muls = 0
        self.max_batch = {}

    def need(self, req):
        """Device bytes a request holds while active: current and next ciphertexts plus its
        share of the multiply scratch."""
        return req.n * (2 * self.b.ct_bytes(req.N) + self.b.mul_scratch_bytes(req.N, 1))

    def run(self, requests, clock=time.perf_counter, sleep=time.sleep):
        """Serve the stream in wall-clock time; returns the requests with t_admit / t_done set."""
        pending = sorted(requests, key=lambda r: r.arrival)
        for r in pending:
            if self.need(r) > self.budget:
                raise ValueError("request %d alone exceeds the memory budget" % r.rid)
        active = {}            # N -> [Request]
        inflight = {}          # N -> [event of previous steps]
        finished = []
        t0 = clock()
        while pending or any(active.values()):
            now = clock() - t0
            # admit arrived requests first come first served while memory allows
            while pending and pending[0].arrival <= now and self.used + self.need(pending[0]) <= self.budget:
                r = pending.pop(0)
                self.used += self.need(r)
                r.t_admit = now
                r.cur = self.b.encrypt(r)
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
                    r.cur = y[off:off + r.n]
                    off += r.n
                    r.level += 1
                    if r.level >= r.depth:
                        r.result = r.cur
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
                elif self.used + self.need(pending[0]) > self.budget:
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
        cts = [x[i:i + 1] for i in range(r.n)]
        for _ in range(r.depth):
            cts = [backend.square(r.N, c) for c in cts]
        r.result = backend.cat(r.N, cts)
        backend.event(r.N).synchronize()
        r.t_done = clock() - t0
        out.append(r)
    return out


def summarize(reqs):
    lat = np.array([r.t_done - r.arrival for r in reqs])
    muls = sum(r.n * r.depth for r in reqs)
    span = max(r.t_done for r in reqs) - min(r.arrival for r in reqs)
    return {"requests": len(reqs), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "mul_relin_per_s": muls / span, "requests_per_s": len(reqs) / span,
            "makespan_s": span}


def demo(n_req=40, rate=20.0, seed=5, budget_gb=64.0):
    """Mixed stream through both servers; returns their summaries."""
    import copy
    b = GpuBackend()
    reqs = poisson_stream(seed, n_req, rate)
    warm = poisson_stream(seed + 1, 3, 1000.0)
    Server(b, int(budget_gb * 2**30)).run(warm)
    srv = Server(b, int(budget_gb * 2**30))
    cont = summarize(srv.run(copy.deepcopy(reqs)))
    cont.update(steps=srv.steps, max_batch={str(k): v for k, v in srv.max_batch.items()})
    seq = summarize(serve_sequential(b, copy.deepcopy(reqs)))
    b.close()
    return {"continuous": cont, "sequential_per_op": seq, "rate_per_s": rate, "n_requests": n_req}


if __name__ == "__main__":
    import json
    print(json.dumps(demo()))
