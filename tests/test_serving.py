"""Serving loop policy (host logic) with a fake backend, and on the GPU the
guarantee that a request's result is the same alone and in the mix."""

import copy

import numpy as np
import pytest

from paper_2204_12201_gb300 import serving

P = 2**31 - 1


class FakeEvent:
    def query(self):
        return True

    def synchronize(self):
        pass


class FakeBackend:
    """Ciphertexts are int64 arrays [n][4]; squaring is elementwise mod P."""

    def __init__(self):
        self.calls = []

    def ct_bytes(self, N):
        return N

    def mul_scalar_bytes(self, N, n):
        return 0

    def mul_scratch_bytes(self, N, n):
        return n * N

    def encrypt(self, req):
        g = np.random.Generator(np.random.PCG64(req.seed))
        return g.integers(0, P, size=(req.n, 4), dtype=np.int64)

    def square(self, N, x):
        self.calls.append((N, x.shape[0]))
        return (x * x) % P

    def cat(self, N, xs):
        return np.concatenate(xs)

    def event(self, N):
        return FakeEvent()

    def synchronize(self):
        pass


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 0.001
        return self.t

    def sleep(self, dt):
        self.t += dt


def expected(req):
    x = FakeBackend().encrypt(req)
    for _ in range(req.depth):
        x = (x * x) % P
    return x


def test_continuous_batching_matches_alone_and_batches_across_requests():
    reqs = serving.poisson_stream(3, 30, rate=2000.0, ring_degrees=(4096, 8192), depth=(1, 5), cts=(1, 4))
    b = FakeBackend()
    clk = FakeClock()
    srv = serving.Server(b, mem_budget_bytes=10**9)
    done = srv.run(copy.deepcopy(reqs), clock=clk, sleep=clk.sleep)
    assert sorted(r.rid for r in done) == [r.rid for r in reqs]
    for r in done:
        assert np.array_equal(r.result, expected(r))
        assert r.t_done >= r.t_admit >= r.arrival
    # requests of the same ring degree shared multiplies: fewer calls than one per request level
    assert srv.steps < sum(r.depth for r in reqs)
    assert max(n for _, n in b.calls) > 4
    assert srv.muls == sum(r.n * r.depth for r in reqs)


def test_admission_respects_the_memory_budget():
    reqs = serving.poisson_stream(4, 20, rate=5000.0, ring_degrees=(4096,), depth=(2, 4), cts=(2, 3))
    b = FakeBackend()
    clk = FakeClock()
    srv = serving.Server(b, mem_budget_bytes=0)
    one = max(srv.need(r) for r in reqs)
    srv.budget = 2 * one
    peak = []
    orig = b.square

    def square(N, x):
        peak.append(srv.used)
        return orig(N, x)

    b.square = square
    done = srv.run(copy.deepcopy(reqs), clock=clk, sleep=clk.sleep)
    assert len(done) == len(reqs)
    assert max(peak) <= srv.budget
    assert srv.used == 0
    for r in done:
        assert np.array_equal(r.result, expected(r))


def test_request_larger_than_budget_is_rejected():
    reqs = serving.poisson_stream(5, 2, rate=10.0, ring_degrees=(4096,), depth=(1, 1), cts=(8, 8))
    srv = serving.Server(FakeBackend(), mem_budget_bytes=10)
    with pytest.raises(ValueError):
        srv.run(reqs)


def test_sequential_baseline_matches():
    reqs = serving.poisson_stream(6, 6, rate=1000.0, ring_degrees=(4096, 8192), depth=(1, 3), cts=(1, 3))
    clk = FakeClock()
    done = serving.serve_sequential(FakeBackend(), copy.deepcopy(reqs), clock=clk, sleep=clk.sleep)
    for r in done:
        assert np.array_equal(r.result, expected(r))
    s = serving.summarize(done)
    assert s["requests"] == 6 and s["p99_s"] >= s["p50_s"] > 0


def test_admission_is_first_come_first_served():
    """A request is admitted no earlier than its arrival, and in arrival order: a small request behind
    a large one that does not fit yet waits for it (no overtaking)."""
    reqs = serving.poisson_stream(7, 12, rate=3000.0, ring_degrees=(4096,), depth=(1, 6), cts=(1, 4))
    b = FakeBackend()
    clk = FakeClock()
    srv = serving.Server(b, mem_budget_bytes=0)
    srv.budget = 2 * max(srv.need(r) for r in reqs)
    done = srv.run(copy.deepcopy(reqs), clock=clk, sleep=clk.sleep)
    admitted = sorted(done, key=lambda r: (r.t_admit, r.arrival))
    assert [r.rid for r in admitted] == [r.rid for r in sorted(reqs, key=lambda r: r.arrival)]
    assert all(r.t_admit >= r.arrival for r in done)


def test_summary_percentiles():
    reqs = [serving.Request(rid=i, N=4096, depth=1, n=2, arrival=float(i), seed=i) for i in range(100)]
    for i, r in enumerate(reqs):
        r.t_done = r.arrival + (i + 1) / 100.0           # latencies 0.01 .. 1.00 s
    s = serving.summarize(reqs)
    assert abs(s["p50_s"] - 0.505) < 1e-9 and abs(s["p99_s"] - 0.9901) < 1e-9
    assert s["requests"] == 100 and abs(s["mul_relin_per_s"] - 200 / (99 + 1.0)) < 1e-9


@pytest.mark.gpu
def test_gpu_result_is_the_same_alone_and_in_the_mix():
    """Bit-exact (the tolerance of every parity check here is equality)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    b = serving.GpuBackend(ring_degrees=(4096, 8192))
    reqs = serving.poisson_stream(7, 10, rate=500.0, ring_degrees=(4096, 8192), depth=(1, 2), cts=(1, 4))
    mixed = serving.Server(b, 8 << 30).run(copy.deepcopy(reqs))
    alone = serving.serve_sequential(b, copy.deepcopy(reqs))
    by_id = {r.rid: r for r in alone}
    for r in mixed:
        assert torch.equal(r.result, by_id[r.rid].result)
        # and it decrypts to the slot values raised to 2^depth
        slots = b.slots(r)
        got = b.ctx[r.N].decrypt(r.result.contiguous()).cpu().numpy()
        want = slots.copy()
        for _ in range(r.depth):
            want = (want * want) % 65537
        assert np.array_equal(got, want)
    b.close()
