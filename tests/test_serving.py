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
    """Ciphertexts are int64 arrays [n][4]; squaring is elementwise mod P.  The multiply's arena grows to the
    largest batch (N bytes per ciphertext) and never shrinks, like the library's."""

    FERMAT = 3

    def __init__(self, resident=1000):
        self.calls = []
        self.arena = {}
        self.resident = resident

    def ct_bytes(self, N):
        return N

    def mul_scratch_bytes(self, N, n):
        return n * N

    def resident_bytes(self):
        return self.resident

    def arena_bytes(self, N):
        return self.arena.get(N, 0)

    def cache_bytes(self):
        return 0

    def fermat_depth(self, N):
        return self.FERMAT

    def slots(self, req):
        g = np.random.Generator(np.random.PCG64(req.seed))
        return g.integers(0, P if req.kind == "chain" else 1 << req.s, size=(req.n, 4), dtype=np.int64)

    def encrypt(self, req):
        return self.slots(req)

    def chains(self, N, x, C):
        return np.concatenate([(x - c) % P for c in range(C)])

    def finish(self, N, d, n, s):
        eq = (1 - d) % P
        return np.stack([sum(eq[c * n:(c + 1) * n] for c in range(1 << s) if (c >> k) & 1) % P for k in range(s)])

    def square(self, N, x):
        self.calls.append((N, x.shape[0]))
        self.arena[N] = max(self.arena.get(N, 0), self.mul_scratch_bytes(N, x.shape[0]))
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
    b = FakeBackend()
    x = b.encrypt(req)
    if req.kind == "bridge":
        d = b.chains(req.N, x, 1 << req.s)
        for _ in range(b.FERMAT):
            d = (d * d) % P
        return b.finish(req.N, d, req.n, req.s)
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
    """What the device holds (resident tables, the arenas as grown by the batches, the active buffers) stays
    within the budget at every step."""
    reqs = serving.poisson_stream(4, 20, rate=5000.0, ring_degrees=(4096,), depth=(2, 4), cts=(2, 3))
    b = FakeBackend()
    clk = FakeClock()
    srv = serving.Server(b, mem_budget_bytes=0)
    one = max(srv.need(r) + b.mul_scratch_bytes(r.N, r.units()) for r in reqs) + b.resident
    srv.budget = 2 * one
    held = []
    orig = b.square

    def square(N, x):
        y = orig(N, x)
        held.append(b.resident + srv.used + sum(b.arena.values()))
        return y

    b.square = square
    done = srv.run(copy.deepcopy(reqs), clock=clk, sleep=clk.sleep)
    assert len(done) == len(reqs)
    assert max(held) <= srv.budget and srv.peak <= srv.budget
    assert srv.used == 0
    for r in done:
        assert np.array_equal(r.result, expected(r))


def test_arena_growth_is_charged_on_admission():
    """Two requests whose buffers fit together, but whose joint batch would grow the arena past the budget,
    run one after the other; once the arena has grown it stays charged."""
    r1 = serving.Request(rid=0, N=4096, depth=3, n=4, arrival=0.0, seed=1)
    r2 = serving.Request(rid=1, N=4096, depth=3, n=4, arrival=0.0001, seed=2)
    b = FakeBackend(resident=0)
    srv = serving.Server(b, mem_budget_bytes=0)
    alone = srv.need(r1) + b.mul_scratch_bytes(4096, 4)
    srv.budget = alone + srv.need(r2) + b.mul_scratch_bytes(4096, 2)   # room for both buffers, not both batches
    clk = FakeClock()
    done = srv.run([r1, r2], clock=clk, sleep=clk.sleep)
    assert max(n for _, n in b.calls) == 4          # never one batch of 8
    by = {r.rid: r for r in done}
    assert by[1].t_admit >= by[0].t_done
    for r in done:
        assert np.array_equal(r.result, expected(r))


def test_bridge_requests_batch_with_chains():
    """Bridge conversions (select mode from differences, squarings and sums) share the batched squarings
    with the chain requests of their ring and give the same bits as alone."""
    reqs = serving.poisson_stream(9, 24, rate=3000.0, ring_degrees=(4096, 8192), depth=(1, 4), cts=(1, 8),
                                  bridge=0.5, bits=(1, 3))
    assert any(r.kind == "bridge" for r in reqs) and any(r.kind == "chain" for r in reqs)
    b = FakeBackend()
    clk = FakeClock()
    srv = serving.Server(b, mem_budget_bytes=10**9)
    done = srv.run(copy.deepcopy(reqs), clock=clk, sleep=clk.sleep)
    assert len(done) == len(reqs)
    for r in done:
        assert np.array_equal(r.result, expected(r)), r.rid
    assert srv.muls == sum(r.units() * r.depth for r in done)
    seq = serving.serve_sequential(FakeBackend(), copy.deepcopy(reqs), clock=clk, sleep=clk.sleep)
    for r in seq:
        assert np.array_equal(r.result, expected(r))


def test_request_larger_than_budget_is_rejected():
    reqs = serving.poisson_stream(5, 2, rate=10.0, ring_degrees=(4096,), depth=(1, 1), cts=(8, 8))
    srv = serving.Server(FakeBackend(), mem_budget_bytes=2000)
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
    srv.budget = b.resident + 2 * max(srv.need(r) + b.mul_scratch_bytes(r.N, r.units()) for r in reqs)
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
    from paper_2204_12201_gb300 import bfhe
    b = serving.GpuBackend(ring_degrees=(4096, 8192))
    reqs = serving.poisson_stream(7, 12, rate=500.0, ring_degrees=(4096, 8192), depth=(1, 2), cts=(1, 4),
                                  bridge=0.3, bits=(1, 2))
    assert any(r.kind == "bridge" for r in reqs)
    mixed = serving.Server(b, 8 << 30).run(copy.deepcopy(reqs))
    alone = serving.serve_sequential(b, copy.deepcopy(reqs))
    by_id = {r.rid: r for r in alone}
    for r in mixed:
        assert torch.equal(r.result, by_id[r.rid].result)
        slots = b.slots(r)
        ctx = b.ctx[r.N]
        if r.kind == "bridge":
            # the library's own conversion (Listing 8, select mode) of the same encrypted input, word for word;
            # on the backend's stream, which the encryption was launched on
            with torch.cuda.stream(b.stream[r.N]):
                want = ctx.mod_to_bits(b.encrypt(r), r.s, 0, (1 << r.s) - 1, bfhe.SELECT)
            b.synchronize()
            assert torch.equal(r.result, want)
            continue
        # a chain decrypts to the slot values raised to 2^depth
        got = ctx.decrypt(r.result.contiguous()).cpu().numpy()
        want = slots.copy()
        for _ in range(r.depth):
            want = (want * want) % 65537
        assert np.array_equal(got, want)
    b.close()
