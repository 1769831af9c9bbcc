"""GPU: mod_to_bits with its candidate tiles replayed from a captured CUDA graph (Sec. 3.2.3, Eq. 2,
Listings 7-8: one Fermat chain per candidate c, then the s products of Listing 8, summed per bit).

With a 4 MiB scratch budget at N = 1024, 2 data primes and t = 12289, a paper-mode call runs two candidates
per tile and a select-mode call four; with graph tiles on, the first tile runs eagerly, the next is captured
and every further full tile replays it (its candidate base read from a device word), and a ragged last tile
runs eagerly.  Every result must equal the untiled eager call word for word, op counts included (the depth
exceeds the noise budget of these parameters, so the check is parity, not decryption); the graph-replayed
bits of one input are also recomputed by the oracle.  Each replay adds exactly one launch
(the word that carries the candidate base), which shows the replay path ran.
"""

import pytest
import torch

from oracle import bfv, bridge
from oracle.params import Params
from paper_2204_12201_gb300 import inputs
from tests.gpu_util import assert_ct_equal, need_gpu

pytestmark = pytest.mark.gpu

LOW_T = dict(N=1024, L=2, alpha=1, t=12289)
BUDGET = 4 << 20


@pytest.fixture(scope="module")
def env():
    need_gpu()
    import __graft_entry__
    __graft_entry__.build()
    from paper_2204_12201_gb300 import bfhe
    ctx = bfhe.Context(**LOW_T)
    ctx.keygen(5)
    yield ctx, bfhe
    ctx.close()


def _run(ctx, bfhe, x, s, lo, hi, mode, graph, budget):
    old = bfhe.scratch_budget()
    ctx.set_graph_tiles(graph)
    try:
        bfhe.set_scratch_budget(budget)
        ctx.op_counts(reset=True)
        l0 = bfhe.launch_count()
        out = ctx.mod_to_bits(x, s, lo, hi, mode)
        torch.cuda.synchronize()
        return out, ctx.op_counts(reset=True), bfhe.launch_count() - l0
    finally:
        bfhe.set_scratch_budget(old)
        ctx.set_graph_tiles(False)


# (mode, candidates lo..hi, candidates per tile at the 4 MiB budget)
CASES = [(bridge.PAPER, 0, 5, 2), (bridge.PAPER, 0, 6, 2), (bridge.SELECT, 0, 11, 4), (bridge.SELECT, 2, 15, 4)]


@pytest.mark.parametrize("mode,lo,hi,per_tile", CASES)
def test_graph_tiles_equal_eager(env, mode, lo, hi, per_tile):
    ctx, bfhe = env
    xv = inputs.slots(61, 2, ctx.N, hi=8)
    x = ctx.encrypt(torch.from_numpy(xv).cuda(), 61)
    s = 4
    ref, ref_counts, _ = _run(ctx, bfhe, x, s, lo, hi, mode, False, 16 << 30)
    eager, eager_counts, eager_launches = _run(ctx, bfhe, x, s, lo, hi, mode, False, BUDGET)
    assert torch.equal(ref, eager) and ref_counts == eager_counts
    total = hi - lo + 1
    replays = total // per_tile - 1
    for rep in range(2):   # the second call reuses the instantiated graph
        got, counts, launches = _run(ctx, bfhe, x, s, lo, hi, mode, True, BUDGET)
        assert torch.equal(got, ref), "graph-replayed bits differ (call %d)" % rep
        assert counts == ref_counts
        assert launches - eager_launches == replays


def test_graph_tiles_match_the_oracle(env):
    ctx, bfhe = env
    prm = Params(**LOW_T)
    keys = bfv.keygen(prm, 5)
    xv = inputs.slots(62, 1, ctx.N, hi=6)
    x = ctx.encrypt(torch.from_numpy(xv).cuda(), 62)
    got, counts, _ = _run(ctx, bfhe, x, 3, 0, 5, bridge.PAPER, True, 2 << 20)   # two candidates per tile
    ev = bridge.Evaluator(prm, keys)
    want = ev.mod_to_bits(bfv.encrypt(prm, keys, [int(v) for v in xv[0]], 62, 0), 3, range(6), bridge.PAPER)
    for k in range(3):
        assert_ct_equal(prm, got[k], [want[k]], "graph-replayed mod_to_bits bit %d" % k)
    assert counts[:3] == ev.counts()


def test_graph_tiles_in_signed_conversion(env):
    """mod_to_sint runs two conversions through the same tile path (Listing 9)."""
    ctx, bfhe = env
    xv = inputs.slots(63, 1, ctx.N, hi=6)
    x = ctx.encrypt(torch.from_numpy(xv).cuda(), 63)
    old = bfhe.scratch_budget()
    try:
        bfhe.set_scratch_budget(BUDGET)
        # six candidates per tile: 13 per conversion give two full tiles and a ragged one
        ref = ctx.mod_to_sint(x, 14, (0, 12), (4088, 4100), bridge.SELECT)
        ctx.set_graph_tiles(True)
        got = ctx.mod_to_sint(x, 14, (0, 12), (4088, 4100), bridge.SELECT)
        torch.cuda.synchronize()
    finally:
        ctx.set_graph_tiles(False)
        bfhe.set_scratch_budget(old)
    assert torch.equal(ref, got)
