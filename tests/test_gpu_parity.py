"""GPU parity: the CUDA library against the oracle, bit for bit, through the C ABI.

Every compared output is an integer array (RNS residues, slot values, key
coefficients), so the bar is exact equality.  Inputs are seeded; ciphertext
inputs are made by the oracle and uploaded, so each operation is checked on
its own; encryption and key generation are compared separately.
"""

import random

import numpy as np
import pytest
import torch

from oracle import bfv, bridge
from oracle.params import Params
from paper_2204_12201_gb300 import inputs
from tests.gpu_util import assert_ct_equal, ct_to_rns, cts_to_device, need_gpu, poly_to_rns

pytestmark = pytest.mark.gpu

C1 = dict(N=4096, L=2, alpha=1)            # the small workload's parameters
SMALL = dict(N=1024, L=3, alpha=1)         # odd limb count, ragged vs. template sizes
ALPHA2 = dict(N=1024, L=4, alpha=2)        # two special primes (mod-down by a 2-prime CRT)
WIDE = dict(N=32768, L=2, alpha=2)         # N = 32768: the two-pass NTT path
LOW_T = dict(N=1024, L=2, alpha=1, t=12289)  # t - 1 = 3 * 2^12: pow with an odd step
MID = dict(N=16384, L=2, alpha=1)          # N = 16384: split-half forward NTT, whole-limb inverse
C4 = dict(N=16384, L=8, alpha=1)           # the benchmark's parameters
L16 = dict(N=1024, L=16, alpha=2)          # the largest limb count, two special primes (the bridge workload's)
BIG_Q = dict(N=1024, L=2, alpha=1, prime_bits=55)   # primes above 2^50: the multiply's transforms stay canonical
BIG_T = dict(N=1024, L=3, alpha=1, t=4294957057)    # the largest t = 1 mod 2048 below 2^32: (t - 1)^2 > 2^63


class Pair:
    """A GPU context and the oracle for the same parameters and key seed."""

    def __init__(self, cfg, seed=1):
        from paper_2204_12201_gb300 import bfhe
        need_gpu()
        self.bfhe = bfhe
        self.prm = Params(**cfg)
        kw = dict(cfg)
        self.ctx = bfhe.Context(**kw)
        self.ctx.keygen(seed)
        self.keys = bfv.keygen(self.prm, seed)

    def enc(self, vals, seed, idx):
        return bfv.encrypt(self.prm, self.keys, [int(v) for v in vals], seed, idx)


_pairs = {}


def pair(name, cfg):
    if name not in _pairs:
        _pairs[name] = Pair(cfg)
    return _pairs[name]


@pytest.mark.parametrize("name,cfg", [("C1", C1), ("SMALL", SMALL), ("ALPHA2", ALPHA2), ("WIDE", WIDE),
                                      ("LOW_T", LOW_T), ("BIG_T", BIG_T)])
def test_params_and_keys(name, cfg):
    P = pair(name, cfg)
    prm = P.prm
    assert P.ctx.primes == prm.q + prm.p + prm.b and P.ctx.K == prm.K
    sk, pk, rlk = P.ctx.export_keys()
    torch.cuda.synchronize()
    assert sk.cpu().numpy().tolist() == P.keys.s
    assert np.array_equal(pk.cpu().numpy(), ct_to_rns(prm, (P.keys.pk0, P.keys.pk1)))
    qp = prm.q + prm.p
    want = np.array([[poly_to_rns(bj, qp), poly_to_rns(aj, qp)] for bj, aj in P.keys.rlk])
    assert np.array_equal(rlk.cpu().numpy(), want)


@pytest.mark.parametrize("name,cfg", [("C1", C1), ("WIDE", WIDE), ("MID", MID)])
def test_ntt_convolution(name, cfg):
    """INTT(NTT(a) . NTT(b)) equals the exact negacyclic product mod q; INTT(NTT(a)) = a."""
    from oracle.poly import negacyclic
    P = pair(name, cfg)
    prm = P.prm
    N, L = prm.N, prm.L
    rng = random.Random(5)
    a = [[rng.randrange(q) for _ in range(N)] for q in prm.q]
    b = [[rng.randrange(q) for _ in range(N)] for q in prm.q]
    da = torch.tensor([a], dtype=torch.int64).cuda()
    db = torch.tensor([b], dtype=torch.int64).cuda()
    P.ctx.ntt(da)
    P.ctx.ntt(db)
    fa, fb = da.cpu().numpy(), db.cpu().numpy()
    prod = np.array([[[int(x) * int(y) % q for x, y in zip(fa[0, i], fb[0, i])] for i, q in enumerate(prm.q)]],
                    dtype=np.int64)
    dp = torch.from_numpy(prod).cuda()
    P.ctx.ntt(dp, inverse=True)
    got = dp.cpu().numpy()[0]
    for i, q in enumerate(prm.q):
        assert np.array_equal(got[i], np.array([x % q for x in negacyclic(a[i], b[i])], dtype=np.int64))
    P.ctx.ntt(da, inverse=True)
    assert np.array_equal(da.cpu().numpy()[0], np.array(a, dtype=np.int64))


@pytest.mark.parametrize("name,cfg", [("C1", C1), ("SMALL", SMALL), ("WIDE", WIDE), ("BIG_T", BIG_T)])
def test_encrypt_decrypt(name, cfg):
    P = pair(name, cfg)
    prm = P.prm
    y = inputs.slots(11, 3, prm.N, hi=prm.t)
    ct = P.ctx.encrypt(torch.from_numpy(y).cuda(), seed=21)
    want = [P.enc(y[i], 21, i) for i in range(3)]
    assert_ct_equal(prm, ct, want, "encrypt")
    # decrypt of the oracle's ciphertexts, and of the GPU's own
    dec = P.ctx.decrypt(cts_to_device(prm, want)).cpu().numpy()
    assert np.array_equal(dec, y)
    assert np.array_equal(P.ctx.decrypt(ct).cpu().numpy(), y)


def test_linear_ops():
    P = pair("C1", C1)
    prm, ctx = P.prm, P.ctx
    t = prm.t
    y = inputs.slots(12, 3, prm.N, hi=t)
    a = [P.enc(y[0], 31, 0)]
    b = [P.enc(y[1], 31, 1)]
    da, db = cts_to_device(prm, a), cts_to_device(prm, b)
    assert_ct_equal(prm, ctx.add(da, db), [bfv.add(prm, a[0], b[0])], "add")
    assert_ct_equal(prm, ctx.sub(da, db), [bfv.sub(prm, a[0], b[0])], "sub")
    assert_ct_equal(prm, ctx.add_const(da, 7), [bfv.add_const(prm, a[0], 7)], "add_const")
    assert_ct_equal(prm, ctx.sub_const(da, t - 1), [bfv.sub_const(prm, a[0], t - 1)], "sub_const")
    assert_ct_equal(prm, ctx.const_sub(1, da), [bfv.const_sub(prm, 1, a[0])], "const_sub")
    assert_ct_equal(prm, ctx.mul_scalar(da, 65536), [bfv.mul_scalar(prm, a[0], 65536)], "mul_scalar")
    w = y[2]
    got = ctx.mul_plain(da, torch.from_numpy(w[None]).cuda())
    assert_ct_equal(prm, got, [bfv.mul_plain(prm, a[0], [int(v) for v in w])], "mul_plain")
    # in-place add (out aliases a)
    ctx.add(da, db, out=da)
    assert_ct_equal(prm, da, [bfv.add(prm, a[0], b[0])], "add in place")


@pytest.mark.parametrize("name,cfg,n", [("C1", C1, 3), ("SMALL", SMALL, 2), ("ALPHA2", ALPHA2, 2),
                                        ("WIDE", WIDE, 1), ("LOW_T", LOW_T, 2), ("MID", MID, 1),
                                        ("L16", L16, 2), ("BIG_Q", BIG_Q, 2), ("BIG_T", BIG_T, 2)])
def test_mul_relin(name, cfg, n):
    P = pair(name, cfg)
    prm = P.prm
    y = inputs.slots(13, 2 * n, prm.N, hi=prm.t)
    a = [P.enc(y[i], 41, i) for i in range(n)]
    b = [P.enc(y[n + i], 41, n + i) for i in range(n)]
    got = P.ctx.mul_relin(cts_to_device(prm, a), cts_to_device(prm, b))
    want = [bfv.mul_relin(prm, P.keys, a[i], b[i]) for i in range(n)]
    assert_ct_equal(prm, got, want, "mul_relin")
    dec = P.ctx.decrypt(got).cpu().numpy()
    want_slots = (y[:n].astype(object) * y[n:].astype(object)) % prm.t   # exact for t up to 2^32
    assert np.array_equal(dec, want_slots.astype(np.int64))


def test_large_t_plain_and_scalar():
    """Slot encoding of a public vector (an NTT over t) and the largest scalar at t just below 2^32."""
    P = pair("BIG_T", BIG_T)
    prm, ctx = P.prm, P.ctx
    t = prm.t
    y = inputs.slots(19, 2, prm.N, lo=t - 1000, hi=t)
    a = [P.enc(y[0], 33, 0)]
    da = cts_to_device(prm, a)
    w = y[1]
    got = ctx.mul_plain(da, torch.from_numpy(w[None]).cuda())
    assert_ct_equal(prm, got, [bfv.mul_plain(prm, a[0], [int(v) for v in w])], "mul_plain")
    want = np.array([int(u) * int(v) % t for u, v in zip(y[0], w)], dtype=np.int64)   # exact: no int64 product
    assert np.array_equal(ctx.decrypt(got).cpu().numpy()[0], want)
    assert_ct_equal(prm, ctx.mul_scalar(da, t - 1), [bfv.mul_scalar(prm, a[0], t - 1)], "mul_scalar")
    assert_ct_equal(prm, ctx.add_const(da, t - 1), [bfv.add_const(prm, a[0], t - 1)], "add_const")


def test_mul_relin_edge_values():
    """Coefficients at the centring boundary (Q-1)/2, (Q+1)/2, 0 and Q-1 and a zero ciphertext."""
    P = pair("SMALL", SMALL)
    prm = P.prm
    Q = prm.Q
    a = P.enc(inputs.slots(14, 1, prm.N, hi=prm.t)[0], 51, 0)
    b = P.enc(inputs.slots(15, 1, prm.N, hi=prm.t)[0], 51, 1)
    special = [(Q - 1) // 2, (Q + 1) // 2, 0, Q - 1, 1]
    a = ([special[k % 5] if k < 10 else x for k, x in enumerate(a[0])], a[1])
    b = (b[0], [special[(k + 2) % 5] if k < 10 else x for k, x in enumerate(b[1])])
    zero = ([0] * prm.N, [0] * prm.N)
    got = P.ctx.mul_relin(cts_to_device(prm, [a, zero]), cts_to_device(prm, [b, b]))
    assert_ct_equal(prm, got, [bfv.mul_relin(prm, P.keys, a, b), zero], "mul_relin edges")


def test_gates_and_counts():
    P = pair("SMALL", SMALL)
    prm, ctx = P.prm, P.ctx
    rng = np.random.default_rng(3)
    bits = rng.integers(0, 2, size=(3, prm.N))
    cts = [P.enc(bits[i], 61, i) for i in range(3)]
    x, y, z = (cts_to_device(prm, [c]) for c in cts)
    for g in range(8):
        ev = bridge.Evaluator(prm, P.keys)
        want = ev.gate(g, *cts)
        ctx.op_counts(reset=True)
        got = ctx.bit_gate(g, x, y, z)
        assert_ct_equal(prm, got, [want], "gate %s" % bridge.GATE_NAMES[g])
        assert ctx.op_counts()[:3] == ev.counts(), bridge.GATE_NAMES[g]


@pytest.mark.parametrize("s", [1, 3, 8])
def test_bits_to_mod(s):
    P = pair("C1", C1)
    prm = P.prm
    vals = inputs.slots(16, 1, prm.N, hi=1 << s)[0]
    planes = inputs.bit_planes(vals, s)
    bits = [P.enc(planes[k], 71, k) for k in range(s)]
    dev = torch.from_numpy(np.stack([ct_to_rns(prm, c)[None] for c in bits])).cuda()   # [s][1][2][L][N]
    ev = bridge.Evaluator(prm, P.keys)
    want = ev.bits_to_mod(bits)
    P.ctx.op_counts(reset=True)
    got = P.ctx.bits_to_mod(dev)
    assert_ct_equal(prm, got, [want], "bits_to_mod")
    assert P.ctx.op_counts()[:3] == ev.counts()
    assert np.array_equal(P.ctx.decrypt(got).cpu().numpy()[0], vals)


@pytest.mark.parametrize("e", [2, 3, 12288])
def test_pow(e):
    P = pair("LOW_T", LOW_T)
    prm = P.prm
    x = P.enc(inputs.slots(17, 1, prm.N, hi=prm.t)[0], 81, 0)
    ev = bridge.Evaluator(prm, P.keys)
    want = ev.pow(x, e)
    P.ctx.op_counts(reset=True)
    got = P.ctx.pow(cts_to_device(prm, [x]), e)
    assert_ct_equal(prm, got, [want], "pow %d" % e)
    assert P.ctx.op_counts()[2] == ev.n_mul == bridge.pow_mul_count(e)


@pytest.mark.parametrize("mode", [bridge.PAPER, bridge.SELECT])
def test_mod_to_bits(mode):
    P = pair("LOW_T", LOW_T)
    prm = P.prm
    s, cands = 2, range(0, 4)
    xs = inputs.slots(18, 1, prm.N, hi=4)[0]
    x = P.enc(xs, 91, 0)
    ev = bridge.Evaluator(prm, P.keys)
    want = ev.mod_to_bits(x, s, cands, mode)
    P.ctx.op_counts(reset=True)
    got = P.ctx.mod_to_bits(cts_to_device(prm, [x]), s, cands[0], cands[-1], mode)
    for k in range(s):
        assert_ct_equal(prm, got[k], [want[k]], "mod_to_bits bit %d" % k)
    assert P.ctx.op_counts()[:3] == ev.counts()


def test_gate_level_matches_gates():
    """One level with every gate type (multiplying gates first, NOT last) on a shared wire array."""
    P = pair("SMALL", SMALL)
    prm, ctx = P.prm, P.ctx
    rng = np.random.default_rng(4)
    bits = rng.integers(0, 2, size=(3, prm.N))
    cts = [P.enc(bits[i], 101, i) for i in range(3)]
    gates = [0, 1, 2, 3, 4, 5, 7, 6]                       # NOT (6) last
    n_w = 3 + len(gates)
    wires = torch.zeros(n_w, 1, 2, prm.L, prm.N, dtype=torch.int64, device="cuda")
    wires[:3] = cts_to_device(prm, cts)[:, None]
    table = torch.tensor([[g, 0, 1, 2, 3 + i] for i, g in enumerate(gates)], dtype=torch.int32, device="cuda")
    ctx.gate_level(wires, table, len(gates), len(gates) - 1)
    for i, g in enumerate(gates):
        want = bridge.Evaluator(prm, P.keys).gate(g, *cts)
        assert_ct_equal(prm, wires[3 + i], [want], "level gate %s" % bridge.GATE_NAMES[g])


@pytest.mark.parametrize("name,cfg", [("C1", C1), ("ALPHA2", ALPHA2), ("L16", L16), ("BIG_Q", BIG_Q)])
def test_square_path(name, cfg):
    """mul_relin(x, x) through the squaring path equals the oracle's x * x."""
    P = pair(name, cfg)
    prm = P.prm
    y = inputs.slots(19, 2, prm.N, hi=prm.t)
    xs = [P.enc(y[i], 111, i) for i in range(2)]
    d = cts_to_device(prm, xs)
    got = P.ctx.mul_relin(d, d)
    assert_ct_equal(prm, got, [bfv.mul_relin(prm, P.keys, x, x) for x in xs], "square")


def test_mul_relin_at_benchmark_parameters():
    """N = 16384, L = 8, alpha = 1 (the bench's ring): keys, one mul_relin and one squaring, bit for bit.
    The oracle takes about a minute here."""
    P = pair("C4", C4)
    prm = P.prm
    sk, pk, _ = P.ctx.export_keys()
    assert sk.cpu().numpy().tolist() == P.keys.s
    assert np.array_equal(pk.cpu().numpy(), ct_to_rns(prm, (P.keys.pk0, P.keys.pk1)))
    y = inputs.slots(20, 2, prm.N, hi=prm.t)
    ct = P.ctx.encrypt(torch.from_numpy(y).cuda(), seed=121)
    a, b = P.enc(y[0], 121, 0), P.enc(y[1], 121, 1)
    assert_ct_equal(prm, ct, [a, b], "encrypt C4")
    got = P.ctx.mul_relin(ct[0:1].contiguous(), ct[1:2].contiguous())
    assert_ct_equal(prm, got, [bfv.mul_relin(prm, P.keys, a, b)], "mul_relin C4")
    sq = P.ctx.mul_relin(got, got)
    p = (y[0] * y[1]) % prm.t
    assert np.array_equal(P.ctx.decrypt(sq).cpu().numpy()[0], (p * p) % prm.t)


# ------------------------------------------------------------ signed conversions (Listings 6 and 9)
@pytest.mark.parametrize("name,cfg,s", [("LOW_T", LOW_T, 1), ("LOW_T", LOW_T, 13), ("C1", C1, 8), ("C1", C1, 16)])
def test_sint_to_mod(name, cfg, s):
    """Two's complement bit planes of signed slots -> SecureMod, against the oracle bit for bit;
    the result decrypts to v mod t (depth 1)."""
    P = pair(name, cfg)
    prm = P.prm
    v = inputs.slots(20 + s, 1, prm.N, lo=-(1 << (s - 1)), hi=1 << (s - 1))[0]
    v[:2] = [-(1 << (s - 1)), (1 << (s - 1)) - 1]          # both ends of the range
    planes = inputs.bit_planes(v % (1 << s), s)
    bits = [P.enc(planes[k], 121, k) for k in range(s)]
    dev = cts_to_device(prm, bits)[:, None]                  # [s][1][2][L][N]
    ev = bridge.Evaluator(prm, P.keys)
    want = ev.sint_to_mod(bits)
    P.ctx.op_counts(reset=True)
    got = P.ctx.sint_to_mod(dev)
    assert_ct_equal(prm, got, [want], "sint_to_mod s=%d" % s)
    assert P.ctx.op_counts()[:3] == ev.counts()
    assert np.array_equal(P.ctx.decrypt(got).cpu().numpy()[0], v % prm.t)


@pytest.mark.parametrize("sign,mode", [(+1, bridge.PAPER), (-1, bridge.SELECT)])
def test_mod_to_sint(sign, mode):
    """Listing 9 at t = 12289, s = 14 (2^s >= t): slots all non-negative (x in [0, 2)) or all
    negative (x in [t-4, t)); candidate ranges are the values x and (2^s - t) + x take."""
    P = pair("LOW_T", LOW_T)
    prm = P.prm
    t, s = prm.t, 14
    lo, hi = (0, 1) if sign > 0 else (t - 4, t - 1)
    xs = inputs.slots(30 + sign, 1, prm.N, lo=lo, hi=hi + 1)[0]
    x = P.enc(xs, 131, 0)
    shift = ((1 << s) - t) % t
    pos_r = (lo, hi)
    neg_r = ((lo + shift) % t, (hi + shift) % t)
    assert neg_r[0] <= neg_r[1]
    ev = bridge.Evaluator(prm, P.keys)
    want = ev.mod_to_sint(x, s, range(pos_r[0], pos_r[1] + 1), range(neg_r[0], neg_r[1] + 1), mode)
    P.ctx.op_counts(reset=True)
    got = P.ctx.mod_to_sint(cts_to_device(prm, [x]), s, pos_r, neg_r, mode)
    for k in range(s):
        assert_ct_equal(prm, got[k], [want[k]], "mod_to_sint bit %d" % k)
    assert P.ctx.op_counts()[:3] == ev.counts()


# ------------------------------------------------------------ guarded fast base extension
@pytest.mark.parametrize("name,cfg", [("C1", C1), ("SMALL", SMALL), ("ALPHA2", ALPHA2), ("L16", L16), ("MID", MID)])
def test_fast_extension_gives_the_same_ciphertexts(name, cfg):
    """With the guarded fast extension on, multiplies (general and squaring) equal the oracle word for
    word, including coefficients at the centring boundary, where the guard sends the extension
    to the exact mixed-radix path."""
    P = pair(name, cfg)
    prm = P.prm
    Q = prm.Q
    y = inputs.slots(61, 4, prm.N, hi=prm.t)
    a = P.enc(y[0], 71, 0)
    b = P.enc(y[1], 71, 1)
    special = [(Q - 1) // 2, (Q + 1) // 2, 0, Q - 1, 1]
    e = ([special[k % 5] if k < 10 else x for k, x in enumerate(a[0])], a[1])
    want = [bfv.mul_relin(prm, P.keys, a, b), bfv.mul_relin(prm, P.keys, e, b), bfv.mul_relin(prm, P.keys, a, a)]
    default = P.ctx.fast_extension
    assert default == (prm.L >= 8)
    try:
        for fast in (False, True):
            P.ctx.set_fast_extension(fast)
            got = P.ctx.mul_relin(cts_to_device(prm, [a, e]), cts_to_device(prm, [b, b]))
            da = cts_to_device(prm, [a])
            sq = P.ctx.mul_relin(da, da)
            assert_ct_equal(prm, got, want[:2], "extension (fast=%s) %s" % (fast, name))
            assert_ct_equal(prm, sq, want[2:], "extension (fast=%s) square %s" % (fast, name))
    finally:
        P.ctx.set_fast_extension(default)


def test_fast_extension_needs_small_moduli():
    from paper_2204_12201_gb300 import bfhe
    P = pair("BIG_Q", BIG_Q)
    assert not P.ctx.fast_extension
    with pytest.raises(bfhe.BfheError):
        P.ctx.set_fast_extension(True)


def test_mod_to_sint_at_t65537():
    """Listing 9 at the workloads' t = 65537 with s = 17 (the least s with 2^s >= t), select mode,
    two candidates per conversion: x in {t-2, t-1} (negative) and its shifted range."""
    P = pair("C1", C1)
    prm = P.prm
    t, s = prm.t, 17
    xs = inputs.slots(33, 1, prm.N, lo=t - 2, hi=t)[0]
    x = P.enc(xs, 141, 0)
    shift = ((1 << s) - t) % t
    pos_r = (t - 2, t - 1)
    neg_r = ((t - 2 + shift) % t, (t - 1 + shift) % t)
    assert neg_r[0] <= neg_r[1]
    ev = bridge.Evaluator(prm, P.keys)
    want = ev.mod_to_sint(x, s, range(pos_r[0], pos_r[1] + 1), range(neg_r[0], neg_r[1] + 1), bridge.SELECT)
    P.ctx.op_counts(reset=True)
    got = P.ctx.mod_to_sint(cts_to_device(prm, [x]), s, pos_r, neg_r, bridge.SELECT)
    for k in range(s):
        assert_ct_equal(prm, got[k], [want[k]], "mod_to_sint bit %d" % k)
    assert P.ctx.op_counts()[:3] == ev.counts()
