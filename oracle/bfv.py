"""Textbook FV/BFV over Z_Q, written out plainly (test infrastructure only).

The paper runs every secure type on BFV through SEAL and describes none of its
internals (Sec. 4.1); the scheme is Fan-Vercauteren's.  Every choice that fixes
ciphertext bits is stated here so that the CUDA library can reproduce it:

* ring R = Z[X]/(X^N + 1); ciphertexts are pairs of polynomials with
  coefficients in [0, Q); keys and randomness come from `philox`;
* slots (FHE batching, Sec. 2.3): slot j holds m(zeta^(2j+1)) mod t; with
  t = 2 there are no slots and encrypt_poly / decrypt_poly carry the
  plaintext polynomial's coefficients directly;
* pk = ([-(a s + e)]_Q, a); relinearisation key for digit j = 0..L-1:
  rlk_j = ([-(a_j s + e_j) + P g_j s^2]_{PQ}, a_j) with the RNS gadget
  g_j = (Q/q_j) * [(Q/q_j)^-1]_{q_j};
* encrypt: (Delta m + pk0 u + e1, pk1 u + e2) mod Q, Delta = floor(Q/t);
* decrypt: m = [round(t [c0 + c1 s]_Q / Q)]_t;
* multiply: lift every input coefficient to the centred range (-Q/2, Q/2],
  form the exact tensor d0 = a0 b0, d1 = a0 b1 + a1 b0, d2 = a1 b1 over Z and
  return [round(t d_k / Q)]_Q (ties are impossible: Q odd, gcd(Q, t) = 1);
* relinearise: unsigned digits delta_j = [c2]_{q_j}, w = sum_j delta_j rlk_j
  mod PQ, out = (c0, c1) + round(w / P) mod Q where round(w / P) = (w - r)/P
  with r the centred residue of w mod P.
"""

import math

import numpy as np

from . import philox as px
from .nt import centered, crt, inv
from .poly import add_poly, negacyclic, sub_poly


# ---------------------------------------------------------------- batching
def _zeta_table(prm):
    t, N = prm.t, prm.N
    tab = np.empty(2 * N, dtype=np.int64)
    z = 1
    for e in range(2 * N):
        tab[e] = z
        z = z * prm.zeta % t
    return tab


def _mulmod(a, b, t):
    """a * b mod t elementwise, exact in int64 for values in [0, t) and t < 2^32: b is split into
    16-bit halves, so no intermediate reaches 2^48."""
    lo = (a * (b & 0xFFFF)) % t
    hi = (a * (b >> 16)) % t
    return (lo + ((hi << 16) % t)) % t


def decode_poly(prm, m):
    """Slots of a plaintext polynomial: y_j = m(zeta^(2j+1)) mod t (plain evaluation).
    Every product is reduced mod t before the sum over k (N terms below t < 2^32 sum below 2^47)."""
    N, t = prm.N, prm.t
    tab = _zeta_table(prm)
    mv = np.array([x % t for x in m], dtype=np.int64)
    k = np.arange(N, dtype=np.int64)
    out = np.empty(N, dtype=np.int64)
    chunk = max(1, (1 << 22) // N)
    for j0 in range(0, N, chunk):
        j = np.arange(j0, min(N, j0 + chunk), dtype=np.int64)
        e = ((2 * j[:, None] + 1) * k[None, :]) % (2 * N)
        out[j0:j0 + len(j)] = _mulmod(tab[e], mv[None, :], t).sum(axis=1) % t
    return [int(x) for x in out]


def encode_slots(prm, y):
    """Inverse of decode: m_k = N^-1 sum_j y_j zeta^(-(2j+1)k) mod t, coefficients in [0, t)."""
    N, t = prm.N, prm.t
    tab = _zeta_table(prm)
    yv = np.array([v % t for v in y], dtype=np.int64)
    j = np.arange(N, dtype=np.int64)
    out = np.empty(N, dtype=np.int64)
    chunk = max(1, (1 << 22) // N)
    for k0 in range(0, N, chunk):
        k = np.arange(k0, min(N, k0 + chunk), dtype=np.int64)
        e = (-(2 * j[None, :] + 1) * k[:, None]) % (2 * N)
        out[k0:k0 + len(k)] = _mulmod(tab[e], yv[None, :], t).sum(axis=1) % t
    ninv = inv(N, t)
    return [int(x) * ninv % t for x in out]


# ---------------------------------------------------------------- keys
class Keys:
    def __init__(self, s, pk0, pk1, rlk):
        self.s = s          # ternary, list of N ints in {-1, 0, 1}
        self.pk0 = pk0      # mod Q
        self.pk1 = pk1      # mod Q
        self.rlk = rlk      # list of L pairs (b_j, a_j), each mod PQ


def uniform_mod(prm, seed, purpose, poly, primes):
    """A polynomial uniform mod prod(primes), drawn limb by limb and joined by CRT."""
    limbs = [px.uniform_poly(seed, purpose, poly, i, q, prm.N) for i, q in enumerate(primes)]
    return [crt([limbs[i][n] for i in range(len(primes))], primes) for n in range(prm.N)]


def keygen(prm, seed):
    N, Q, P = prm.N, prm.Q, prm.P
    s = px.ternary_poly(seed, px.SK, 0, N)
    a = uniform_mod(prm, seed, px.PK_A, 0, prm.q)
    e = px.cbd_poly(seed, px.PK_E, 0, N)
    as_ = negacyclic(a, s)
    pk0 = [(-(x + y)) % Q for x, y in zip(as_, e)]
    s2 = negacyclic(s, s)
    PQ = P * Q
    pq_primes = prm.q + prm.p
    rlk = []
    for j, qj in enumerate(prm.q):
        aj = uniform_mod(prm, seed, px.RLK_A, j, pq_primes)
        ej = px.cbd_poly(seed, px.RLK_E, j, N)
        Qj = Q // qj
        gj = Qj * inv(Qj, qj)
        ajs = negacyclic(aj, s)
        bj = [(-(x + y) + P * gj * z) % PQ for x, y, z in zip(ajs, ej, s2)]
        rlk.append((bj, aj))
    return Keys(s, pk0, a, rlk)


# ---------------------------------------------------------------- encrypt / decrypt
def encrypt(prm, keys, slots, seed, idx=0):
    """Public-key encryption of one slot vector; idx selects the randomness stream."""
    if not prm.batching:
        raise ValueError("no batching at t = %d" % prm.t)
    return encrypt_poly(prm, keys, encode_slots(prm, slots), seed, idx)


def encrypt_poly(prm, keys, m, seed, idx=0):
    """Public-key encryption of the plaintext polynomial m (coefficients in [0, t))."""
    N, Q = prm.N, prm.Q
    u = px.ternary_poly(seed, px.ENC_U, idx, N)
    e1 = px.cbd_poly(seed, px.ENC_E1, idx, N)
    e2 = px.cbd_poly(seed, px.ENC_E2, idx, N)
    pu0 = negacyclic(keys.pk0, u)
    pu1 = negacyclic(keys.pk1, u)
    c0 = [(prm.delta * mk + x + e) % Q for mk, x, e in zip(m, pu0, e1)]
    c1 = [(x + e) % Q for x, e in zip(pu1, e2)]
    return (c0, c1)


def phase(prm, keys, ct):
    """[c0 + c1 s (+ c2 s^2)]_Q in [0, Q)."""
    Q = prm.Q
    v = [x + y for x, y in zip(ct[0], negacyclic(ct[1], keys.s))]
    if len(ct) == 3:
        s2 = negacyclic(keys.s, keys.s)
        v = [x + y for x, y in zip(v, negacyclic(ct[2], s2))]
    return [x % Q for x in v]


def round_div(x, d):
    """round(x / d) for an odd positive d and any integer x (ties cannot occur)."""
    return (2 * x + d) // (2 * d)


def decrypt_poly(prm, keys, ct):
    v = phase(prm, keys, ct)
    return [round_div(prm.t * x, prm.Q) % prm.t for x in v]


def decrypt(prm, keys, ct):
    if not prm.batching:
        raise ValueError("no batching at t = %d" % prm.t)
    return decode_poly(prm, decrypt_poly(prm, keys, ct))


def noise_budget(prm, keys, ct):
    """log2(Q/2) - log2 max|[t v]_Q| (centred); decryption is correct while it is > 0."""
    v = phase(prm, keys, ct)
    worst = max(abs(centered(prm.t * x, prm.Q)) for x in v)
    if worst == 0:
        return float(prm.Q.bit_length())
    return math.log2(prm.Q / 2) - math.log2(worst)


# ---------------------------------------------------------------- linear ops
def trivial(prm, c):
    """Trivial encryption (Delta [c]_t, 0) of the constant polynomial c."""
    c0 = [0] * prm.N
    c0[0] = prm.delta * (c % prm.t) % prm.Q
    return (c0, [0] * prm.N)


def add(prm, a, b):
    return (add_poly(a[0], b[0], prm.Q), add_poly(a[1], b[1], prm.Q))


def sub(prm, a, b):
    return (sub_poly(a[0], b[0], prm.Q), sub_poly(a[1], b[1], prm.Q))


def negate(prm, a):
    return ([(-x) % prm.Q for x in a[0]], [(-x) % prm.Q for x in a[1]])


def add_const(prm, a, c):
    """a + c for a public constant c: adds Delta [c]_t to coefficient 0 of c0."""
    return add(prm, a, trivial(prm, c))


def sub_const(prm, a, c):
    """a - c (= a - trivial(c))."""
    return sub(prm, a, trivial(prm, c))


def const_sub(prm, c, a):
    """c - a (= trivial(c) - a)."""
    return sub(prm, trivial(prm, c), a)


def mul_scalar(prm, a, c):
    """Multiply both components by the integer c in [0, t)."""
    c %= prm.t
    return ([x * c % prm.Q for x in a[0]], [x * c % prm.Q for x in a[1]])


def mul_plain(prm, a, slots):
    """Slot-wise product with a public vector: pt = encode(slots) in [0, t)^N."""
    pt = encode_slots(prm, slots)
    Q = prm.Q
    return ([x % Q for x in negacyclic(a[0], pt)], [x % Q for x in negacyclic(a[1], pt)])


# ---------------------------------------------------------------- multiply
def tensor(prm, a, b):
    """Exact tensor of centred lifts over Z: (a0 b0, a0 b1 + a1 b0, a1 b1)."""
    Q = prm.Q
    a0, a1 = [centered(x, Q) for x in a[0]], [centered(x, Q) for x in a[1]]
    b0, b1 = [centered(x, Q) for x in b[0]], [centered(x, Q) for x in b[1]]
    d0 = negacyclic(a0, b0)
    d1 = [x + y for x, y in zip(negacyclic(a0, b1), negacyclic(a1, b0))]
    d2 = negacyclic(a1, b1)
    return d0, d1, d2


def scale_round(prm, d):
    """[round(t d / Q)]_Q coefficient-wise."""
    return [round_div(prm.t * x, prm.Q) % prm.Q for x in d]


def mul(prm, a, b):
    """Ciphertext product without relinearisation: a 3-component ciphertext."""
    d0, d1, d2 = tensor(prm, a, b)
    return (scale_round(prm, d0), scale_round(prm, d1), scale_round(prm, d2))


def mod_down(prm, w):
    """round(w / P) mod Q for w in [0, PQ): (w - [w]_P centred) / P."""
    P, Q = prm.P, prm.Q
    return [((x - centered(x, P)) // P) % Q for x in w]


def key_switch_parts(prm, keys, c2):
    """w = sum_j [c2]_{q_j} * rlk_j mod PQ, for both key components."""
    PQ = prm.P * prm.Q
    w0 = [0] * prm.N
    w1 = [0] * prm.N
    for j, qj in enumerate(prm.q):
        dj = [x % qj for x in c2]
        bj, aj = keys.rlk[j]
        w0 = [x + y for x, y in zip(w0, negacyclic(dj, bj))]
        w1 = [x + y for x, y in zip(w1, negacyclic(dj, aj))]
    return [x % PQ for x in w0], [x % PQ for x in w1]


def relin(prm, keys, ct3):
    c0, c1, c2 = ct3
    w0, w1 = key_switch_parts(prm, keys, c2)
    Q = prm.Q
    return (add_poly(c0, mod_down(prm, w0), Q), add_poly(c1, mod_down(prm, w1), Q))


def mul_relin(prm, keys, a, b):
    return relin(prm, keys, mul(prm, a, b))


# ---------------------------------------------------------------- RNS view
def to_rns(poly, primes):
    """[len(primes)][N] residues of a polynomial (the layout the GPU library stores)."""
    return [[x % q for x in poly] for q in primes]


def from_rns(limbs, primes):
    N = len(limbs[0])
    return [crt([limbs[i][n] for i in range(len(primes))], primes) for n in range(N)]
