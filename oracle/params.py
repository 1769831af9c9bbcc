"""Parameter rule shared (by specification, not by code) with the CUDA library.

The paper fixes only n = 2^15, t = 2^16 + 1 and 128-bit security and lets SEAL
pick the rest (Sec. 4.1).  This build fixes the remaining choices as follows:

* every modulus is a prime q = 1 (mod 2N) below 2^prime_bits, taken from ONE
  downward scan over q = 2N*k + 1 (k decreasing), skipping t;
* the first L primes of the scan are the data primes q_0 > ... > q_{L-1}
  (Q = prod q_i), the next alpha are the special primes p_0 > ... (P), the
  next K are the auxiliary primes b_0 > ... (B) of the exact multiply;
* K is the smallest count with B > 2 t N Q, which makes the exact tensor
  (|d| <= N Q^2 / 2) and the rounded quotient round(t d / Q) representable
  in the centred range of the moduli QB and B respectively;
* Delta = floor(Q / t); the slot root is zeta = g^((t-1)/2N) mod t with g the
  least primitive root of t;
* t < 2^32, the plaintext moduli the library accepts;
* t = 2 (Sec. 4.1 and 4.3 run the bit-level benchmarks with t = 2 as well):
  no batching (2 is not 1 mod 2N), so plaintexts are polynomials with
  coefficients mod 2 and there is no slot root.
"""

from dataclasses import dataclass, field

from .nt import is_prime, least_primitive_root, prod


def scan_primes(N, count, prime_bits, exclude=()):
    """First `count` primes q = 1 mod 2N below 2^prime_bits, in decreasing order."""
    step = 2 * N
    k = ((1 << prime_bits) - 2) // step
    out = []
    while len(out) < count:
        if k <= 0:
            raise ValueError("not enough NTT-friendly primes below 2^%d" % prime_bits)
        q = step * k + 1
        if q not in exclude and is_prime(q):
            out.append(q)
        k -= 1
    return out


@dataclass
class Params:
    N: int
    L: int
    alpha: int
    t: int = 65537
    prime_bits: int = 50
    q: list = field(default_factory=list)      # data primes
    p: list = field(default_factory=list)      # special primes
    b: list = field(default_factory=list)      # auxiliary primes
    Q: int = 0
    P: int = 0
    B: int = 0
    K: int = 0
    delta: int = 0
    zeta: int = 0
    batching: bool = True

    def __post_init__(self):
        N, t = self.N, self.t
        if N & (N - 1) or N < 2:
            raise ValueError("N must be a power of two")
        self.batching = t != 2
        if self.batching and (not is_prime(t) or (t - 1) % (2 * N)):
            raise ValueError("batching needs a prime t = 1 mod 2N (or t = 2 without batching)")
        if t >= 1 << 32:
            raise ValueError("t must be below 2^32 (the slot transforms reduce products of two values below t)")
        head = scan_primes(N, self.L + self.alpha, self.prime_bits, exclude=(t,))
        self.q = head[: self.L]
        self.p = head[self.L:]
        self.Q = prod(self.q)
        self.P = prod(self.p)
        # auxiliary base: keep drawing from the same scan until B > 2 t N Q
        K = 1
        while True:
            allp = scan_primes(N, self.L + self.alpha + K, self.prime_bits, exclude=(t,))
            B = prod(allp[self.L + self.alpha:])
            if B > 2 * t * N * self.Q:
                break
            K += 1
        self.b = allp[self.L + self.alpha:]
        self.B = B
        self.K = K
        self.delta = self.Q // t
        if self.batching:
            g = least_primitive_root(t)
            self.zeta = pow(g, (t - 1) // (2 * N), t)

    @property
    def PQ(self):
        return self.P * self.Q


# Parameter sets of the synthetic workloads (ring degree, data primes, special
# primes); all use t = 65537 and 50-bit primes.
C1 = dict(N=4096, L=2, alpha=1)     # SecureMod pairs + 8-bit ripple adder
C2 = dict(N=8192, L=4, alpha=1)     # 16-bit comparator and 16x16 multiplier
C3 = dict(N=32768, L=16, alpha=2)   # mod_to_bits, c in 0..255
C4 = dict(N=16384, L=8, alpha=1)    # genotype-shaped dot products + bridge
