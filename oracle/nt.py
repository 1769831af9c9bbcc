"""Elementary number theory for the oracle (test infrastructure only).

Deterministic Miller-Rabin with the first twelve prime bases is exact for
every n < 3.18e23, which covers every 64-bit candidate modulus.
"""

MR_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)


def is_prime(n):
    """Deterministic Miller-Rabin primality test for n < 3.18e23."""
    if n < 2:
        return False
    for p in MR_BASES:
        if n % p == 0:
            return n == p
    d, r = n - 1, 0
    while d % 2 == 0:
        d //= 2
        r += 1
    for a in MR_BASES:
        x = pow(a, d, n)
        if x == 1 or x == n - 1:
            continue
        for _ in range(r - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def inv(a, m):
    """Inverse of a modulo m (raises ValueError if gcd(a, m) != 1)."""
    return pow(a % m, -1, m)


def factor_small(n):
    """Distinct prime factors of n by trial division (n up to ~2^40)."""
    fs = []
    d = 2
    while d * d <= n:
        if n % d == 0:
            fs.append(d)
            while n % d == 0:
                n //= d
        d += 1 if d == 2 else 2
    if n > 1:
        fs.append(n)
    return fs


def least_primitive_root(p):
    """Smallest generator of the multiplicative group of the prime field Z_p."""
    fs = factor_small(p - 1)
    g = 2
    while True:
        if all(pow(g, (p - 1) // f, p) != 1 for f in fs):
            return g
        g += 1


def crt(residues, moduli):
    """The unique x in [0, prod(moduli)) with x = r_i mod m_i (pairwise coprime)."""
    M = 1
    for m in moduli:
        M *= m
    x = 0
    for r, m in zip(residues, moduli):
        Mi = M // m
        x += r * Mi * inv(Mi, m)
    return x % M


def centered(x, M):
    """Representative of x mod M in (-M/2, M/2] (M odd here, so [-(M-1)/2, (M-1)/2])."""
    x %= M
    return x - M if x > (M - 1) // 2 else x


def prod(xs):
    r = 1
    for x in xs:
        r *= x
    return r
