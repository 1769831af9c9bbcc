"""Exact products in Z[X]/(X^N + 1) (test infrastructure only).

BFV multiplies polynomials in the ring R = Z[X]/(X^N + 1) (Fan-Vercauteren,
the scheme the paper runs on through SEAL).  The oracle forms the exact
integer product: the linear convolution c = a * b over Z is read off one big
integer product A(2^w) * B(2^w) (Kronecker substitution, a library multiply
as a single step), and X^N = -1 folds it: r_k = c_k - c_{k+N}.
"""


def _width(a, b):
    ma = max((abs(x) for x in a), default=0)
    mb = max((abs(x) for x in b), default=0)
    bound = max(len(a), len(b)) * ma * mb + 1   # |c_k| <= n * max|a| * max|b|
    bound = max(bound, ma, mb)            # the packed inputs must fit too
    w = bound.bit_length() + 2            # room for the sign offset
    return (w + 7) // 8                   # bytes per slot


def _pack(v, wb):
    pos = b"".join((x if x > 0 else 0).to_bytes(wb, "little") for x in v)
    neg = b"".join((-x if x < 0 else 0).to_bytes(wb, "little") for x in v)
    return int.from_bytes(pos, "little") - int.from_bytes(neg, "little")


def linear_product(a, b):
    """Full linear convolution of two integer sequences (length len(a)+len(b)-1)."""
    if not a or not b:
        return []
    wb = _width(a, b)
    C = _pack(a, wb) * _pack(b, wb)
    n = len(a) + len(b) - 1
    half = 1 << (8 * wb - 1)
    off = int.from_bytes(half.to_bytes(wb, "little") * n, "little")
    raw = (C + off).to_bytes(wb * n, "little")
    return [int.from_bytes(raw[i * wb:(i + 1) * wb], "little") - half for i in range(n)]


def negacyclic(a, b):
    """a * b in Z[X]/(X^N + 1), exact over the integers."""
    N = len(a)
    assert len(b) == N
    c = linear_product(a, b)
    c += [0] * (2 * N - len(c))
    return [c[k] - c[k + N] for k in range(N)]


def negacyclic_schoolbook(a, b):
    """Same product by the O(N^2) definition; used only to pin `negacyclic`."""
    N = len(a)
    r = [0] * N
    for i in range(N):
        for j in range(N):
            k = i + j
            if k < N:
                r[k] += a[i] * b[j]
            else:
                r[k - N] -= a[i] * b[j]
    return r


def mod_poly(a, M):
    return [x % M for x in a]


def add_poly(a, b, M):
    return [(x + y) % M for x, y in zip(a, b)]


def sub_poly(a, b, M):
    return [(x - y) % M for x, y in zip(a, b)]
