// kernels.cu -- sampling, pointwise, exact RNS and linear kernels of the BFV evaluator.
//
// Randomness: Philox4x64-10 (Salmon et al., SC'11) with key (seed, purpose)
// and counter (block, poly, limb, kind): uniform residues use the word pair
// (w_hi, w_lo) of block n>>1 at offset 2(n&1) reduced as (w_hi 2^64 + w_lo)
// mod q; small samples use word n&3 of block n>>2 (kind 1): ternary {0, 1,
// -1}[w mod 3], centred binomial popcount(w & (2^21-1)) - popcount((w >> 21)
// & (2^21-1)).
//
// The exact base extensions (lift, scale-and-round, mod-down, decryption's
// last step) are in ext.cu.
#include "kernels.cuh"

namespace {

constexpr int TPB = 256;

inline int grid_for(size_t work) {
    size_t b = (work + TPB - 1) / TPB;
    if (b > (size_t)1 << 30) b = (size_t)1 << 30;
    return (int)(b ? b : 1);
}

// ---------------------------------------------------------------- Philox4x64-10
__device__ __forceinline__ void philox4x64(u64 c[4], u64 k0, u64 k1) {
    const u64 M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const u64 W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += W0;
            k1 += W1;
        }
        const u64 lo0 = M0 * c[0], hi0 = __umul64hi(M0, c[0]);
        const u64 lo1 = M1 * c[2], hi1 = __umul64hi(M1, c[2]);
        const u64 n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

__global__ void k_sample_uniform(u64* out, int n_polys, int n_limbs, LimbMap map, PrimeTab tab, const u64* R2,
                                 u64 seed, u64 purpose, u64 poly_base, int N) {
    const size_t half = (size_t)N >> 1;
    const size_t total = (size_t)n_polys * n_limbs * half;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t blk = idx % half;
        const int limb = (int)((idx / half) % n_limbs);
        const int poly = (int)(idx / (half * n_limbs));
        const int p = map(limb);
        const u64 q = tab.q[p], qinv = tab.qinv[p], mu = tab.mu[p], r2 = R2[p];
        u64 c[4] = {(u64)blk, poly_base + (u64)poly, (u64)limb, 0ull};
        philox4x64(c, seed, purpose);
        u64* o = out + ((size_t)poly * n_limbs + limb) * N + 2 * blk;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const u64 lo = c[2 * h], hi = reduce64(c[2 * h + 1], q, mu);
            const u64 t1 = redc(hi, lo, q, qinv);                 // (hi 2^64 + lo) 2^-64
            o[h] = redc(__umul64hi(t1, r2), t1 * r2, q, qinv);   // * 2^128 * 2^-64
        }
    }
}

__global__ void k_sample_small(i64* out, int n_polys, u64 seed, u64 purpose, u64 poly_base, int cbd, int N) {
    const size_t quarter = (size_t)N >> 2;
    const size_t total = (size_t)n_polys * quarter;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t blk = idx % quarter;
        const int poly = (int)(idx / quarter);
        u64 c[4] = {(u64)blk, poly_base + (u64)poly, 0ull, 1ull};
        philox4x64(c, seed, purpose);
        i64* o = out + (size_t)poly * N + 4 * blk;
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const u64 w = c[h];
            if (cbd) {
                o[h] = (i64)__popcll(w & 0x1FFFFFull) - (i64)__popcll((w >> 21) & 0x1FFFFFull);
            } else {
                const u64 m = w % 3ull;
                o[h] = m == 0 ? 0 : (m == 1 ? 1 : -1);
            }
        }
    }
}

__global__ void k_spread(const i64* in, u64* out, int n_polys, int n_limbs, LimbMap map, PrimeTab tab, int N) {
    const size_t total = (size_t)n_polys * n_limbs * N;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(idx % N);
        const int limb = (int)((idx / N) % n_limbs);
        const int poly = (int)(idx / ((size_t)N * n_limbs));
        const u64 q = tab.q[map(limb)];
        const i64 v = in[(size_t)poly * N + k];
        out[idx] = v >= 0 ? (u64)v : q - (u64)(-v);
    }
}

// ---------------------------------------------------------------- pointwise (NTT domain)
__global__ void k_pointwise(const u64* A, const u64* B, u64* out, int n, int polys, int n_limbs, LimbMap map,
                            PrimeTab tab, PwStrides s, int N) {
    const size_t total = (size_t)n * polys * n_limbs * N;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(idx % N);
        const int limb = (int)((idx / N) % n_limbs);
        const size_t cp = idx / ((size_t)N * n_limbs);
        const int p = (int)(cp % polys);
        const size_t c = cp / polys;
        const int pi = map(limb);
        const u64 q = tab.q[pi], qinv = tab.qinv[pi];
        const size_t off = (size_t)limb * N + k;
        const u64 a = A[c * s.a_cs + p * s.a_ps + off];
        const u64 b = B[c * s.b_cs + p * s.b_ps + off];
        out[c * s.o_cs + p * s.o_ps + off] = redc(__umul64hi(a, b), a * b, q, qinv);
    }
}

// tensor in place: X[c][0..3] = (a0, a1, b0, b1) -> X[c][0..2] = (d0, d1, d2), Montgomery factor 2^-64
// Each thread takes two consecutive words (one 16-byte load per operand; N is even, so a pair never
// straddles limbs, and every limb starts 16-byte aligned).
__device__ __forceinline__ void tensor_word(u64 a0, u64 a1, u64 b0, u64 b1, u64 q, u64 qinv, u64& d0, u64& d1,
                                            u64& d2) {
    d0 = redc(__umul64hi(a0, b0), a0 * b0, q, qinv);
    u64 hi = 0, lo = 0;
    mac128(hi, lo, a0, b1);
    mac128(hi, lo, a1, b0);
    d1 = redc(hi, lo, q, qinv);
    d2 = redc(__umul64hi(a1, b1), a1 * b1, q, qinv);
}

__global__ void k_tensor(u64* X, int n, int LK, LimbMap map, PrimeTab tab, int N) {
    const size_t plane = (size_t)LK * N, half = plane / 2;
    const size_t total = (size_t)n * half;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t c = idx / half, off = (idx % half) * 2;
        const int pi = map((int)(off / N));
        const u64 q = tab.q[pi], qinv = tab.qinv[pi];
        ulonglong2* x = reinterpret_cast<ulonglong2*>(X + c * 4 * plane + off);
        const size_t p2 = half;   // one plane in 16-byte units
        const ulonglong2 a0 = x[0], a1 = x[p2], b0 = x[2 * p2], b1 = x[3 * p2];
        u64 e0, e1, e2, f0, f1, f2;
        tensor_word(a0.x, a1.x, b0.x, b1.x, q, qinv, e0, e1, e2);
        tensor_word(a0.y, a1.y, b0.y, b1.y, q, qinv, f0, f1, f2);
        x[0] = make_ulonglong2(e0, f0);
        x[p2] = make_ulonglong2(e1, f1);
        x[2 * p2] = make_ulonglong2(e2, f2);
    }
}

// squaring: X[c][0..1] = (a0, a1) -> X[c][0..2] = (a0^2, 2 a0 a1, a1^2), same sums as the general tensor
__global__ void k_tensor_sq(u64* X, int n, int LK, LimbMap map, PrimeTab tab, int N) {
    const size_t plane = (size_t)LK * N, half = plane / 2;
    const size_t total = (size_t)n * half;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t c = idx / half, off = (idx % half) * 2;
        const int pi = map((int)(off / N));
        const u64 q = tab.q[pi], qinv = tab.qinv[pi];
        ulonglong2* x = reinterpret_cast<ulonglong2*>(X + c * 4 * plane + off);
        const size_t p2 = half;
        const ulonglong2 a0 = x[0], a1 = x[p2];
        u64 e0, e1, e2, f0, f1, f2;
        tensor_word(a0.x, a1.x, a0.x, a1.x, q, qinv, e0, e1, e2);
        tensor_word(a0.y, a1.y, a0.y, a1.y, q, qinv, f0, f1, f2);
        x[0] = make_ulonglong2(e0, f0);
        x[p2] = make_ulonglong2(e1, f1);
        x[2 * p2] = make_ulonglong2(e2, f2);
    }
}

// z = sl + sm 2^28 + sh 2^56 as a 128-bit (hi, lo)
__device__ __forceinline__ void join28(u64 sl, u64 sm, u64 sh, u64& hi, u64& lo) {
    const u64 mlo = sm << 28, hlo = sh << 56;
    u64 r = sl + mlo;
    u64 c = r < mlo ? 1ull : 0ull;
    lo = r + hlo;
    c += lo < hlo ? 1ull : 0ull;
    hi = (sm >> 36) + (sh >> 8) + c;
}

// key-switch inner product: W[c][comp][k] = sum_j Dg[c][j][k] * rlk[j][comp][k]  (REDC).
// A thread owns one word (k, coefficient) of Q u P: it keeps the 2L key words of that word in
// registers and walks a group of ciphertexts, so the key is read once per group.  Up to 8 data primes
// the digits of the next two ciphertexts are in flight while the current one is accumulated; above 8
// there is no look-ahead, so that two CTAs of 256 threads still fit an SM (at 16 primes: 166 -> 128
// registers, +3% mul_relin at N = 32768).
// SPLIT (every prime below 2^50, so digits < 64q < 2^56 and key words < 2^50): each operand is cut at bit
// 28, a = ah 2^28 + al, b = bh 2^28 + bl (al, ah, bl < 2^28, bh < 2^22), and the three partial sums
// sum al bl, sum (al bh + ah bl), sum ah bh (weights 1, 2^28, 2^56) are 32 x 32 -> 64-bit multiply-adds into
// 64-bit accumulators: below 16 (2^56 + 2^56) = 2^61 for up to 16 terms, so none overflows; they are joined
// into the 128-bit sum once per output.  Otherwise each term is a full 64 x 64 -> 128-bit product.
template <int L, bool SPLIT>
__global__ void __launch_bounds__(256, 2) k_inner(const u64* Dg, const u64* rlk, u64* W, int n, int QP,
                                                              int cpg, PrimeTab tab, int N) {
    static_assert(!SPLIT || L <= 16, "the split sums are bounded for at most 16 terms");
    constexpr int D = L <= 8 ? 2 : 0;
    constexpr uint32_t M28 = (1u << 28) - 1;
    const size_t plane = (size_t)QP * N;
    const int groups = (n + cpg - 1) / cpg;
    const size_t total = plane * groups;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t off = idx % plane;
        const int grp = (int)(idx / plane);
        const int k = (int)(off / N);
        const u64 q = tab.q[k], qinv = tab.qinv[k];
        u64 k0[L], k1[L];   // SPLIT: (bh << 32) | bl
#pragma unroll
        for (int j = 0; j < L; ++j) {
            k0[j] = rlk[((size_t)j * 2 + 0) * plane + off];
            k1[j] = rlk[((size_t)j * 2 + 1) * plane + off];
            if constexpr (SPLIT) {
                k0[j] = ((k0[j] >> 28) << 32) | ((uint32_t)k0[j] & M28);
                k1[j] = ((k1[j] >> 28) << 32) | ((uint32_t)k1[j] & M28);
            }
        }
        const int c0 = grp * cpg, c_end = min(n, (grp + 1) * cpg);
        u64 buf[D + 1][L];
#pragma unroll
        for (int b = 0; b < D; ++b) {
            if (c0 + b < c_end) {
                const u64* d = Dg + (size_t)(c0 + b) * L * plane + off;
#pragma unroll
                for (int j = 0; j < L; ++j) buf[b][j] = d[(size_t)j * plane];
            }
        }
        for (int c = c0; c < c_end; ++c) {
            if (c + D < c_end) {
                const u64* d = Dg + (size_t)(c + D) * L * plane + off;
#pragma unroll
                for (int j = 0; j < L; ++j) buf[D][j] = d[(size_t)j * plane];
            }
            u64 h0 = 0, l0 = 0, h1 = 0, l1 = 0;
            if constexpr (SPLIT) {
                u64 s0l = 0, s0m = 0, s0h = 0, s1l = 0, s1m = 0, s1h = 0;
#pragma unroll
                for (int j = 0; j < L; ++j) {
                    const uint32_t al = (uint32_t)buf[0][j] & M28, ah = (uint32_t)(buf[0][j] >> 28);
                    const uint32_t b0l = (uint32_t)k0[j], b0h = (uint32_t)(k0[j] >> 32);
                    const uint32_t b1l = (uint32_t)k1[j], b1h = (uint32_t)(k1[j] >> 32);
                    s0l += (u64)al * b0l;
                    s0m += (u64)al * b0h;
                    s0m += (u64)ah * b0l;
                    s0h += (u64)ah * b0h;
                    s1l += (u64)al * b1l;
                    s1m += (u64)al * b1h;
                    s1m += (u64)ah * b1l;
                    s1h += (u64)ah * b1h;
                }
                join28(s0l, s0m, s0h, h0, l0);
                join28(s1l, s1m, s1h, h1, l1);
            } else {
#pragma unroll
                for (int j = 0; j < L; ++j) {
                    mac128(h0, l0, buf[0][j], k0[j]);
                    mac128(h1, l1, buf[0][j], k1[j]);
                }
            }
            W[((size_t)c * 2 + 0) * plane + off] = redc(h0, l0, q, qinv);
            W[((size_t)c * 2 + 1) * plane + off] = redc(h1, l1, q, qinv);
#pragma unroll
            for (int b = 0; b < D; ++b)
#pragma unroll
                for (int j = 0; j < L; ++j) buf[b][j] = buf[b + 1][j];
        }
    }
}

// the same inner product for 17 or more data primes (insecure test-only parameter sets): sizes at run time,
// one thread per (ciphertext, word), the key re-read per ciphertext
__global__ void k_inner_n(const u64* Dg, const u64* rlk, u64* W, int n, int QP, int L, PrimeTab tab, int N) {
    const size_t plane = (size_t)QP * N;
    const size_t total = plane * n;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t off = idx % plane;
        const size_t c = idx / plane;
        const int k = (int)(off / N);
        const u64 q = tab.q[k], qinv = tab.qinv[k];
        const u64* d = Dg + c * L * plane + off;
        u64 h0 = 0, l0 = 0, h1 = 0, l1 = 0;
#pragma unroll 1
        for (int j = 0; j < L; ++j) {
            const u64 dj = d[(size_t)j * plane];
            mac128(h0, l0, dj, rlk[((size_t)j * 2 + 0) * plane + off]);
            mac128(h1, l1, dj, rlk[((size_t)j * 2 + 1) * plane + off]);
        }
        W[(c * 2 + 0) * plane + off] = redc(h0, l0, q, qinv);
        W[(c * 2 + 1) * plane + off] = redc(h1, l1, q, qinv);
    }
}

// ---------------------------------------------------------------- encode/decode, encrypt, keygen
__global__ void k_permute(const u64* in, u64* out, const uint32_t* brv, int n, int scatter, int N, u64 t,
                          uint32_t* flags) {
    const size_t total = (size_t)n * N;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(idx % N);
        const size_t base = idx - j;
        if (scatter) {
            const u64 v = in[idx];   // a slot value being encoded: must be < t
            if (v >= t) atomicOr(flags, BFHE_FLAG_PLAINTEXT);
            out[base + brv[j]] = v;
        } else {
            out[idx] = in[base + brv[j]];
        }
    }
}

__global__ void k_enc_finish(u64* ct, const u64* M, const i64* e1, const i64* e2, int n, int L, const u64* qtab,
                             const u64* delta, int N, u64 t, uint32_t* flags) {
    const size_t total = (size_t)n * L * N;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(idx % N);
        const int i = (int)((idx / N) % L);
        const size_t c = idx / ((size_t)N * L);
        const u64 q = qtab[i];
        const u64 m = M[c * N + k];
        if (i == 0 && m >= t) atomicOr(flags, BFHE_FLAG_PLAINTEXT);   // plaintext coefficients must be < t
        const i64 a = e1[c * N + k], b = e2[c * N + k];
        u64* c0 = ct + (c * 2 * L + i) * N + k;
        u64* c1 = c0 + (size_t)L * N;
        u64 v = add_mod(*c0, shoup(m, delta[i], delta[L + i], q), q);
        v = a >= 0 ? add_mod(v, (u64)a, q) : sub_mod(v, (u64)(-a), q);
        *c0 = v;
        u64 w = *c1;
        *c1 = b >= 0 ? add_mod(w, (u64)b, q) : sub_mod(w, (u64)(-b), q);
    }
}

// out = -(as + e) [+ [P]_{q_j} s2 on limb j of poly j when gadget]
__global__ void k_neg_add_small(const u64* as, const i64* e, u64* out, int n_polys, int n_limbs, LimbMap map,
                                PrimeTab tab, const u64* s2, int gadget, const u64* Pq, int L, int N) {
    const size_t total = (size_t)n_polys * n_limbs * N;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(idx % N);
        const int limb = (int)((idx / N) % n_limbs);
        const int poly = (int)(idx / ((size_t)N * n_limbs));
        const u64 q = tab.q[map(limb)];
        const i64 ev = e[(size_t)poly * N + k];
        u64 v = as[idx];
        v = ev >= 0 ? add_mod(v, (u64)ev, q) : sub_mod(v, (u64)(-ev), q);
        v = v == 0 ? 0 : q - v;
        if (gadget && limb == poly) {
            const u64 g = shoup(s2[(size_t)limb * N + k], Pq[limb], Pq[L + limb], q);
            v = add_mod(v, g, q);
        }
        out[idx] = v;
    }
}

// ---------------------------------------------------------------- linear ops
__device__ __forceinline__ u64 apply(u64 acc, u64 v, int c, u64 q) {
    switch (c) {
        case 1: return add_mod(acc, v, q);
        case 2: return add_mod(add_mod(acc, v, q), v, q);
        case -1: return sub_mod(acc, v, q);
        case -2: return sub_mod(sub_mod(acc, v, q), v, q);
        default: return acc;
    }
}

__constant__ int c_gate_coef[8][5] = {
    // cc  cx  cy  cz  cp
    {0, 0, 0, 0, 1},     // AND  = xy
    {0, 1, 1, 0, -1},    // OR   = x + y - xy
    {0, 1, 1, 0, -2},    // XOR  = x + y - 2xy
    {1, 0, 0, 0, -1},    // NAND = 1 - xy
    {1, -1, -1, 0, 1},   // NOR  = 1 - (x + y - xy)
    {1, -1, -1, 0, 2},   // XNOR = 1 - (x + y - 2xy)
    {1, -1, 0, 0, 0},    // NOT  = 1 - x
    {0, 0, 0, 1, 1},     // MUX  = x (y - z) + z
};

__device__ __forceinline__ u64 lin_word(int cc, int cx, int cy, int cz, int cp, u64 cval, const u64* x,
                                        const u64* y, const u64* z, const u64* p, size_t o, int comp, int k,
                                        u64 q, u64 dw, u64 dws) {
    u64 acc = 0;
    if (cc != 0 && comp == 0 && k == 0) acc = apply(acc, shoup(cval, dw, dws, q), cc, q);
    if (cx) acc = apply(acc, x[o], cx, q);
    if (cy) acc = apply(acc, y[o], cy, q);
    if (cz) acc = apply(acc, z[o], cz, q);
    if (cp) acc = apply(acc, p[o], cp, q);
    return acc;
}

__global__ void k_lincomb(u64* out, const u64* x, const u64* y, const u64* z, const u64* p, LinCoef cf, u64 cval,
                          size_t n, int L, const u64* qtab, const u64* delta, int N) {
    const size_t total = n * 2 * L * N;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(idx % N);
        const int i = (int)((idx / N) % L);
        const int comp = (int)((idx / ((size_t)N * L)) & 1);
        out[idx] = lin_word(cf.cc, cf.cx, cf.cy, cf.cz, cf.cp, cval, x, y, z, p, idx, comp, k, qtab[i], delta[i],
                            delta[L + i]);
    }
}

struct ScalarPairs {
    u64 w[BFHE_MAX_L], ws[BFHE_MAX_L];
};

__global__ void k_mul_scalar(const u64* a, u64* out, ScalarPairs sp, size_t n, int L, const u64* qtab, int N) {
    const size_t total = n * 2 * L * N;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)((idx / N) % L);
        out[idx] = shoup(a[idx], sp.w[i], sp.ws[i], qtab[i]);
    }
}

// Listing 5: r = v[s-1]; r += r + v[i], i = s-2 .. 0
__global__ void k_horner(const u64* bits, uint32_t s, u64* out, size_t n, int L, const u64* qtab, int N) {
    const size_t words = n * 2 * L * N;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < words;
         idx += (size_t)gridDim.x * blockDim.x) {
        const u64 q = qtab[(idx / N) % L];
        u64 r = bits[(size_t)(s - 1) * words + idx];
        for (int i = (int)s - 2; i >= 0; --i) r = add_mod(r, add_mod(r, bits[(size_t)i * words + idx], q), q);
        out[idx] = r;
    }
}

// gather gate operands: A[g] = wires[x], B[g] = wires[y] (MUX: wires[y] - wires[z])
__global__ void k_gather_ops(u64* A, u64* B, const u64* wires, size_t ctw, const int32_t* table, int n_gates,
                             int L, const u64* qtab, int N) {
    const size_t total = (size_t)n_gates * ctw;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int g = (int)(idx / ctw);
        const size_t o = idx % ctw;
        const int32_t* e = table + 5 * g;
        const u64 q = qtab[(o / N) % L];
        A[idx] = wires[(size_t)e[1] * ctw + o];
        const u64 yv = wires[(size_t)e[2] * ctw + o];
        B[idx] = (e[0] & 0xff) == BFHE_MUX ? sub_mod(yv, wires[(size_t)e[3] * ctw + o], q) : yv;
    }
}

// gate epilogue: wires[out] = lin(op)(x, y, z, prod[g]); entries g >= n_mul have no product
__global__ void k_gate_epilogue(u64* wires, size_t ctw, const int32_t* table, int n_gates, int n_mul,
                                const u64* prod, int L, const u64* qtab, const u64* delta, int N) {
    const size_t total = (size_t)n_gates * ctw;
    const size_t per_comp = (size_t)L * N;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int g = (int)(idx / ctw);
        const size_t o = idx % ctw;
        const int32_t* e = table + 5 * g;
        const int op = e[0] & 0xff;
        int cc, cx, cy, cz, cp;
        if (op == BFHE_OP_MUL) {
            cc = cx = cy = cz = 0;
            cp = 1;
        } else if (op == BFHE_OP_LIN) {
            const int code = e[0] >> 8;
            cc = code / 125 - 2;
            cx = (code / 25) % 5 - 2;
            cy = (code / 5) % 5 - 2;
            cz = code % 5 - 2;
            cp = 0;
        } else {
            const int* cf = c_gate_coef[op & 7];
            cc = cf[0];
            cx = cf[1];
            cy = cf[2];
            cz = cf[3];
            cp = cf[4];
        }
        if (g >= n_mul) cp = 0;
        const int i = (int)((o / N) % L);
        const int k = (int)(o % N);
        const int comp = (int)((o / per_comp) & 1);
        const u64* x = wires + (size_t)e[1] * ctw;
        const u64* y = wires + (size_t)e[2] * ctw;
        const u64* z = wires + (size_t)e[3] * ctw;
        const u64* p = g < n_mul ? prod + (size_t)g * ctw : nullptr;
        wires[(size_t)e[4] * ctw + o] =
            lin_word(cc, cx, cy, cz, cp, 1, x, y, z, p, o, comp, k, qtab[i], delta[i], delta[L + i]);
    }
}

// integer-pipe probe: 8 independent lazy Shoup chains per thread
__global__ void k_probe_modmul(u64* out, uint32_t iters, u64 q, u64 w, u64 ws) {
    u64 x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = (u64)threadIdx.x * 977u + (u64)blockIdx.x * 131u + (u64)i;
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = shoup_lazy(x[i], w, ws, q);
    }
    u64 s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s ^= x[i];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// trivial ciphertexts (Delta bit_k(c_base + c), 0), layout [s][C][n][2][L][N]
__global__ void k_trivial_bits(u64* out, uint32_t s, u64 c_base, const u64* cbp, int C, size_t n, int L,
                               const u64* delta, int N) {
    if (cbp) c_base = *cbp;
    const size_t ctw = (size_t)2 * L * N;
    const size_t total = (size_t)s * C * n * ctw;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t o = idx % ctw;
        const size_t rest = idx / ctw;
        const int c = (int)((rest / n) % C);
        const int kbit = (int)(rest / (n * C));
        const int i = (int)(o / N);   // < L only for c0
        u64 v = 0;
        if (o < (size_t)L * N && (o % N) == 0 && (((c_base + c) >> kbit) & 1)) v = delta[i];
        out[idx] = v;
    }
}

// bits[k][i] += sum over c of src (PAPER: src [s][C][n]; SELECT: src [C][n], only if bit k of c)
__global__ void k_accumulate(u64* bits, const u64* src, uint32_t s, u64 c_base, const u64* cbp, int C, size_t n,
                             int select, int L, const u64* qtab, int N) {
    if (cbp) c_base = *cbp;
    const size_t ctw = (size_t)2 * L * N;
    const size_t words = n * ctw;
    const size_t total = (size_t)s * words;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int kbit = (int)(idx / words);
        const size_t w = idx % words;
        const u64 q = qtab[(w / N) % L];
        u64 acc = bits[idx];
        for (int c = 0; c < C; ++c) {
            if (select) {
                if (((c_base + c) >> kbit) & 1) acc = add_mod(acc, src[(size_t)c * words + w], q);
            } else {
                acc = add_mod(acc, src[((size_t)kbit * C + c) * words + w], q);
            }
        }
        bits[idx] = acc;
    }
}

// out[c][i] = x[i] - (c_base + c)   (layout [C][n])
__global__ void k_sub_const_chains(const u64* x, u64* out, u64 c_base, const u64* cbp, int C, size_t n, int L,
                                   const u64* qtab, const u64* delta, u64 t, int N) {
    if (cbp) c_base = *cbp;
    const size_t ctw = (size_t)2 * L * N;
    const size_t words = n * ctw;
    const size_t total = (size_t)C * words;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(idx / words);
        const size_t w = idx % words;
        const size_t o = w % ctw;
        u64 v = x[w];
        if (o < (size_t)L * N && (o % N) == 0) {
            const int i = (int)(o / N);
            const u64 q = qtab[i];
            const u64 cv = (c_base + c) % t;
            v = sub_mod(v, shoup(cv, delta[i], delta[L + i], q), q);
        }
        out[idx] = v;
    }
}

// one device word (the candidate base read by a replayed mod_to_bits tile)
__global__ void k_set_word(u64* w, u64 v) { *w = v; }

}  // namespace

// ================================================================== launchers
#define LAUNCH(kern, work, ...)                                                   \
    do {                                                                          \
        auto* _kfn = kern;                                                        \
        _kfn<<<grid_for(work), TPB, 0, st>>>(__VA_ARGS__);                       \
        BFHE_LAUNCH_CHECK(#kern);                                                \
    } while (0)

int launch_sample_uniform(const bfhe_ctx* ctx, u64* out, int n_polys, int n_limbs, LimbMap map, u64 seed,
                          u64 purpose, u64 poly_base, cudaStream_t st) {
    LAUNCH(k_sample_uniform, (size_t)n_polys * n_limbs * ctx->N / 2, out, n_polys, n_limbs, map, ctx->tab, ctx->d_R2,
           seed, purpose, poly_base, (int)ctx->N);
    return BFHE_OK;
}

int launch_sample_small(const bfhe_ctx* ctx, i64* out, int n_polys, u64 seed, u64 purpose, u64 poly_base, int cbd,
                        cudaStream_t st) {
    LAUNCH(k_sample_small, (size_t)n_polys * ctx->N / 4, out, n_polys, seed, purpose, poly_base, cbd, (int)ctx->N);
    return BFHE_OK;
}

int launch_spread(const bfhe_ctx* ctx, const i64* in, u64* out, int n_polys, int n_limbs, LimbMap map,
                  cudaStream_t st) {
    LAUNCH(k_spread, (size_t)n_polys * n_limbs * ctx->N, in, out, n_polys, n_limbs, map, ctx->tab, (int)ctx->N);
    return BFHE_OK;
}

int launch_pointwise(const bfhe_ctx* ctx, const u64* A, const u64* B, u64* out, int n, int polys, int n_limbs,
                     LimbMap map, PwStrides s, cudaStream_t st) {
    LAUNCH(k_pointwise, (size_t)n * polys * n_limbs * ctx->N, A, B, out, n, polys, n_limbs, map, ctx->tab, s,
           (int)ctx->N);
    return BFHE_OK;
}

int launch_tensor(const bfhe_ctx* ctx, u64* X, int n, int square, cudaStream_t st) {
    // per word of Q u B: 4 read, 3 written (squaring: 2 read)
    ProfScope ps(ctx, BFHE_K_TENSOR, st, 4.0 * n * (ctx->L + ctx->K) * ctx->N,
                 (square ? 40.0 : 56.0) * n * (ctx->L + ctx->K) * ctx->N);
    const int LK = (int)(ctx->L + ctx->K);
    if (square)
        LAUNCH(k_tensor_sq, (size_t)n * LK * ctx->N / 2, X, n, LK, ctx->mapQB(), ctx->tab, (int)ctx->N);
    else
        LAUNCH(k_tensor, (size_t)n * LK * ctx->N / 2, X, n, LK, ctx->mapQB(), ctx->tab, (int)ctx->N);
    return BFHE_OK;
}

template <int L>
int run_inner(const bfhe_ctx* ctx, const u64* Dg, u64* W, int n, cudaStream_t st) {
    const int QP = (int)(ctx->L + ctx->alpha);
    const int cpg = n < 4 ? 1 : (n + 3) / 4;   // four groups: enough threads, key read four times
    const size_t work = (size_t)QP * ctx->N * ((n + cpg - 1) / cpg);
    if (ctx->prime_bits <= 50)   // digits below 64q < 2^56 (lazy transforms), key words below 2^50
        LAUNCH((k_inner<L, true>), work, Dg, ctx->d_rlk_ntt, W, n, QP, cpg, ctx->tab, (int)ctx->N);
    else
        LAUNCH((k_inner<L, false>), work, Dg, ctx->d_rlk_ntt, W, n, QP, cpg, ctx->tab, (int)ctx->N);
    return BFHE_OK;
}

#define SWITCH_L(Lv, FN, ...)                                                                                  \
    switch (Lv) {                                                                                              \
        case 1: return FN<1>(__VA_ARGS__);                                                                     \
        case 2: return FN<2>(__VA_ARGS__);                                                                     \
        case 3: return FN<3>(__VA_ARGS__);                                                                     \
        case 4: return FN<4>(__VA_ARGS__);                                                                     \
        case 5: return FN<5>(__VA_ARGS__);                                                                     \
        case 6: return FN<6>(__VA_ARGS__);                                                                     \
        case 7: return FN<7>(__VA_ARGS__);                                                                     \
        case 8: return FN<8>(__VA_ARGS__);                                                                     \
        case 9: return FN<9>(__VA_ARGS__);                                                                     \
        case 10: return FN<10>(__VA_ARGS__);                                                                   \
        case 11: return FN<11>(__VA_ARGS__);                                                                   \
        case 12: return FN<12>(__VA_ARGS__);                                                                   \
        case 13: return FN<13>(__VA_ARGS__);                                                                   \
        case 14: return FN<14>(__VA_ARGS__);                                                                   \
        case 15: return FN<15>(__VA_ARGS__);                                                                   \
        case 16: return FN<16>(__VA_ARGS__);                                                                   \
        default: break;                                                                                        \
    }

int launch_inner(const bfhe_ctx* ctx, const u64* Dg, u64* W, int n, cudaStream_t st) {
    // per word of Q u P: L digits read and 2 words written per ciphertext, the key's 2L words once
    ProfScope ps(ctx, BFHE_K_INNER, st, 2.0 * ctx->L * n * (ctx->L + ctx->alpha) * ctx->N,
                 8.0 * (ctx->L + ctx->alpha) * ctx->N * ((double)n * (ctx->L + 2) + 2.0 * ctx->L));
    SWITCH_L(ctx->L, run_inner, ctx, Dg, W, n, st)
    if (ctx->L > BFHE_MAX_L) return set_error(BFHE_EINVAL, "unsupported number of data primes");
    const int QP = (int)(ctx->L + ctx->alpha);
    LAUNCH(k_inner_n, (size_t)QP * ctx->N * n, Dg, ctx->d_rlk_ntt, W, n, QP, (int)ctx->L, ctx->tab, (int)ctx->N);
    return BFHE_OK;
}

int launch_permute(const bfhe_ctx* ctx, const u64* in, u64* out, int n, int scatter, cudaStream_t st) {
    LAUNCH(k_permute, (size_t)n * ctx->N, in, out, ctx->d_brv, n, scatter, (int)ctx->N, ctx->t, ctx->d_flags);
    return BFHE_OK;
}

int launch_enc_finish(const bfhe_ctx* ctx, u64* ct, const u64* M, const i64* e1, const i64* e2, int n,
                      cudaStream_t st) {
    LAUNCH(k_enc_finish, (size_t)n * ctx->L * ctx->N, ct, M, e1, e2, n, (int)ctx->L, ctx->tab.q, ctx->d_delta_q,
           (int)ctx->N, ctx->t, ctx->d_flags);
    return BFHE_OK;
}

int launch_neg_add_small(const bfhe_ctx* ctx, const u64* as, const i64* e, u64* out, int n_polys, int n_limbs,
                         LimbMap map, const u64* s2, int gadget, cudaStream_t st) {
    LAUNCH(k_neg_add_small, (size_t)n_polys * n_limbs * ctx->N, as, e, out, n_polys, n_limbs, map, ctx->tab, s2,
           gadget, ctx->d_P_q, (int)ctx->L, (int)ctx->N);
    return BFHE_OK;
}

int launch_lincomb(const bfhe_ctx* ctx, u64* out, const u64* x, const u64* y, const u64* z, const u64* p,
                   LinCoef cf, u64 cval, size_t n, cudaStream_t st) {
    LAUNCH(k_lincomb, n * ctx->ct_words(), out, x, y, z, p, cf, cval, n, (int)ctx->L, ctx->tab.q, ctx->d_delta_q,
           (int)ctx->N);
    return BFHE_OK;
}

int launch_mul_scalar(const bfhe_ctx* ctx, const u64* a, u64 c, u64* out, size_t n, cudaStream_t st) {
    ScalarPairs sp;
    for (uint32_t i = 0; i < ctx->L; ++i) {
        const u64 q = ctx->primes[i];
        const u64 w = c % q;
        sp.w[i] = w;
        sp.ws[i] = (u64)(((u128)w << 64) / q);
    }
    LAUNCH(k_mul_scalar, n * ctx->ct_words(), a, out, sp, n, (int)ctx->L, ctx->tab.q, (int)ctx->N);
    return BFHE_OK;
}

int launch_horner(const bfhe_ctx* ctx, const u64* bits, uint32_t s, u64* out, size_t n, cudaStream_t st) {
    LAUNCH(k_horner, n * ctx->ct_words(), bits, s, out, n, (int)ctx->L, ctx->tab.q, (int)ctx->N);
    return BFHE_OK;
}

int launch_gather(const bfhe_ctx* ctx, u64* dst, const u64* wires, size_t n, const int32_t* table, int n_gates,
                  int field, int sub_field, cudaStream_t st) {
    // field/sub_field are unused by this layout: dst holds A then B ([2][n_gates][n] ciphertexts)
    (void)field;
    (void)sub_field;
    const size_t ctw = n * ctx->ct_words();
    u64* A = dst;
    u64* B = dst + (size_t)n_gates * ctw;
    LAUNCH(k_gather_ops, (size_t)n_gates * ctw, A, B, wires, ctw, table, n_gates, (int)ctx->L, ctx->tab.q,
           (int)ctx->N);
    return BFHE_OK;
}

int launch_gate_epilogue(const bfhe_ctx* ctx, u64* wires, size_t n, const int32_t* table, int n_gates,
                         const u64* prod, int n_mul, cudaStream_t st) {
    const size_t ctw = n * ctx->ct_words();
    LAUNCH(k_gate_epilogue, (size_t)n_gates * ctw, wires, ctw, table, n_gates, n_mul, prod, (int)ctx->L, ctx->tab.q,
           ctx->d_delta_q, (int)ctx->N);
    return BFHE_OK;
}

int launch_trivial_bits(const bfhe_ctx* ctx, u64* out, uint32_t s, u64 c_base, const u64* cbp, int C, size_t n,
                        cudaStream_t st) {
    LAUNCH(k_trivial_bits, (size_t)s * C * n * ctx->ct_words(), out, s, c_base, cbp, C, n, (int)ctx->L, ctx->d_delta_q,
           (int)ctx->N);
    return BFHE_OK;
}

int launch_accumulate(const bfhe_ctx* ctx, u64* bits, const u64* src, uint32_t s, u64 c_base, const u64* cbp, int C,
                      size_t n, int select, cudaStream_t st) {
    LAUNCH(k_accumulate, (size_t)s * n * ctx->ct_words(), bits, src, s, c_base, cbp, C, n, select, (int)ctx->L, ctx->tab.q,
           (int)ctx->N);
    return BFHE_OK;
}

int launch_sub_const_chains(const bfhe_ctx* ctx, const u64* x, u64* out, u64 c_base, const u64* cbp, int C, size_t n,
                            cudaStream_t st) {
    LAUNCH(k_sub_const_chains, (size_t)C * n * ctx->ct_words(), x, out, c_base, cbp, C, n, (int)ctx->L, ctx->tab.q,
           ctx->d_delta_q, ctx->t, (int)ctx->N);
    return BFHE_OK;
}

int launch_set_word(u64* w, u64 v, cudaStream_t st) {
    k_set_word<<<1, 1, 0, st>>>(w, v);
    BFHE_LAUNCH_CHECK("k_set_word");
    return BFHE_OK;
}

int launch_probe_modmul(u64* out, int blocks, int threads, uint32_t iters, u64 q, u64 w, u64 ws, cudaStream_t st) {
    k_probe_modmul<<<blocks, threads, 0, st>>>(out, iters, q, w, ws);
    BFHE_LAUNCH_CHECK("k_probe_modmul");
    return BFHE_OK;
}
