// ext.cu -- exact base extensions of the multiply and of decryption.
//
// The multiply lifts each input coefficient to the centred range and extends
// it exactly to the auxiliary base (k_modup); scale-and-round computes
// round(t d / Q) as y = (t d - r) / Q with r the centred residue of t d mod Q,
// by two exact extensions (Q -> B for r, B -> Q for y; k_scale); mod-down
// extends the special-prime part to Q (k_moddown); decryption extends to t
// (k_dec_finish).  Extensions run Garner's mixed-radix conversion, or, when
// the context enables it, the guarded fast conversion (a fixed-point overflow
// count with a mixed-radix fallback near the rounding boundary).  Both give
// the same integers.
#include "kernels.cuh"

namespace {

constexpr int TPB = 256;

inline int grid_for(size_t work) {
    size_t b = (work + TPB - 1) / TPB;
    if (b > (size_t)1 << 30) b = (size_t)1 << 30;
    return (int)(b ? b : 1);
}

// ---------------------------------------------------------------- exact base extension
// Inputs x_i may be lazy (< 2 s_i); digits come out canonical.  Inner steps keep
// u in [0, 2 s_i): u + s_i - v_j < 3 s_i goes straight into a lazy Shoup product.
template <int NS>
__device__ __forceinline__ bool garner(const u64 (&x)[NS], const ExtDesc& d, u64 (&v)[NS]) {
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        const u64 si = d.src_q[i];
        u64 u = x[i];
#pragma unroll
        for (int j = 0; j < i; ++j) {
            u64 vj = v[j];
            vj = vj >= si ? vj - si : vj;
            u = shoup_lazy(u + si - vj, d.ginv[i * NS + j], d.ginv_s[i * NS + j], si);
        }
        u = u >= si ? u - si : u;
        v[i] = u;
    }
    int state = 0;
#pragma unroll
    for (int i = NS - 1; i >= 0; --i) {
        const u64 h = d.hdig[i];
        if (state == 0) state = v[i] > h ? 1 : (v[i] < h ? -1 : 0);
    }
    return state > 0;   // x > (S-1)/2: the centred value is x - S
}

// value mod T_j of the centred integer with digits v (SMALL: T may be far below the sources).
// Without SMALL every digit is < 2 T_j, so Horner runs lazily below 4 T_j.
template <int NS, bool SMALL>
__device__ __forceinline__ u64 ext_eval(const u64 (&v)[NS], bool neg, const ExtDesc& d, int j) {
    const u64 T = d.dst_q[j];
    u64 acc;
    if (SMALL) {
        const u64 mu = d.dst_mu[j];
        acc = reduce64(v[NS - 1], T, mu);
#pragma unroll
        for (int i = NS - 2; i >= 0; --i) {
            acc = shoup(acc, d.radix[j * NS + i], d.radix_s[j * NS + i], T);
            acc = add_mod(acc, reduce64(v[i], T, mu), T);
        }
    } else {
        acc = v[NS - 1];
#pragma unroll
        for (int i = NS - 2; i >= 0; --i)
            acc = shoup_lazy(acc, d.radix[j * NS + i], d.radix_s[j * NS + i], T) + v[i];
        const u64 T2 = T << 1;
        acc = acc >= T2 ? acc - T2 : acc;
        acc = acc >= T ? acc - T : acc;
    }
    if (neg) acc = sub_mod(acc, d.smod[j], T);
    return acc;
}

// The guarded fast extension's per-source factors and 26-bit limb pairs for NS sources and ND targets, passed by
// value as a kernel parameter (it sits in the constant bank): with the loops over sources and targets unrolled,
// every factor is an operand of the multiply-add that uses it, with no load instruction.
template <int NS, int ND>
struct FastTab {
    uint2 c[ND][NS];        // (low, high) 26-bit limbs of [(S/s_i) 2^64]_{T_j}
    u64 qh[NS], qhs[NS];    // [(S/s_i)^-1]_{s_i} and its Shoup companion
    u64 ghi[NS], glo[NS];   // floor(2^128 / s_i): high and low words
};

template <int NS, int ND>
FastTab<NS, ND> fast_tab(const ExtHost& h) {
    FastTab<NS, ND> t{};
    if (h.n != NS || h.m != ND) return t;   // only the instances the launchers use are ever filled
    for (int j = 0; j < ND; ++j)
        for (int i = 0; i < NS; ++i) t.c[j][i] = make_uint2(h.c26[((size_t)j * NS + i) * 2], h.c26[((size_t)j * NS + i) * 2 + 1]);
    for (int i = 0; i < NS; ++i) {
        t.qh[i] = h.qhinv[i];
        t.qhs[i] = h.qhinv_s[i];
        t.ghi[i] = h.g_hi[i];
        t.glo[i] = h.g_lo[i];
    }
    return t;
}

// Guarded fast exact extension (all moduli below 2^50), first half: y_i = [x_i (S/s_i)^-1]_{s_i} split
// into 26-bit limbs, and v = round(sum_i y_i / s_i) from the 64.64 fixed-point sum of
// floor(y_i floor(2^128/s_i) / 2^64) (each term at most 2 units below y_i 2^64 / s_i).  Returns false
// when the fraction lies within 2n + 2 units of 1/2: then the caller takes the exact mixed-radix path.
template <int NS, int ND>
__device__ __forceinline__ bool fast_prep(const u64 (&x)[NS], const ExtDesc& d, const FastTab<NS, ND>& ft,
                                          uint32_t (&y0)[NS], uint32_t (&y1)[NS], int& v) {
    u64 lo = 0, hi = 0;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        const u64 s = d.src_q[i];
        const u64 y = shoup(x[i], ft.qh[i], ft.qhs[i], s);
        y0[i] = (uint32_t)(y & 0x3FFFFFFull);
        y1[i] = (uint32_t)(y >> 26);
        const u64 term = y * ft.ghi[i] + __umul64hi(y, ft.glo[i]);
        lo += term;
        hi += lo < term ? 1ull : 0ull;
    }
    const u64 half = 1ull << 63;
    if (lo > half) {
        v = (int)hi + 1;
        return true;
    }
    if (lo + (u64)(2 * NS + 2) <= half) {
        v = (int)hi;
        return true;
    }
    return false;
}

// second half: sum_i y_i [(S/s_i) 2^64]_{T_j} with the 26-bit limb products accumulated in four 64-bit
// words (no carries below 2^13 sources), one Montgomery reduction, minus [v S]_{T_j}; canonical result
template <int NS, int ND>
__device__ __forceinline__ u64 fast_eval(const uint32_t (&y0)[NS], const uint32_t (&y1)[NS], int v, const ExtDesc& d,
                                         const FastTab<NS, ND>& ft, int j) {
    u64 p00 = 0, p01 = 0, p10 = 0, p11 = 0;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        const uint32_t c0 = ft.c[j][i].x, c1 = ft.c[j][i].y;
        p00 += (u64)y0[i] * c0;
        p01 += (u64)y0[i] * c1;
        p10 += (u64)y1[i] * c0;
        p11 += (u64)y1[i] * c1;
    }
    const u64 mid = p01 + p10;                       // weight 2^26
    u64 lo = p00 + (mid << 26);
    u64 hi = (mid >> 38) + (lo < p00 ? 1ull : 0ull);
    const u64 top = p11 << 52;                       // weight 2^52
    lo += top;
    hi += (p11 >> 12) + (lo < top ? 1ull : 0ull);
    const u64 T = d.dst_q[j];
    return sub_mod(redc(hi, lo, T, d.dst_qinv[j]), d.vS[(size_t)j * (NS + 1) + v], T);
}

// the same sum with three limb products per term (Karatsuba): the weight-2^26 part is
// sum (y0 + y1)(c0 + c1) - sum y0 c0 - sum y1 c1, the same integer (every factor below 2^27, every product
// below 2^54, so each sum fits 64 bits for fewer than 2^10 sources); scale-and-round takes this form, the base
// extension of the multiply's inputs keeps four products (fewer registers)
template <int NS, int ND>
__device__ __forceinline__ u64 fast_eval3(const uint32_t (&y0)[NS], const uint32_t (&y1)[NS], int v, const ExtDesc& d,
                                          const FastTab<NS, ND>& ft, int j) {
    static_assert(NS < 1024, "the three-product sums are bounded for fewer than 2^10 sources");
    u64 p00 = 0, pm = 0, p11 = 0;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        const uint32_t c0 = ft.c[j][i].x, c1 = ft.c[j][i].y;
        p00 += (u64)y0[i] * c0;
        p11 += (u64)y1[i] * c1;
        pm += (u64)(y0[i] + y1[i]) * (c0 + c1);
    }
    const u64 mid = pm - p00 - p11;                  // weight 2^26
    u64 lo = p00 + (mid << 26);
    u64 hi = (mid >> 38) + (lo < p00 ? 1ull : 0ull);
    const u64 top = p11 << 52;                       // weight 2^52
    lo += top;
    hi += (p11 >> 12) + (lo < top ? 1ull : 0ull);
    const u64 T = d.dst_q[j];
    return sub_mod(redc(hi, lo, T, d.dst_qinv[j]), d.vS[(size_t)j * (NS + 1) + v], T);
}

// X[c][slot] (slots a0 a1 b0 b1; only a0 a1 when squaring): Q limbs copied, B limbs = centred extension
template <int NS, bool FAST>
__global__ void __launch_bounds__(256, NS <= 8 ? 4 : 2) k_modup(const u64* A, const u64* B, u64* X, int n, int slots, int K, ExtDesc ext, int N,
                        uint32_t* flags, FastTab<FAST ? NS : 1, FAST ? NS + 1 : 1> ft) {
    const size_t total = (size_t)n * slots * N;
    const int LK = NS + K;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(idx % N);
        const size_t pp = idx / N;
        const size_t c = pp / slots;
        const int slot = (int)(pp % slots);
        const u64* src = (slot < 2 ? A : B) + (c * 2 + (slot & 1)) * (size_t)NS * N + k;
        u64* dst = X + (c * 4 + slot) * (size_t)LK * N + k;
        u64 x[NS];
        bool bad = false;
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            x[i] = src[(size_t)i * N];
            dst[(size_t)i * N] = x[i];
            bad |= x[i] >= ext.src_q[i];
        }
        if (bad) atomicOr(flags, BFHE_FLAG_RESIDUE);
        if constexpr (FAST) {
            uint32_t y0[NS], y1[NS];
            int vv = 0;
            if (fast_prep<NS, NS + 1>(x, ext, ft, y0, y1, vv)) {   // the fast path has K = NS + 1 targets
#pragma unroll
                for (int j = 0; j < NS + 1; ++j)
                    dst[(size_t)(NS + j) * N] = fast_eval<NS, NS + 1>(y0, y1, vv, ext, ft, j);
                continue;
            }
        }
        u64 v[NS];
        const bool neg = garner<NS>(x, ext, v);
        for (int j = 0; j < K; ++j) dst[(size_t)(NS + j) * N] = ext_eval<NS, false>(v, neg, ext, j);
    }
}

// pair (w, Shoup(w)) of the twist table row f of prime p at coefficient k: f = 1 is N^-1 psi^-k R,
// f = 2 is t N^-1 psi^-k R (mod the prime)
__device__ __forceinline__ ulonglong2 twist_at(const u64* twist, int p, int f, int k, int N) {
    return __ldg(reinterpret_cast<const ulonglong2*>(twist) + ((size_t)p * 3 + f) * N + k);
}

// scale-and-round of the tensor (X slots 0..2, Q u B limbs) into C3 [n][3][L][N].  The inverse transforms
// leave the tensor untwisted: the first product of each limb, by t, also carries the twist N^-1 psi^-k R.
template <int NS, int KS, bool FAST>
__global__ void __launch_bounds__(256, 2) k_scale(const u64* X, u64* C3, int n, ExtDesc eQB, ExtDesc eBQ, const u64* twist, int nP,
                        const u64* Qinv_b, const u64* bq, int N, FastTab<FAST ? NS : 1, FAST ? KS : 1> fq,
                        FastTab<FAST ? KS : 1, FAST ? NS : 1> fb) {
    const size_t total = (size_t)n * 3 * N;
    constexpr int LK = NS + KS;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(idx % N);
        const size_t cp = idx / N;
        const size_t c = cp / 3;
        const int comp = (int)(cp % 3);
        const u64* d = X + (c * 4 + comp) * (size_t)LK * N + k;
        u64 r[NS];
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            const u64 qi = eQB.src_q[i];
            const ulonglong2 f = twist_at(twist, i, 2, k, N);
            r[i] = shoup_lazy(d[(size_t)i * N], f.x, f.y, qi);   // [t d]_{q_i}, < 2 q_i
        }
        // r -> B (centred), then y = (t d - r) / Q in B
        u64 y[KS];
        {
            uint32_t r0[NS], r1[NS];
            int vv = 0;
            bool fast = false;
            if constexpr (FAST) fast = fast_prep<NS, KS>(r, eQB, fq, r0, r1, vv);
            u64 v[NS];
            bool neg = false;
            if (!fast) neg = garner<NS>(r, eQB, v);
#pragma unroll
            for (int j = 0; j < KS; ++j) {
                const u64 bj = bq[j];
                const int pj = NS + (nP - 1 - NS - KS) + j;                      // prime index of b_j
                const ulonglong2 f = twist_at(twist, pj, 2, k, N);
                const u64 td = shoup_lazy(d[(size_t)(NS + j) * N], f.x, f.y, bj);   // [t d]_{b_j}, < 2 b_j
                u64 rb;
                if constexpr (FAST)
                    rb = fast ? fast_eval3<NS, KS>(r0, r1, vv, eQB, fq, j) : ext_eval<NS, false>(v, neg, eQB, j);
                else rb = ext_eval<NS, false>(v, neg, eQB, j);
                y[j] = shoup_lazy(td + bj - rb, Qinv_b[j], Qinv_b[KS + j], bj);  // (t d - r) / Q, < 2 b_j
            }
        }
        // y -> Q (centred)
        u64* o = C3 + cp * (size_t)NS * N + k;
        if constexpr (FAST) {
            uint32_t y0[KS], y1[KS];
            int vy = 0;
            if (fast_prep<KS, NS>(y, eBQ, fb, y0, y1, vy)) {
#pragma unroll
                for (int i = 0; i < NS; ++i) o[(size_t)i * N] = fast_eval3<KS, NS>(y0, y1, vy, eBQ, fb, i);
                continue;
            }
        }
        u64 w[KS];
        const bool negy = garner<KS>(y, eBQ, w);
#pragma unroll
        for (int i = 0; i < NS; ++i) o[(size_t)i * N] = ext_eval<KS, false>(w, negy, eBQ, i);
    }
}

// Scale-and-round in two passes (fast path, 10 or more data primes, where the one-pass kernel needs more than
// 128 registers and runs one CTA per SM), so that each pass holds one extension's digits in registers:
// pass A writes y = (t d - r) / Q over B (words below 2 b_j) to Yt [n][3][KS][N]; pass B extends y to Q.
// Measured at N = 32768, L = 16: mul_relin +10.6%, squarings +12.1%; at L = 8 the one-pass kernel is 1% faster.
template <int NS, int KS>
__global__ void __launch_bounds__(256, 2) k_scale_a(const u64* X, u64* Yt, int n, ExtDesc eQB, const u64* twist, int nP,
                                                    const u64* Qinv_b, const u64* bq, int N, FastTab<NS, KS> fq) {
    const size_t total = (size_t)n * 3 * N;
    constexpr int LK = NS + KS;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(idx % N);
        const size_t cp = idx / N;
        const size_t c = cp / 3;
        const int comp = (int)(cp % 3);
        const u64* d = X + (c * 4 + comp) * (size_t)LK * N + k;
        u64* yo = Yt + cp * (size_t)KS * N + k;
        uint32_t r0[NS], r1[NS];
        int vv = 0;
        bool fast;
        {
            u64 r[NS];
#pragma unroll
            for (int i = 0; i < NS; ++i) {
                const ulonglong2 f = twist_at(twist, i, 2, k, N);
                r[i] = shoup_lazy(d[(size_t)i * N], f.x, f.y, eQB.src_q[i]);
            }
            fast = fast_prep<NS, KS>(r, eQB, fq, r0, r1, vv);
        }
        if (!fast) {
            // the exact mixed-radix path near the rounding boundary (rare): recompute r from memory
            u64 r[NS], v[NS];
#pragma unroll
            for (int i = 0; i < NS; ++i) {
                const ulonglong2 f = twist_at(twist, i, 2, k, N);
                r[i] = shoup_lazy(d[(size_t)i * N], f.x, f.y, eQB.src_q[i]);
            }
            const bool neg = garner<NS>(r, eQB, v);
            for (int j = 0; j < KS; ++j) {
                const u64 bj = bq[j];
                const int pj = NS + (nP - 1 - NS - KS) + j;
                const ulonglong2 f = twist_at(twist, pj, 2, k, N);
                const u64 td = shoup_lazy(d[(size_t)(NS + j) * N], f.x, f.y, bj);
                const u64 rb = ext_eval<NS, false>(v, neg, eQB, j);
                yo[(size_t)j * N] = shoup_lazy(td + bj - rb, Qinv_b[j], Qinv_b[KS + j], bj);
            }
            continue;
        }
#pragma unroll 1
        for (int j = 0; j < KS; ++j) {
            const u64 bj = bq[j];
            const int pj = NS + (nP - 1 - NS - KS) + j;
            const ulonglong2 f = twist_at(twist, pj, 2, k, N);
            const u64 td = shoup_lazy(d[(size_t)(NS + j) * N], f.x, f.y, bj);
            const u64 rb = fast_eval3<NS, KS>(r0, r1, vv, eQB, fq, j);
            yo[(size_t)j * N] = shoup_lazy(td + bj - rb, Qinv_b[j], Qinv_b[KS + j], bj);
        }
    }
}

template <int NS, int KS>
__global__ void __launch_bounds__(256, 2) k_scale_b(const u64* Yt, u64* C3, int n, ExtDesc eBQ, int N,
                                                    FastTab<KS, NS> fb) {
    const size_t total = (size_t)n * 3 * N;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(idx % N);
        const size_t cp = idx / N;
        const u64* yi = Yt + cp * (size_t)KS * N + k;
        u64 y[KS];
#pragma unroll
        for (int j = 0; j < KS; ++j) y[j] = yi[(size_t)j * N];
        u64* o = C3 + cp * (size_t)NS * N + k;
        uint32_t y0[KS], y1[KS];
        int vy = 0;
        if (fast_prep<KS, NS>(y, eBQ, fb, y0, y1, vy)) {
#pragma unroll
            for (int i = 0; i < NS; ++i) o[(size_t)i * N] = fast_eval3<KS, NS>(y0, y1, vy, eBQ, fb, i);
            continue;
        }
        u64 w[KS];
        const bool negy = garner<KS>(y, eBQ, w);
#pragma unroll
        for (int i = 0; i < NS; ++i) o[(size_t)i * N] = ext_eval<KS, false>(w, negy, eBQ, i);
    }
}

// out[c][comp] = C3[c][comp] + round(W / P) mod Q, W over Q u P (coefficient form, untwisted: each word is
// first multiplied by the twist N^-1 psi^-k R that the inverse transform left out)
template <int NA>
__global__ void k_moddown(const u64* W, const u64* C3, u64* out, int n, int L, ExtDesc ePQ, const u64* Pinv,
                          const u64* qtab, const u64* twist, int N) {
    // two consecutive coefficients per thread (N is even, every limb starts 16-byte aligned): 16-byte accesses
    const size_t half = (size_t)N >> 1;
    const size_t total = (size_t)n * 2 * half;
    const int QP = L + NA;
    const ulonglong2* tw2 = reinterpret_cast<const ulonglong2*>(twist);
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(idx % half) * 2;
        const size_t cp = idx / half;
        const size_t c = cp >> 1;
        const int comp = (int)(cp & 1);
        const u64* w = W + cp * (size_t)QP * N + k;
        u64 x0[NA], x1[NA], v0[NA], v1[NA];
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            const ulonglong2 ww = *reinterpret_cast<const ulonglong2*>(w + (size_t)(L + a) * N);
            const ulonglong2* f = tw2 + ((size_t)(L + a) * 3 + 1) * N + k;
            const ulonglong2 f0 = __ldg(f), f1 = __ldg(f + 1);
            x0[a] = shoup_lazy(ww.x, f0.x, f0.y, ePQ.src_q[a]);   // < 2 p_a
            x1[a] = shoup_lazy(ww.y, f1.x, f1.y, ePQ.src_q[a]);
        }
        const bool neg0 = garner<NA>(x0, ePQ, v0), neg1 = garner<NA>(x1, ePQ, v1);
        const u64* cin = C3 + (c * 3 + comp) * (size_t)L * N + k;
        u64* o = out + cp * (size_t)L * N + k;
        for (int i = 0; i < L; ++i) {
            const u64 qi = qtab[i], pw = Pinv[i], pws = Pinv[L + i];
            const ulonglong2* f = tw2 + ((size_t)i * 3 + 1) * N + k;
            const ulonglong2 f0 = __ldg(f), f1 = __ldg(f + 1);
            const ulonglong2 ww = *reinterpret_cast<const ulonglong2*>(w + (size_t)i * N);
            const ulonglong2 cc = *reinterpret_cast<const ulonglong2*>(cin + (size_t)i * N);
            const u64 w0 = shoup_lazy(ww.x, f0.x, f0.y, qi), w1 = shoup_lazy(ww.y, f1.x, f1.y, qi);   // < 2 q_i
            const u64 y0 = shoup(sub_mod(w0, ext_eval<NA, false>(v0, neg0, ePQ, i), qi), pw, pws, qi);
            const u64 y1 = shoup(sub_mod(w1, ext_eval<NA, false>(v1, neg1, ePQ, i), qi), pw, pws, qi);
            *reinterpret_cast<ulonglong2*>(o + (size_t)i * N) = make_ulonglong2(add_mod(cc.x, y0, qi), add_mod(cc.y, y1, qi));
        }
    }
}

// decrypt: m = [-r Q^-1]_t with r the centred [t (c0 + c1 s)]_Q
template <int NS>
__global__ void k_dec_finish(const u64* V, const u64* ct, u64* M, int n, ExtDesc eQt, const u64* tmod, int nP,
                             u64 Qinv_t, int N, uint32_t* flags) {
    const size_t total = (size_t)n * N;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(idx % N);
        const size_t c = idx / N;
        u64 r[NS], v[NS];
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            const u64 qi = eQt.src_q[i];
            const u64 c0 = ct[(c * 2 * NS + i) * N + k];
            if (c0 >= qi) atomicOr(flags, BFHE_FLAG_RESIDUE);
            const u64 vi = add_mod(V[(c * NS + i) * N + k], c0, qi);
            r[i] = shoup(vi, tmod[i], tmod[nP + i], qi);
        }
        const bool neg = garner<NS>(r, eQt, v);
        const u64 t = eQt.dst_q[0];
        const u64 rho = ext_eval<NS, true>(v, neg, eQt, 0);        // [r]_t
        const u64 mneg = rho == 0 ? 0 : t - rho;
        M[idx] = (mneg * Qinv_t) % t;
    }
}

// ---------------------------------------------------------------- more than 16 data primes
// The insecure test-only parameter sets with 17..BFHE_MAX_L data primes run the same exact arithmetic with
// sizes known only at run time (digits in local memory, loops not unrolled), so that they need no template
// instance per size; the guarded fast extension is not offered there.
constexpr int NMAX = BFHE_MAX_L + 1;

__device__ bool garner_n(const u64* x, const ExtDesc& d, u64* v, int ns) {
#pragma unroll 1
    for (int i = 0; i < ns; ++i) {
        const u64 si = d.src_q[i];
        u64 u = x[i];
#pragma unroll 1
        for (int j = 0; j < i; ++j) {
            u64 vj = v[j];
            vj = vj >= si ? vj - si : vj;
            u = shoup_lazy(u + si - vj, d.ginv[i * ns + j], d.ginv_s[i * ns + j], si);
        }
        v[i] = u >= si ? u - si : u;
    }
    int state = 0;
#pragma unroll 1
    for (int i = ns - 1; i >= 0 && state == 0; --i) {
        const u64 h = d.hdig[i];
        state = v[i] > h ? 1 : (v[i] < h ? -1 : 0);
    }
    return state > 0;
}

__device__ u64 ext_eval_n(const u64* v, bool neg, const ExtDesc& d, int j, int ns, bool small) {
    const u64 T = d.dst_q[j];
    u64 acc;
    if (small) {
        const u64 mu = d.dst_mu[j];
        acc = reduce64(v[ns - 1], T, mu);
#pragma unroll 1
        for (int i = ns - 2; i >= 0; --i) {
            acc = shoup(acc, d.radix[j * ns + i], d.radix_s[j * ns + i], T);
            acc = add_mod(acc, reduce64(v[i], T, mu), T);
        }
    } else {
        acc = v[ns - 1];
#pragma unroll 1
        for (int i = ns - 2; i >= 0; --i) acc = shoup_lazy(acc, d.radix[j * ns + i], d.radix_s[j * ns + i], T) + v[i];
        const u64 T2 = T << 1;
        acc = acc >= T2 ? acc - T2 : acc;
        acc = acc >= T ? acc - T : acc;
    }
    if (neg) acc = sub_mod(acc, d.smod[j], T);
    return acc;
}

__global__ void k_modup_n(const u64* A, const u64* B, u64* X, int n, int slots, int K, ExtDesc ext, int N,
                          uint32_t* flags) {
    const int ns = ext.n_src;
    const size_t total = (size_t)n * slots * N;
    const int LK = ns + K;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(idx % N);
        const size_t pp = idx / N;
        const size_t c = pp / slots;
        const int slot = (int)(pp % slots);
        const u64* src = (slot < 2 ? A : B) + (c * 2 + (slot & 1)) * (size_t)ns * N + k;
        u64* dst = X + (c * 4 + slot) * (size_t)LK * N + k;
        u64 x[NMAX], v[NMAX];
        bool bad = false;
        for (int i = 0; i < ns; ++i) {
            x[i] = src[(size_t)i * N];
            dst[(size_t)i * N] = x[i];
            bad |= x[i] >= ext.src_q[i];
        }
        if (bad) atomicOr(flags, BFHE_FLAG_RESIDUE);
        const bool neg = garner_n(x, ext, v, ns);
        for (int j = 0; j < K; ++j) dst[(size_t)(ns + j) * N] = ext_eval_n(v, neg, ext, j, ns, false);
    }
}

__global__ void k_scale_n(const u64* X, u64* C3, int n, ExtDesc eQB, ExtDesc eBQ, const u64* twist, int nP,
                          const u64* Qinv_b, const u64* bq, int N) {
    const int ns = eQB.n_src, ks = eBQ.n_src, LK = ns + ks;
    const size_t total = (size_t)n * 3 * N;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(idx % N);
        const size_t cp = idx / N;
        const size_t c = cp / 3;
        const int comp = (int)(cp % 3);
        const u64* d = X + (c * 4 + comp) * (size_t)LK * N + k;
        u64 r[NMAX], v[NMAX], y[NMAX];
        for (int i = 0; i < ns; ++i) {
            const ulonglong2 f = twist_at(twist, i, 2, k, N);
            r[i] = shoup_lazy(d[(size_t)i * N], f.x, f.y, eQB.src_q[i]);
        }
        const bool neg = garner_n(r, eQB, v, ns);
        for (int j = 0; j < ks; ++j) {
            const u64 bj = bq[j];
            const int pj = ns + (nP - 1 - ns - ks) + j;
            const ulonglong2 f = twist_at(twist, pj, 2, k, N);
            const u64 td = shoup_lazy(d[(size_t)(ns + j) * N], f.x, f.y, bj);
            const u64 rb = ext_eval_n(v, neg, eQB, j, ns, false);
            y[j] = shoup_lazy(td + bj - rb, Qinv_b[j], Qinv_b[ks + j], bj);
        }
        const bool negy = garner_n(y, eBQ, v, ks);
        u64* o = C3 + cp * (size_t)ns * N + k;
        for (int i = 0; i < ns; ++i) o[(size_t)i * N] = ext_eval_n(v, negy, eBQ, i, ks, false);
    }
}

__global__ void k_dec_finish_n(const u64* V, const u64* ct, u64* M, int n, ExtDesc eQt, const u64* tmod, int nP,
                               u64 Qinv_t, int N, uint32_t* flags) {
    const int ns = eQt.n_src;
    const size_t total = (size_t)n * N;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(idx % N);
        const size_t c = idx / N;
        u64 r[NMAX], v[NMAX];
        for (int i = 0; i < ns; ++i) {
            const u64 qi = eQt.src_q[i];
            const u64 c0 = ct[(c * 2 * ns + i) * N + k];
            if (c0 >= qi) atomicOr(flags, BFHE_FLAG_RESIDUE);
            r[i] = shoup(add_mod(V[(c * ns + i) * N + k], c0, qi), tmod[i], tmod[nP + i], qi);
        }
        const bool neg = garner_n(r, eQt, v, ns);
        const u64 t = eQt.dst_q[0];
        const u64 rho = ext_eval_n(v, neg, eQt, 0, ns, true);
        const u64 mneg = rho == 0 ? 0 : t - rho;
        M[idx] = (mneg * Qinv_t) % t;
    }
}

}  // namespace

// ================================================================== launchers
#define LAUNCH(kern, work, ...)                                                   \
    do {                                                                          \
        auto* _kfn = kern;                                                        \
        _kfn<<<grid_for(work), TPB, 0, st>>>(__VA_ARGS__);                       \
        BFHE_LAUNCH_CHECK(#kern);                                                \
    } while (0)

template <int NS>
int run_modup(const bfhe_ctx* ctx, const u64* A, const u64* B, u64* X, int n, int slots, cudaStream_t st) {
    const size_t work = (size_t)n * slots * ctx->N;
    if (ctx->fast_ext && ctx->ext_QB.fast_ok && (int)ctx->K == NS + 1)
        LAUNCH((k_modup<NS, true>), work, A, B, X, n, slots, (int)ctx->K, ctx->ext_QB, (int)ctx->N, ctx->d_flags,
               fast_tab<NS, NS + 1>(ctx->exth_QB));
    else
        LAUNCH((k_modup<NS, false>), work, A, B, X, n, slots, (int)ctx->K, ctx->ext_QB, (int)ctx->N, ctx->d_flags,
               FastTab<1, 1>{});
    return BFHE_OK;
}

template <int NS>
int run_scale(const bfhe_ctx* ctx, const u64* X, u64* C3, int n, cudaStream_t st, u64* tmp) {
    const size_t work = (size_t)n * 3 * ctx->N;
    const u64* bq = ctx->tab.q + ctx->L + ctx->alpha;
    const bool fast = ctx->fast_ext && ctx->ext_QB.fast_ok && ctx->ext_BQ.fast_ok;
    if constexpr (NS >= 10) {
        if (tmp && fast) {
            LAUNCH((k_scale_a<NS, NS + 1>), work, X, tmp, n, ctx->ext_QB, ctx->tab.twist, (int)ctx->nP,
                   ctx->d_Qinv_b, bq, (int)ctx->N, fast_tab<NS, NS + 1>(ctx->exth_QB));
            LAUNCH((k_scale_b<NS, NS + 1>), work, tmp, C3, n, ctx->ext_BQ, (int)ctx->N,
                   fast_tab<NS + 1, NS>(ctx->exth_BQ));
            return BFHE_OK;
        }
    }
    if (fast)
        LAUNCH((k_scale<NS, NS + 1, true>), work, X, C3, n, ctx->ext_QB, ctx->ext_BQ, ctx->tab.twist, (int)ctx->nP,
               ctx->d_Qinv_b, bq, (int)ctx->N, fast_tab<NS, NS + 1>(ctx->exth_QB), fast_tab<NS + 1, NS>(ctx->exth_BQ));
    else
        LAUNCH((k_scale<NS, NS + 1, false>), work, X, C3, n, ctx->ext_QB, ctx->ext_BQ, ctx->tab.twist, (int)ctx->nP,
               ctx->d_Qinv_b, bq, (int)ctx->N, FastTab<1, 1>{}, FastTab<1, 1>{});
    return BFHE_OK;
}

template <int NS>
int run_dec_finish(const bfhe_ctx* ctx, const u64* V, const u64* ct, u64* M, int n, cudaStream_t st) {
    const size_t work = (size_t)n * ctx->N;
    LAUNCH(k_dec_finish<NS>, work, V, ct, M, n, ctx->ext_Qt, ctx->d_tmod, (int)ctx->nP, ctx->Qinv_t, (int)ctx->N,
           ctx->d_flags);
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

int launch_modup(const bfhe_ctx* ctx, const u64* A, const u64* B, u64* X, int n, int slots, cudaStream_t st) {
    const double L_ = ctx->L, K_ = ctx->K;
    // L limbs read, L + K written per coefficient of each input poly
    ProfScope ps(ctx, BFHE_K_MODUP, st, (double)slots * n * ctx->N * (L_ * (L_ - 1) / 2 + K_ * (L_ - 1)),
                 8.0 * slots * n * ctx->N * (2 * L_ + K_));
    SWITCH_L(ctx->L, run_modup, ctx, A, B, X, n, slots, st)
    if (ctx->L > BFHE_MAX_L) return set_error(BFHE_EINVAL, "unsupported number of data primes");
    LAUNCH(k_modup_n, (size_t)n * slots * ctx->N, A, B, X, n, slots, (int)ctx->K, ctx->ext_QB, (int)ctx->N,
           ctx->d_flags);
    return BFHE_OK;
}

int launch_scale(const bfhe_ctx* ctx, const u64* X, u64* C3, int n, cudaStream_t st, u64* tmp) {
    if (ctx->K != ctx->L + 1) return set_error(BFHE_EINVAL, "auxiliary base must have L+1 primes");
    const double L_ = ctx->L, K_ = ctx->K;
    // per coefficient of each of 3 polys: L + K limbs read, L written
    ProfScope ps(ctx, BFHE_K_SCALE, st,
                 3.0 * n * ctx->N * (2 * L_ + 3 * K_ + L_ * (L_ - 1) / 2 + K_ * (L_ - 1) + K_ * (K_ - 1) / 2 + L_ * (K_ - 1)),
                 24.0 * n * ctx->N * (2 * L_ + K_));
    SWITCH_L(ctx->L, run_scale, ctx, X, C3, n, st, tmp)
    if (ctx->L > BFHE_MAX_L) return set_error(BFHE_EINVAL, "unsupported number of data primes");
    LAUNCH(k_scale_n, (size_t)n * 3 * ctx->N, X, C3, n, ctx->ext_QB, ctx->ext_BQ, ctx->tab.twist, (int)ctx->nP,
           ctx->d_Qinv_b, ctx->tab.q + ctx->L + ctx->alpha, (int)ctx->N);
    return BFHE_OK;
}

int launch_moddown(const bfhe_ctx* ctx, const u64* W, const u64* C3, u64* out, int n, cudaStream_t st) {
    const double A_ = ctx->alpha;
    // work: the rounding division by P, plus the twist the inverse transform left to this kernel
    // per coefficient of each of 2 polys: L + alpha words of W and L of C3 read, L written
    ProfScope ps(ctx, BFHE_K_MODDOWN, st, 2.0 * n * ctx->N * (A_ * (A_ - 1) / 2 + ctx->L * A_ + ctx->L + A_),
                 16.0 * n * ctx->N * (3.0 * ctx->L + A_));
    const size_t work = (size_t)n * ctx->N;   // two coefficients per thread
    if (ctx->alpha == 1)
        LAUNCH(k_moddown<1>, work, W, C3, out, n, (int)ctx->L, ctx->ext_PQ, ctx->d_Pinv_q, ctx->tab.q, ctx->tab.twist,
               (int)ctx->N);
    else if (ctx->alpha == 2)
        LAUNCH(k_moddown<2>, work, W, C3, out, n, (int)ctx->L, ctx->ext_PQ, ctx->d_Pinv_q, ctx->tab.q, ctx->tab.twist,
               (int)ctx->N);
    else
        return set_error(BFHE_EINVAL, "alpha must be 1 or 2");
    return BFHE_OK;
}

int launch_dec_finish(const bfhe_ctx* ctx, const u64* V, const u64* ct, u64* M, int n, cudaStream_t st) {
    SWITCH_L(ctx->L, run_dec_finish, ctx, V, ct, M, n, st)
    if (ctx->L > BFHE_MAX_L) return set_error(BFHE_EINVAL, "unsupported number of data primes");
    LAUNCH(k_dec_finish_n, (size_t)n * ctx->N, V, ct, M, n, ctx->ext_Qt, ctx->d_tmod, (int)ctx->nP, ctx->Qinv_t,
           (int)ctx->N, ctx->d_flags);
    return BFHE_OK;
}

