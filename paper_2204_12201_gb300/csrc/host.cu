// host.cu -- parameter rule, constant tables, context lifetime, scratch and errors.
//
// The moduli follow one rule (the paper fixes n, t and the security level
// and lets SEAL choose the rest, Sec. 4.1): primes q = 1 (mod 2N) below
// 2^prime_bits from one downward scan over q = 2N k + 1 (k decreasing,
// skipping t), tested by deterministic Miller-Rabin with the first twelve
// prime bases; the first L are the data primes, the next alpha the special
// primes, the next K the auxiliary base, K the least count with B > 2 t N Q.
// The slot root is zeta = g^((t-1)/2N) mod t with g the least primitive root
// of t (the encode/decode NTT uses psi = zeta, so slot j = m(zeta^(2j+1))).
#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>

#include "common.cuh"

namespace {

thread_local std::string g_last_error;
std::atomic<uint64_t> g_launches{0};

u64 mulmod(u64 a, u64 b, u64 m) { return (u64)((u128)a * b % m); }

u64 powmod(u64 a, u64 e, u64 m) {
    u64 r = 1 % m;
    a %= m;
    while (e) {
        if (e & 1) r = mulmod(r, a, m);
        a = mulmod(a, a, m);
        e >>= 1;
    }
    return r;
}

bool is_prime(u64 n) {
    static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (u64 p : bases)
        if (n % p == 0) return n == p;
    u64 d = n - 1;
    int r = 0;
    while ((d & 1) == 0) {
        d >>= 1;
        ++r;
    }
    for (u64 a : bases) {
        u64 x = powmod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int i = 0; i < r - 1; ++i) {
            x = mulmod(x, x, n);
            if (x == n - 1) {
                comp = false;
                break;
            }
        }
        if (comp) return false;
    }
    return true;
}

u64 invmod(u64 a, u64 p) { return powmod(a % p, p - 2, p); }   // p prime

u64 shoup_of(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

u64 least_primitive_root(u64 p) {
    std::vector<u64> fs;
    u64 n = p - 1;
    for (u64 d = 2; d * d <= n; d += (d == 2 ? 1 : 2)) {
        if (n % d == 0) {
            fs.push_back(d);
            while (n % d == 0) n /= d;
        }
    }
    if (n > 1) fs.push_back(n);
    for (u64 g = 2;; ++g) {
        bool ok = true;
        for (u64 f : fs)
            if (powmod(g, (p - 1) / f, p) == 1) {
                ok = false;
                break;
            }
        if (ok) return g;
    }
}

// a primitive 2N-th root of unity mod q (any one serves the NTT)
u64 root_2n(u64 q, uint32_t N) {
    for (u64 g = 2;; ++g) {
        u64 psi = powmod(g, (q - 1) / (2 * (u64)N), q);
        if (powmod(psi, N, q) == q - 1) return psi;
    }
}

std::vector<u64> scan_primes(uint32_t N, int count, uint32_t bits, u64 skip) {
    std::vector<u64> out;
    const u64 step = 2 * (u64)N;
    u64 k = (((u64)1 << bits) - 2) / step;
    while ((int)out.size() < count && k > 0) {
        const u64 q = step * k + 1;
        if (q != skip && is_prime(q)) out.push_back(q);
        --k;
    }
    return out;
}

// Garner digits of the integer with residues x (same formula as the device)
std::vector<u64> garner_host(const std::vector<u64>& x, const std::vector<u64>& s) {
    const size_t n = s.size();
    std::vector<u64> v(n);
    for (size_t i = 0; i < n; ++i) {
        u64 u = x[i] % s[i];
        for (size_t j = 0; j < i; ++j) {
            u64 vj = v[j] % s[i];
            u = (u + s[i] - vj) % s[i];
            u = mulmod(u, invmod(s[j] % s[i], s[i]), s[i]);
        }
        v[i] = u;
    }
    return v;
}

// host staging of the constant arena
struct Arena {
    std::vector<u64> words;
    size_t add(const std::vector<u64>& v) {
        size_t off = words.size();
        words.insert(words.end(), v.begin(), v.end());
        // keep 16-byte alignment of every table
        if (words.size() & 1) words.push_back(0);
        return off;
    }
};

struct ExtOffsets {
    int n, m, fast_ok;
    size_t src_q, ginv, ginv_s, hdig, dst_q, dst_mu, radix, radix_s, smod;
    size_t qhinv, qhinv_s, g_hi, g_lo, c26, dst_qinv, vS;
};

ExtOffsets build_ext(Arena& ar, const std::vector<u64>& src, const std::vector<u64>& dst, ExtHost* host = nullptr) {
    const int n = (int)src.size(), m = (int)dst.size();
    std::vector<u64> ginv(n * n, 0), ginv_s(n * n, 0), hres(n), radix(m * n), radix_s(m * n), smod(m), mu(m);
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < i; ++j) {
            const u64 w = invmod(src[j] % src[i], src[i]);
            ginv[i * n + j] = w;
            ginv_s[i * n + j] = shoup_of(w, src[i]);
        }
        hres[i] = (src[i] - 1) / 2;   // (S-1)/2 = -1/2 mod s_i
    }
    const std::vector<u64> hdig = garner_host(hres, src);
    for (int j = 0; j < m; ++j) {
        u64 prod = 1 % dst[j];
        for (int i = 0; i < n; ++i) {
            const u64 w = src[i] % dst[j];
            radix[j * n + i] = w;
            radix_s[j * n + i] = shoup_of(w, dst[j]);
            prod = mulmod(prod, w, dst[j]);
        }
        smod[j] = prod;
        mu[j] = (u64)(((u128)1 << 64) / dst[j]);
    }
    // guarded fast path tables
    bool fast_ok = true;
    for (u64 v : src) fast_ok = fast_ok && v < ((u64)1 << 50);
    for (u64 v : dst) fast_ok = fast_ok && v < ((u64)1 << 50);
    std::vector<u64> qhinv(n), qhinv_s(n), g_hi(n), g_lo(n), dqinv(m), vS((size_t)m * (n + 1));
    std::vector<u64> c26w(((size_t)m * n * 2 + 1) / 2 + 1, 0);   // uint32 pairs packed in u64 words
    uint32_t* c26 = reinterpret_cast<uint32_t*>(c26w.data());
    for (int i = 0; i < n; ++i) {
        u64 qh = 1;   // (S / s_i) mod s_i
        for (int k = 0; k < n; ++k)
            if (k != i) qh = mulmod(qh, src[k] % src[i], src[i]);
        qhinv[i] = invmod(qh, src[i]);
        qhinv_s[i] = shoup_of(qhinv[i], src[i]);
        const u128 g = (~(u128)0) / src[i];   // floor(2^128 / s) for s not a power of two
        g_hi[i] = (u64)(g >> 64);
        g_lo[i] = (u64)g;
    }
    for (int j = 0; j < m; ++j) {
        const u64 T = dst[j];
        u64 x = T;   // Newton: T * x = 1 mod 2^64
        for (int it = 0; it < 6; ++it) x *= 2 - T * x;
        dqinv[j] = (u64)0 - x;
        const u64 R = (u64)(((u128)1 << 64) % T);
        u64 S_T = 1 % T;
        for (int k = 0; k < n; ++k) S_T = mulmod(S_T, src[k] % T, T);
        for (int v = 0; v <= n; ++v) vS[(size_t)j * (n + 1) + v] = mulmod((u64)v % T, S_T, T);
        for (int i = 0; i < n; ++i) {
            u64 qh = 1 % T;   // (S / s_i) mod T
            for (int k = 0; k < n; ++k)
                if (k != i) qh = mulmod(qh, src[k] % T, T);
            const u64 cv = mulmod(qh, R, T);
            c26[((size_t)j * n + i) * 2 + 0] = (uint32_t)(cv & 0x3FFFFFFull);
            c26[((size_t)j * n + i) * 2 + 1] = (uint32_t)(cv >> 26);
        }
    }
    if (host) {
        host->n = n;
        host->m = m;
        host->c26.assign(c26, c26 + (size_t)m * n * 2);
        host->qhinv = qhinv;
        host->qhinv_s = qhinv_s;
        host->g_hi = g_hi;
        host->g_lo = g_lo;
    }
    ExtOffsets o;
    o.n = n;
    o.m = m;
    o.fast_ok = fast_ok ? 1 : 0;
    o.qhinv = ar.add(qhinv);
    o.qhinv_s = ar.add(qhinv_s);
    o.g_hi = ar.add(g_hi);
    o.g_lo = ar.add(g_lo);
    o.c26 = ar.add(c26w);
    o.dst_qinv = ar.add(dqinv);
    o.vS = ar.add(vS);
    o.src_q = ar.add(src);
    o.ginv = ar.add(ginv);
    o.ginv_s = ar.add(ginv_s);
    o.hdig = ar.add(hdig);
    o.dst_q = ar.add(dst);
    o.dst_mu = ar.add(mu);
    o.radix = ar.add(radix);
    o.radix_s = ar.add(radix_s);
    o.smod = ar.add(smod);
    return o;
}

ExtDesc ext_ptrs(const u64* base, const ExtOffsets& o) {
    ExtDesc d;
    d.n_src = o.n;
    d.n_dst = o.m;
    d.src_q = base + o.src_q;
    d.ginv = base + o.ginv;
    d.ginv_s = base + o.ginv_s;
    d.hdig = base + o.hdig;
    d.dst_q = base + o.dst_q;
    d.dst_mu = base + o.dst_mu;
    d.radix = base + o.radix;
    d.radix_s = base + o.radix_s;
    d.smod = base + o.smod;
    d.qhinv = base + o.qhinv;
    d.qhinv_s = base + o.qhinv_s;
    d.g_hi = base + o.g_hi;
    d.g_lo = base + o.g_lo;
    d.c26 = reinterpret_cast<const uint32_t*>(base + o.c26);
    d.dst_qinv = base + o.dst_qinv;
    d.vS = base + o.vS;
    d.fast_ok = o.fast_ok;
    return d;
}

std::vector<u64> pair_table(const std::vector<u64>& w, const std::vector<u64>& q) {
    std::vector<u64> out(2 * w.size());
    for (size_t i = 0; i < w.size(); ++i) {
        out[i] = w[i];
        out[w.size() + i] = shoup_of(w[i], q[i]);
    }
    return out;
}

}  // namespace

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

extern "C" uint64_t bfhe_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

// ------------------------------------------------------------------ errors
int set_error(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

int cuda_check(cudaError_t e, const char* where) {
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? BFHE_ENOMEM : BFHE_ECUDA;
}

extern "C" const char* bfhe_last_error(void) { return g_last_error.c_str(); }

extern "C" const char* bfhe_strerror(int code) {
    switch (code) {
        case BFHE_OK: return "ok";
        case BFHE_EINVAL: return "invalid argument";
        case BFHE_ENOMEM: return "out of device memory";
        case BFHE_ECUDA: return "CUDA error";
        case BFHE_ETIMEOUT: return "device wait timed out";
        case BFHE_ESTATE: return "call out of order";
        default: return "unknown error";
    }
}

// ------------------------------------------------------------------ launch timing
static cudaEvent_t take_event(const bfhe_ctx* c) {
    if (!c->prof_pool.empty()) {
        cudaEvent_t e = c->prof_pool.back();
        c->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

ProfScope::ProfScope(const bfhe_ctx* ctx, int k, cudaStream_t s, double w, double by)
    : c(ctx), cls(k), work(w), bytes(by), st(s) {
    if (!c->prof_on || c->capturing) return;
    a = take_event(c);
    b = take_event(c);
    if (a && b) cudaEventRecord(a, st);
}

ProfScope::~ProfScope() {
    if (!a || !b) return;
    cudaEventRecord(b, st);
    c->prof_pending.push_back(bfhe_ctx::ProfRec{cls, work, bytes, a, b});
}

extern "C" int bfhe_profile(bfhe_ctx* ctx, int enable) {
    if (!ctx) return set_error(BFHE_EINVAL, "null context");
    ctx->prof_on = enable != 0;
    return BFHE_OK;
}

extern "C" int bfhe_profile_read(bfhe_ctx* ctx, double* ms_out, uint64_t* launches_out, double* work_out,
                                 double* bytes_out) {
    if (!ctx || !ms_out || !launches_out) return set_error(BFHE_EINVAL, "null argument");
    for (int k = 0; k < BFHE_K_COUNT; ++k) {
        ms_out[k] = 0;
        launches_out[k] = 0;
        if (work_out) work_out[k] = 0;
        if (bytes_out) bytes_out[k] = 0;
    }
    int rc = BFHE_OK;
    for (auto& r : ctx->prof_pending) {
        float ms = 0;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess) rc = cuda_check(e, "profile events");
        if (r.cls >= 0 && r.cls < BFHE_K_COUNT) {
            ms_out[r.cls] += ms;
            launches_out[r.cls] += 1;
            if (work_out) work_out[r.cls] += r.work;
            if (bytes_out) bytes_out[r.cls] += r.bytes;
        }
        ctx->prof_pool.push_back(r.a);
        ctx->prof_pool.push_back(r.b);
    }
    ctx->prof_pending.clear();
    return rc;
}

// ------------------------------------------------------------------ scratch
size_t mul_scratch_bytes(const bfhe_ctx* ctx, size_t n) {
    const size_t L = ctx->L, K = ctx->K, QP = ctx->L + ctx->alpha, N = ctx->N;
    return n * (4 * (L + K) + 3 * L + L * QP + 2 * QP) * N * sizeof(u64);
}

int ctx_scratch(bfhe_ctx* ctx, size_t bytes, void** out) {
    if (bytes <= ctx->scratch_bytes) {
        *out = ctx->scratch;
        return BFHE_OK;
    }
    BFHE_CUDA(cudaSetDevice(ctx->device));
    BFHE_CUDA(cudaDeviceSynchronize());
    if (ctx->scratch) BFHE_CUDA(cudaFree(ctx->scratch));
    ctx->scratch = nullptr;
    ctx->scratch_bytes = 0;
    const size_t want = (bytes + 255) & ~(size_t)255;
    cudaError_t e = cudaMalloc(&ctx->scratch, want);
    if (e != cudaSuccess) {
        ctx->scratch = nullptr;
        return cuda_check(e, "scratch cudaMalloc");
    }
    ctx->scratch_bytes = want;
    *out = ctx->scratch;
    return BFHE_OK;
}

// ------------------------------------------------------------------ context
// The parameter rule (validation, moduli, auxiliary base size) on the host alone.
struct ParamRule {
    uint32_t N, logN, L, alpha, bits, K;
    u64 t;
    bool batching;
    std::vector<u64> moduli;   // data, special, auxiliary (not t)
};

static int param_rule(const bfhe_params* prm, ParamRule* r) {
    if (!prm) return set_error(BFHE_EINVAL, "null argument");
    const uint32_t N = prm->N;
    if (N < 1024 || N > 32768 || (N & (N - 1))) return set_error(BFHE_EINVAL, "N must be a power of two in [1024, 32768]");
    if (prm->L < 1 || prm->L > BFHE_MAX_L) return set_error(BFHE_EINVAL, "L must be in [1, 32]");
    if (prm->alpha < 1 || prm->alpha > BFHE_MAX_ALPHA) return set_error(BFHE_EINVAL, "alpha must be 1 or 2");
    const uint32_t bits = prm->prime_bits ? prm->prime_bits : 50;
    if (bits < 30 || bits > 58) return set_error(BFHE_EINVAL, "prime_bits must be in [30, 58]");   // NTT bound 64q <= 2^64
    const u64 t = prm->t;
    const bool batching = t != 2;
    if (batching && (t < 3 || t >= ((u64)1 << 32) || !is_prime(t) || (t - 1) % (2 * (u64)N) != 0))
        return set_error(BFHE_EINVAL, "t must be 2 or a prime < 2^32 with t = 1 mod 2N");
    r->N = N;
    r->logN = 0;
    while ((1u << r->logN) < N) ++r->logN;
    r->L = prm->L;
    r->alpha = prm->alpha;
    r->bits = bits;
    r->t = t;
    r->batching = batching;

    // primes: data, special, then grow the auxiliary base until B > 2 t N Q (B, Q as exact logs)
    const int head = (int)(r->L + r->alpha);
    std::vector<u64> all = scan_primes(N, head + 64, bits, t);
    if ((int)all.size() < head + 2) return set_error(BFHE_EINVAL, "not enough NTT-friendly primes");
    // compare B > 2 t N Q with big integers held as little-endian 32-bit limbs
    auto mul_small = [](std::vector<uint32_t>& a, u64 m) {
        u128 carry = 0;
        for (auto& w : a) {
            u128 v = (u128)w * m + carry;
            w = (uint32_t)v;
            carry = v >> 32;
        }
        while (carry) {
            a.push_back((uint32_t)carry);
            carry >>= 32;
        }
    };
    auto greater = [](const std::vector<uint32_t>& a, const std::vector<uint32_t>& b) {
        size_t na = a.size(), nb = b.size();
        while (na && a[na - 1] == 0) --na;
        while (nb && b[nb - 1] == 0) --nb;
        if (na != nb) return na > nb;
        for (size_t i = na; i-- > 0;)
            if (a[i] != b[i]) return a[i] > b[i];
        return false;
    };
    std::vector<uint32_t> rhs{1};
    for (uint32_t i = 0; i < r->L; ++i) mul_small(rhs, all[i]);
    mul_small(rhs, 2 * t);
    mul_small(rhs, N);
    std::vector<uint32_t> B{1};
    int K = 0;
    while (!greater(B, rhs)) {
        if (head + K >= (int)all.size()) return set_error(BFHE_EINVAL, "auxiliary base too large");
        mul_small(B, all[head + K]);
        ++K;
    }
    r->K = (uint32_t)K;
    if (r->K != r->L + 1) return set_error(BFHE_EINVAL, "parameter rule gives K != L + 1 (unsupported)");
    for (int i = 0; i < head + K; ++i)
        if (all[i] < ((u64)1 << (bits - 1))) return set_error(BFHE_EINVAL, "a modulus fell below 2^(prime_bits-1)");
    r->moduli.assign(all.begin(), all.begin() + head + K);
    return BFHE_OK;
}

extern "C" int bfhe_param_primes(const bfhe_params* prm, uint64_t* primes_out, uint32_t* K_out) {
    if (!primes_out || !K_out) return set_error(BFHE_EINVAL, "null argument");
    ParamRule r;
    const int rc = param_rule(prm, &r);
    if (rc != BFHE_OK) return rc;
    for (size_t i = 0; i < r.moduli.size(); ++i) primes_out[i] = r.moduli[i];
    *K_out = r.K;
    return BFHE_OK;
}

extern "C" int bfhe_ctx_create(const bfhe_params* prm, int device, bfhe_ctx** out) {
    if (!prm || !out) return set_error(BFHE_EINVAL, "null argument");
    *out = nullptr;
    ParamRule rule;
    const int prc = param_rule(prm, &rule);
    if (prc != BFHE_OK) return prc;
    const uint32_t N = rule.N;
    const uint32_t bits = rule.bits;
    const u64 t = rule.t;
    const bool batching = rule.batching;

    bfhe_ctx* c = new bfhe_ctx();
    c->device = device;
    c->N = N;
    c->logN = rule.logN;
    c->L = rule.L;
    c->alpha = rule.alpha;
    c->prime_bits = bits;
    c->t = t;
    c->batching = batching;
    const int K = (int)rule.K;
    c->K = rule.K;
    c->primes = rule.moduli;
    c->primes.push_back(t);
    c->nP = (uint32_t)c->primes.size();
    const uint32_t L = c->L, A = c->alpha, nP = c->nP;

    // bit reversal
    c->brv.resize(N);
    for (uint32_t k = 0; k < N; ++k) {
        uint32_t r = 0;
        for (uint32_t b = 0; b < c->logN; ++b)
            if (k & (1u << b)) r |= 1u << (c->logN - 1 - b);
        c->brv[k] = r;
    }

    // per-prime tables
    Arena ar;
    std::vector<u64> qv(c->primes), qinv(nP), mu(nP), R2(nP);
    std::vector<u64> tw((size_t)nP * N * 2), itw((size_t)nP * N * 2), twist((size_t)nP * 3 * N * 2);
    std::vector<u64> twl((size_t)nP * 3 * N * 2);
    for (uint32_t p = 0; p < nP; ++p) {
        const u64 q = c->primes[p];
        if (p == nP - 1 && !batching) {
            // t = 2: no slot transform; its table rows stay zero and are never read
            mu[p] = (u64)(((u128)1 << 64) / q);
            continue;
        }
        u64 x = q;   // Newton: q * x = 1 mod 2^64
        for (int it = 0; it < 6; ++it) x *= 2 - q * x;
        qinv[p] = (u64)0 - x;
        mu[p] = (u64)(((u128)1 << 64) / q);
        const u64 R = (u64)(((u128)1 << 64) % q);
        R2[p] = mulmod(R, R, q);
        const u64 psi = (p == nP - 1) ? powmod(least_primitive_root(q), (q - 1) / (2 * (u64)N), q) : root_2n(q, N);
        const u64 ipsi = invmod(psi, q);
        // powers psi^k and psi^-k, k < 2N
        std::vector<u64> pw(2 * N), ipw(2 * N);
        pw[0] = ipw[0] = 1;
        for (uint32_t k = 1; k < 2 * N; ++k) {
            pw[k] = mulmod(pw[k - 1], psi, q);
            ipw[k] = mulmod(ipw[k - 1], ipsi, q);
        }
        // forward: psi^brv(k)
        for (uint32_t k = 0; k < N; ++k) {
            const size_t o = ((size_t)p * N + k) * 2;
            tw[o] = pw[c->brv[k]];
            tw[o + 1] = shoup_of(tw[o], q);
        }
        // the forward's last pass (E = 2^le words per thread, stages on bits b < le): the entries of stage b,
        // [N >> (b+1), N >> b), regrouped so that lanes of a warp read consecutive entries: thread tg's g-th
        // twiddle (standard entry (N >> (b+1)) + tg B + g, B = E >> (b+1)) at (N >> (b+1)) + g (N / E) + tg
        for (uint32_t le = 3; le <= 5; ++le) {
            const size_t o = ((size_t)p * 3 + (le - 3)) * N * 2;
            const size_t ot = (size_t)p * N * 2;
            for (uint32_t k = 0; k < (N >> le); ++k) {
                twl[o + 2 * k] = tw[ot + 2 * k];
                twl[o + 2 * k + 1] = tw[ot + 2 * k + 1];
            }
            const uint32_t T = N >> le;
            for (uint32_t b = 0; b < le; ++b) {
                const uint32_t lo = N >> (b + 1), B = (1u << le) >> (b + 1);
                for (uint32_t r = 0; r < lo; ++r) {
                    const uint32_t d = lo + (r % B) * T + r / B;
                    twl[o + 2 * (size_t)d] = tw[ot + 2 * (size_t)(lo + r)];
                    twl[o + 2 * (size_t)d + 1] = tw[ot + 2 * (size_t)(lo + r) + 1];
                }
            }
        }
        // inverse DIT: entry 2^b + j (j < 2^b) = omega^-((N >> (b+1)) j) = psi^-(2 (N >> (b+1)) j)
        itw[(size_t)p * N * 2] = 1;
        itw[(size_t)p * N * 2 + 1] = shoup_of(1, q);
        for (uint32_t b = 0; (1u << b) < N; ++b) {
            for (uint32_t j = 0; j < (1u << b); ++j) {
                const size_t o = ((size_t)p * N + (1u << b) + j) * 2;
                const u64 e = (2ull * (N >> (b + 1)) * j) % (2ull * N);
                itw[o] = ipw[e];
                itw[o + 1] = shoup_of(itw[o], q);
            }
        }
        // twist N^-1 psi^-m: plain, times R, and times t R (scale-and-round takes the multiply's inverse
        // transforms untwisted and folds the twist into its own product by t)
        const u64 ninv = invmod(N % q, q), tq = t % q;
        for (uint32_t m = 0; m < N; ++m) {
            const u64 v0 = mulmod(ninv, ipw[m], q), v1 = mulmod(v0, R, q), v2 = mulmod(v1, tq, q);
            const u64 vs[3] = {v0, v1, v2};
            for (int f = 0; f < 3; ++f) {
                const size_t o = (((size_t)p * 3 + f) * N + m) * 2;
                twist[o] = vs[f];
                twist[o + 1] = shoup_of(vs[f], q);
            }
        }
    }
    const size_t o_q = ar.add(qv), o_qinv = ar.add(qinv), o_mu = ar.add(mu), o_R2 = ar.add(R2);
    const size_t o_tw = ar.add(tw), o_twl = ar.add(twl), o_itw = ar.add(itw), o_twist = ar.add(twist);
    std::vector<u64> brv_packed((N + 1) / 2);
    for (uint32_t k = 0; k < N; k += 2)
        brv_packed[k / 2] = (u64)c->brv[k] | ((u64)(k + 1 < N ? c->brv[k + 1] : 0) << 32);
    const size_t o_brv = ar.add(brv_packed);

    // base extensions
    std::vector<u64> Qp(c->primes.begin(), c->primes.begin() + L);
    std::vector<u64> Pp(c->primes.begin() + L, c->primes.begin() + L + A);
    std::vector<u64> Bp(c->primes.begin() + L + A, c->primes.begin() + L + A + K);
    std::vector<u64> Tp{t};
    const ExtOffsets eQB = build_ext(ar, Qp, Bp, &c->exth_QB), eBQ = build_ext(ar, Bp, Qp, &c->exth_BQ),
                     ePQ = build_ext(ar, Pp, Qp), eQt = build_ext(ar, Qp, Tp);

    // scalar constants
    u64 Qt = 1;
    for (u64 q : Qp) Qt = mulmod(Qt, q % t, t);
    c->Qinv_t = invmod(Qt, t);
    std::vector<u64> tmod(nP), delta(L), Qinv_b(K), Pinv_q(L), P_q(L);
    for (uint32_t p = 0; p < nP; ++p) tmod[p] = t % c->primes[p];
    for (uint32_t i = 0; i < L; ++i) {
        const u64 q = Qp[i];
        delta[i] = mulmod((q - Qt % q) % q, invmod(t % q, q), q);   // -[Q]_t t^-1 mod q_i
        u64 pm = 1;
        for (u64 pp : Pp) pm = mulmod(pm, pp % q, q);
        P_q[i] = pm;
        Pinv_q[i] = invmod(pm, q);
    }
    for (int j = 0; j < K; ++j) {
        u64 qm = 1;
        for (u64 q : Qp) qm = mulmod(qm, q % Bp[j], Bp[j]);
        Qinv_b[j] = invmod(qm, Bp[j]);
    }
    const size_t o_tmod = ar.add(pair_table(tmod, c->primes));
    const size_t o_delta = ar.add(pair_table(delta, Qp));
    const size_t o_Qinvb = ar.add(pair_table(Qinv_b, Bp));
    const size_t o_Pinvq = ar.add(pair_table(Pinv_q, Qp));
    const size_t o_Pq = ar.add(pair_table(P_q, Qp));

    // upload
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_arena, ar.words.size() * sizeof(u64));
    if (e == cudaSuccess)
        e = cudaMemcpy(c->d_arena, ar.words.data(), ar.words.size() * sizeof(u64), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        int rc = cuda_check(e, "context tables");
        if (c->d_arena) cudaFree(c->d_arena);
        delete c;
        return rc;
    }
    cudaError_t fe = cudaMalloc(&c->d_flags, 256);
    if (fe == cudaSuccess) fe = cudaMemset(c->d_flags, 0, 256);
    if (fe != cudaSuccess) {
        int rc = cuda_check(fe, "context flags");
        cudaFree(c->d_arena);
        if (c->d_flags) cudaFree(c->d_flags);
        delete c;
        return rc;
    }
    c->arena_bytes = ar.words.size() * sizeof(u64);
    const u64* base = (const u64*)c->d_arena;
    c->tab.q = base + o_q;
    c->tab.qinv = base + o_qinv;
    c->tab.mu = base + o_mu;
    c->tab.tw = base + o_tw;
    c->tab.twl = base + o_twl;
    c->tab.itw = base + o_itw;
    c->tab.twist = base + o_twist;
    c->d_R2 = base + o_R2;
    c->d_brv = (uint32_t*)(base + o_brv);
    c->ext_QB = ext_ptrs(base, eQB);
    c->ext_BQ = ext_ptrs(base, eBQ);
    c->ext_PQ = ext_ptrs(base, ePQ);
    c->ext_Qt = ext_ptrs(base, eQt);
    // the guarded fast extension measures faster from 8 data primes up (slower at 2)
    c->fast_ext = c->L >= 8 && c->L <= BFHE_MAX_L_UNROLLED && c->ext_QB.fast_ok && c->ext_BQ.fast_ok;
    c->d_tmod = base + o_tmod;
    c->d_delta_q = base + o_delta;
    c->d_Qinv_b = base + o_Qinvb;
    c->d_Pinv_q = base + o_Pinvq;
    c->d_P_q = base + o_Pq;
    *out = c;
    return BFHE_OK;
}

extern "C" void bfhe_ctx_destroy(bfhe_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    cudaFree(ctx->d_arena);
    cudaFree(ctx->d_flags);
    cudaFree(ctx->scratch);
    cudaFree(ctx->d_sk);
    cudaFree(ctx->d_sk_ntt);
    cudaFree(ctx->d_pk);
    cudaFree(ctx->d_pk_ntt);
    cudaFree(ctx->d_rlk_ntt);
    for (auto& r : ctx->prof_pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : ctx->prof_pool) cudaEventDestroy(e);
    if (ctx->tile_exec) cudaGraphExecDestroy(ctx->tile_exec);
    if (ctx->cap_in) cudaEventDestroy(ctx->cap_in);
    if (ctx->cap_out) cudaEventDestroy(ctx->cap_out);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    cudaFree(ctx->d_cbase);
    delete ctx;
}

extern "C" int bfhe_ctx_device_bytes(const bfhe_ctx* ctx, size_t* out) {
    if (!ctx || !out) return set_error(BFHE_EINVAL, "null argument");
    const size_t N = ctx->N, L = ctx->L, QP = ctx->L + ctx->alpha;
    out[0] = ctx->arena_bytes + 256;   // tables and the flag word
    out[1] = ctx->d_sk ? (N + QP * N + 4 * L * N + 2 * L * QP * N) * sizeof(u64) : 0;
    out[2] = ctx->scratch_bytes;
    out[3] = ctx->d_cbase ? sizeof(u64) : 0;
    return BFHE_OK;
}

extern "C" size_t bfhe_mul_scratch_bytes(const bfhe_ctx* ctx, size_t n) { return ctx ? mul_scratch_bytes(ctx, n) : 0; }

extern "C" int bfhe_ctx_primes(const bfhe_ctx* ctx, uint64_t* primes_out, uint32_t* K_out) {
    if (!ctx || !primes_out) return set_error(BFHE_EINVAL, "null argument");
    for (uint32_t i = 0; i + 1 < ctx->nP; ++i) primes_out[i] = ctx->primes[i];
    if (K_out) *K_out = ctx->K;
    return BFHE_OK;
}

extern "C" int bfhe_op_counts(bfhe_ctx* ctx, uint64_t out[4], int reset) {
    if (!ctx || !out) return set_error(BFHE_EINVAL, "null argument");
    for (int i = 0; i < 4; ++i) out[i] = ctx->counts[i];
    if (reset)
        for (int i = 0; i < 4; ++i) ctx->counts[i] = 0;
    return BFHE_OK;
}
