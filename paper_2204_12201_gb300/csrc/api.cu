// api.cu -- the C ABI (include/bfhe.h): validation, scratch layout and kernel sequencing.
#include <algorithm>
#include <mutex>
#include <string>

#include "kernels.cuh"

namespace {

// Philox purposes (key word 1)
enum : u64 { P_SK = 1, P_PK_A = 2, P_PK_E = 3, P_RLK_A = 4, P_RLK_E = 5, P_ENC_U = 6, P_ENC_E1 = 7, P_ENC_E2 = 8 };

inline cudaStream_t S(void* s) { return (cudaStream_t)s; }

// device-memory budget for one call's scratch (batches beyond it are tiled)
size_t g_scratch_budget = (size_t)16 << 30;

#define CHECK_CTX(ctx)                                                     \
    do {                                                                   \
        if (!(ctx)) return set_error(BFHE_EINVAL, "null context");         \
    } while (0)
#define CHECK_KEYS(ctx)                                                    \
    do {                                                                   \
        if (!(ctx)->have_keys) return set_error(BFHE_ESTATE, "no keys: call bfhe_keygen first"); \
    } while (0)
#define RC(x)                                \
    do {                                     \
        int _rc = (x);                       \
        if (_rc != BFHE_OK) return _rc;      \
    } while (0)

size_t mul_words_per_ct(const bfhe_ctx* c) { return mul_scratch_bytes(c, 1) / sizeof(u64); }

// most ciphertexts per multiply launch sequence, per log2 N (0: as many as the scratch holds); set by the
// autotuner through bfhe_set_mul_tile
size_t g_mul_tile[16] = {};

// out[i] = a[i] * b[i] (relinearised), n ciphertexts, scratch of `scratch_words` words
int mul_relin_impl(bfhe_ctx* c, const u64* A, const u64* B, u64* out, size_t n, u64* scratch,
                   size_t scratch_words, cudaStream_t st) {
    const size_t N = c->N, L = c->L, K = c->K, LK = L + K, QP = L + c->alpha;
    const size_t per = mul_words_per_ct(c);
    size_t tile = scratch_words / per;
    if (tile == 0) return set_error(BFHE_ENOMEM, "scratch too small for one multiply");
    if (c->logN < 16 && g_mul_tile[c->logN] && g_mul_tile[c->logN] < tile) tile = g_mul_tile[c->logN];
    const size_t ctw = c->ct_words();
    for (size_t c0 = 0; c0 < n; c0 += tile) {
        const int m = (int)std::min(tile, n - c0);
        u64* X = scratch;                                  // [m][4][LK][N]
        u64* C3 = X + (size_t)m * 4 * LK * N;              // [m][3][L][N]
        u64* Dg = C3 + (size_t)m * 3 * L * N;              // [m][L][QP][N]
        u64* W = Dg + (size_t)m * L * QP * N;              // [m][2][QP][N]
        const u64* a = A + c0 * ctw;
        const u64* b = B + c0 * ctw;
        u64* o = out + c0 * ctw;
        // a squaring (a == b) extends and transforms a0, a1 only; the tensor sums are the same
        const int sq = (A == B) ? 1 : 0;
        const int slots = sq ? 2 : 4;
        RC(launch_modup(c, a, b, X, m, slots, st));
        NttIO iox;
        iox.in = X;
        iox.out = X;
        iox.n_inner = slots;
        iox.in_os = iox.out_os = 4 * LK * N;
        iox.in_is = iox.out_is = LK * N;
        iox.in_ls = iox.out_ls = N;
        RC(launch_ntt_fwd(c, iox, slots * m, (int)LK, c->mapQB(), st, 1));   // tensor takes lazy words
        RC(launch_tensor(c, X, m, sq, st));
        NttIO io3;
        io3.in = X;
        io3.out = X;
        io3.n_inner = 3;
        io3.in_os = io3.out_os = 4 * LK * N;
        io3.in_is = io3.out_is = LK * N;
        io3.in_ls = io3.out_ls = N;
        RC(launch_ntt_inv(c, io3, 3 * m, (int)LK, c->mapQB(), 1, st, 2));   // scale applies the twist
        // scale's intermediate y [m][3][K][N] (two-pass form) lives in the digit buffer, dead until the digit
        // transforms
        RC(launch_scale(c, X, C3, m, st, (L * QP >= 3 * K) ? Dg : nullptr));
        NttIO iod;   // digit j of c2 (limb j of C3 slot 2), reduced into every prime of Q u P
        iod.in = C3 + 2 * L * N;
        iod.out = Dg;
        iod.n_inner = (int)L;
        iod.in_os = 3 * L * N;
        iod.in_is = N;
        iod.in_ls = 0;
        iod.out_os = L * QP * N;
        iod.out_is = QP * N;
        iod.out_ls = N;
        RC(launch_ntt_fwd(c, iod, m * (int)L, (int)QP, c->mapQP(), st, 1));   // so does the inner product
        RC(launch_inner(c, Dg, W, m, st));
        RC(launch_ntt_inv(c, ntt_io(W, W, QP, N), 2 * m, (int)QP, c->mapQP(), 1, st, 2));   // so does mod-down
        RC(launch_moddown(c, W, C3, o, m, st));
    }
    return BFHE_OK;
}

// multiply-scratch words granted to a call that keeps `fixed_words` and multiplies n_mul ciphertexts
size_t mul_words_for(const bfhe_ctx* c, size_t fixed_words, size_t n_mul) {
    const size_t per = mul_words_per_ct(c);
    size_t budget_words = g_scratch_budget / sizeof(u64);
    size_t want_mul = n_mul * per;
    if (fixed_words + want_mul > budget_words) {
        const size_t room = budget_words > fixed_words ? budget_words - fixed_words : 0;
        want_mul = std::max(per, (room / per) * per);
    }
    return n_mul == 0 ? 0 : want_mul;
}

int scratch_for(bfhe_ctx* c, size_t fixed_words, size_t n_mul, u64** fixed, u64** mul, size_t* mul_words) {
    const size_t want_mul = mul_words_for(c, fixed_words, n_mul);
    void* p;
    RC(ctx_scratch(c, (fixed_words + want_mul) * sizeof(u64), &p));
    *fixed = (u64*)p;
    *mul = (u64*)p + fixed_words;
    *mul_words = want_mul;
    return BFHE_OK;
}

int pow_impl(bfhe_ctx* c, const u64* x, u64 e, u64* out, size_t n, u64* bufs, u64* mul, size_t mul_words,
             cudaStream_t st) {
    // Listing 7: pow(b, e) = pow(b*b, e >> 1) [* b if e odd]; unrolled: squarings b^(2^d) for
    // d = 1..top, then the odd-bit factors multiplied in from the deepest level up.
    const size_t ctw = c->ct_words();
    int top = 63 - __builtin_clzll(e);
    // bufs: [2][n] ping-pong for the squaring chain, then one slot per set bit below top
    u64* cur = bufs;
    u64* nxt = bufs + n * ctw;
    u64* saved = bufs + 2 * n * ctw;
    std::vector<std::pair<int, u64*>> keep;
    int nkeep = 0;
    const u64* base = x;
    if ((e & 1) && top > 0) {
        keep.push_back({0, (u64*)x});
    }
    for (int d = 1; d <= top; ++d) {
        RC(mul_relin_impl(c, base, base, nxt, n, mul, mul_words, st));
        c->counts[2] += n;
        std::swap(cur, nxt);
        base = cur;
        if (d < top && ((e >> d) & 1)) {
            u64* slot = saved + (size_t)nkeep * n * ctw;
            BFHE_CUDA(cudaMemcpyAsync(slot, cur, n * ctw * sizeof(u64), cudaMemcpyDeviceToDevice, st));
            keep.push_back({d, slot});
            ++nkeep;
        }
    }
    // r = b^(2^top); then r *= b^(2^d) for set bits d < top, deepest first
    const u64* r = base;
    for (int k = (int)keep.size() - 1; k >= 0; --k) {
        u64* dst = (r == cur) ? nxt : cur;
        RC(mul_relin_impl(c, r, keep[k].second, dst, n, mul, mul_words, st));
        c->counts[2] += n;
        r = dst;
    }
    if (r != out) BFHE_CUDA(cudaMemcpyAsync(out, r, n * ctw * sizeof(u64), cudaMemcpyDeviceToDevice, st));
    return BFHE_OK;
}

size_t pow_buf_words(const bfhe_ctx* c, u64 e, size_t n) {
    int pc = __builtin_popcountll(e);
    return (size_t)(2 + pc) * n * c->ct_words();
}

}  // namespace

// ------------------------------------------------------------------ ABI
extern "C" int bfhe_check(bfhe_ctx* c, void* stream, uint32_t* flags_out) {
    CHECK_CTX(c);
    uint32_t f = 0;
    BFHE_CUDA(cudaStreamSynchronize(S(stream)));
    BFHE_CUDA(cudaMemcpy(&f, c->d_flags, sizeof(f), cudaMemcpyDeviceToHost));
    BFHE_CUDA(cudaMemset(c->d_flags, 0, sizeof(f)));
    if (flags_out) *flags_out = f;
    if (f) {
        std::string m = "out-of-range input seen on the device:";
        if (f & BFHE_FLAG_PLAINTEXT) m += " a plaintext value >= t;";
        if (f & BFHE_FLAG_RESIDUE) m += " a ciphertext residue >= its prime;";
        return set_error(BFHE_EINVAL, m);
    }
    return BFHE_OK;
}

extern "C" int bfhe_set_fast_extension(bfhe_ctx* c, int on) {
    CHECK_CTX(c);
    if (on && !(c->ext_QB.fast_ok && c->ext_BQ.fast_ok))
        return set_error(BFHE_EINVAL, "the fast extension needs every modulus below 2^50");
    if (on && c->L > BFHE_MAX_L_UNROLLED)
        return set_error(BFHE_EINVAL, "the fast extension is built for at most 16 data primes");
    c->fast_ext = on != 0;
    return BFHE_OK;
}

extern "C" int bfhe_set_graph_tiles(bfhe_ctx* c, int on) {
    CHECK_CTX(c);
    c->graph_tiles = on != 0;
    return BFHE_OK;
}

extern "C" int bfhe_graph_tiles(const bfhe_ctx* c) {
    if (!c) return set_error(BFHE_EINVAL, "null context");
    return c->graph_tiles ? 1 : 0;
}

extern "C" int bfhe_fast_extension(const bfhe_ctx* c) {
    if (!c) return set_error(BFHE_EINVAL, "null context");
    return c->fast_ext ? 1 : 0;
}

extern "C" int bfhe_set_scratch_budget(size_t bytes) {
    // one multiply at the largest parameters needs far less than 1 MiB x 64; below 1 MiB nothing fits
    if (bytes < ((size_t)1 << 20)) return set_error(BFHE_EINVAL, "scratch budget below 1 MiB");
    g_scratch_budget = bytes;
    return BFHE_OK;
}

extern "C" size_t bfhe_scratch_budget(void) { return g_scratch_budget; }

extern "C" int bfhe_set_mul_tile(uint32_t logN, size_t max_ct) {
    if (logN < 10 || logN > 15) return set_error(BFHE_EINVAL, "logN must be in [10, 15]");
    g_mul_tile[logN] = max_ct;
    return BFHE_OK;
}

extern "C" size_t bfhe_mul_tile(uint32_t logN) { return logN < 16 ? g_mul_tile[logN] : 0; }

extern "C" int bfhe_reserve(bfhe_ctx* c, size_t n) {
    CHECK_CTX(c);
    void* p;
    return ctx_scratch(c, std::min(mul_scratch_bytes(c, n) + 8 * n * c->ct_words() * sizeof(u64), g_scratch_budget), &p);
}

extern "C" int bfhe_keygen(bfhe_ctx* c, uint64_t seed, void* stream) {
    CHECK_CTX(c);
    const size_t N = c->N, L = c->L, QP = c->L + c->alpha;
    cudaStream_t st = S(stream);
    BFHE_CUDA(cudaSetDevice(c->device));
    if (!c->d_sk) {
        BFHE_CUDA(cudaMalloc(&c->d_sk, N * sizeof(i64)));
        BFHE_CUDA(cudaMalloc(&c->d_sk_ntt, QP * N * sizeof(u64)));
        BFHE_CUDA(cudaMalloc(&c->d_pk, 2 * L * N * sizeof(u64)));
        BFHE_CUDA(cudaMalloc(&c->d_pk_ntt, 2 * L * N * sizeof(u64)));
        BFHE_CUDA(cudaMalloc(&c->d_rlk_ntt, L * 2 * QP * N * sizeof(u64)));
    }
    // scratch: A[L][N], AS[L][N], e[N], S2[QP][N], ASj[L][QP][N], Bj[L][QP][N], ej[L][N]
    const size_t words = 2 * L * N + N + QP * N + 2 * L * QP * N + L * N;
    void* p;
    RC(ctx_scratch(c, words * sizeof(u64), &p));
    u64* A = (u64*)p;
    u64* AS = A + L * N;
    i64* e = (i64*)(AS + L * N);
    u64* S2 = (u64*)(e + N);
    u64* ASj = S2 + QP * N;
    u64* Bj = ASj + L * QP * N;
    i64* ej = (i64*)(Bj + L * QP * N);

    // secret key, ternary, and its NTT over Q u P
    RC(launch_sample_small(c, c->d_sk, 1, seed, P_SK, 0, 0, st));
    RC(launch_spread(c, c->d_sk, c->d_sk_ntt, 1, (int)QP, c->mapQP(), st));
    RC(launch_ntt_fwd(c, ntt_io(c->d_sk_ntt, c->d_sk_ntt, QP, N), 1, (int)QP, c->mapQP(), st));
    // pk = (-(a s + e), a)
    RC(launch_sample_uniform(c, A, 1, (int)L, c->mapQ(), seed, P_PK_A, 0, st));
    BFHE_CUDA(cudaMemcpyAsync(c->d_pk + L * N, A, L * N * sizeof(u64), cudaMemcpyDeviceToDevice, st));
    RC(launch_ntt_fwd(c, ntt_io(A, A, L, N), 1, (int)L, c->mapQ(), st));
    PwStrides s1{0, 0, 0, 0, 0, 0};
    RC(launch_pointwise(c, A, c->d_sk_ntt, AS, 1, 1, (int)L, c->mapQ(), s1, st));
    RC(launch_ntt_inv(c, ntt_io(AS, AS, L, N), 1, (int)L, c->mapQ(), 1, st));
    RC(launch_sample_small(c, e, 1, seed, P_PK_E, 0, 1, st));
    RC(launch_neg_add_small(c, AS, e, c->d_pk, 1, (int)L, c->mapQ(), nullptr, 0, st));
    RC(launch_ntt_fwd(c, ntt_io(c->d_pk, c->d_pk_ntt, L, N), 2, (int)L, c->mapQ(), st));
    // s^2 over Q u P (coefficient form)
    RC(launch_pointwise(c, c->d_sk_ntt, c->d_sk_ntt, S2, 1, 1, (int)QP, c->mapQP(), s1, st));
    RC(launch_ntt_inv(c, ntt_io(S2, S2, QP, N), 1, (int)QP, c->mapQP(), 1, st));
    // relinearisation keys: a_j uniform over Q u P, NTT straight into rlk[j][1]
    u64* Araw = Bj;   // staging for the raw a_j before NTT
    RC(launch_sample_uniform(c, Araw, (int)L, (int)QP, c->mapQP(), seed, P_RLK_A, 0, st));
    NttIO ioa;
    ioa.in = Araw;
    ioa.out = c->d_rlk_ntt + QP * N;
    ioa.n_inner = 1;
    ioa.in_os = QP * N;
    ioa.in_is = 0;
    ioa.in_ls = N;
    ioa.out_os = 2 * QP * N;
    ioa.out_is = 0;
    ioa.out_ls = N;
    RC(launch_ntt_fwd(c, ioa, (int)L, (int)QP, c->mapQP(), st));
    PwStrides s2{2 * QP * N, 0, 0, 0, QP * N, 0};
    RC(launch_pointwise(c, c->d_rlk_ntt + QP * N, c->d_sk_ntt, ASj, (int)L, 1, (int)QP, c->mapQP(), s2, st));
    RC(launch_ntt_inv(c, ntt_io(ASj, ASj, QP, N), (int)L, (int)QP, c->mapQP(), 1, st));
    RC(launch_sample_small(c, ej, (int)L, seed, P_RLK_E, 0, 1, st));
    RC(launch_neg_add_small(c, ASj, ej, Bj, (int)L, (int)QP, c->mapQP(), S2, 1, st));
    NttIO iob = ioa;
    iob.in = Bj;
    iob.out = c->d_rlk_ntt;
    RC(launch_ntt_fwd(c, iob, (int)L, (int)QP, c->mapQP(), st));
    c->have_keys = true;
    return BFHE_OK;
}

extern "C" int bfhe_export_keys(bfhe_ctx* c, int64_t* sk, uint64_t* pk, uint64_t* rlk, void* stream) {
    CHECK_CTX(c);
    CHECK_KEYS(c);
    const size_t N = c->N, L = c->L, QP = c->L + c->alpha;
    cudaStream_t st = S(stream);
    if (sk) BFHE_CUDA(cudaMemcpyAsync(sk, c->d_sk, N * sizeof(i64), cudaMemcpyDeviceToDevice, st));
    if (pk) BFHE_CUDA(cudaMemcpyAsync(pk, c->d_pk, 2 * L * N * sizeof(u64), cudaMemcpyDeviceToDevice, st));
    if (rlk) RC(launch_ntt_inv(c, ntt_io(c->d_rlk_ntt, rlk, QP, N), (int)(2 * L), (int)QP, c->mapQP(), 0, st));
    return BFHE_OK;
}

namespace {

// (Delta M + pk0 u + e1, pk1 u + e2) for plaintext polynomials M [n][N] (coefficients < t);
// scratch: u/e1/e2 [3][n][N], U [n][L][N]
int encrypt_core(bfhe_ctx* c, const u64* M, size_t n, uint64_t seed, u64* ct_out, u64* scratch, cudaStream_t st) {
    const size_t N = c->N, L = c->L;
    i64* u = (i64*)scratch;
    i64* e1 = u + n * N;
    i64* e2 = e1 + n * N;
    u64* U = (u64*)(e2 + n * N);
    RC(launch_sample_small(c, u, (int)n, seed, P_ENC_U, 0, 0, st));
    RC(launch_sample_small(c, e1, (int)n, seed, P_ENC_E1, 0, 1, st));
    RC(launch_sample_small(c, e2, (int)n, seed, P_ENC_E2, 0, 1, st));
    RC(launch_spread(c, u, U, (int)n, (int)L, c->mapQ(), st));
    RC(launch_ntt_fwd(c, ntt_io(U, U, L, N), (int)n, (int)L, c->mapQ(), st));
    PwStrides s{L * N, 0, 0, L * N, 2 * L * N, L * N};
    RC(launch_pointwise(c, U, c->d_pk_ntt, ct_out, (int)n, 2, (int)L, c->mapQ(), s, st));
    RC(launch_ntt_inv(c, ntt_io(ct_out, ct_out, L, N), (int)(2 * n), (int)L, c->mapQ(), 1, st));
    RC(launch_enc_finish(c, ct_out, M, e1, e2, (int)n, st));
    return BFHE_OK;
}

// M [n][N] = [round(t [c0 + c1 s]_Q / Q)]_t; scratch V [n][L][N]
int decrypt_core(bfhe_ctx* c, const u64* ct, size_t n, u64* M, u64* V, cudaStream_t st) {
    const size_t N = c->N, L = c->L;
    NttIO io;
    io.in = ct + L * N;
    io.out = V;
    io.n_inner = 1;
    io.in_os = 2 * L * N;
    io.in_is = 0;
    io.in_ls = N;
    io.out_os = L * N;
    io.out_is = 0;
    io.out_ls = N;
    RC(launch_ntt_fwd(c, io, (int)n, (int)L, c->mapQ(), st));
    PwStrides s{L * N, 0, 0, 0, L * N, 0};
    RC(launch_pointwise(c, V, c->d_sk_ntt, V, (int)n, 1, (int)L, c->mapQ(), s, st));
    RC(launch_ntt_inv(c, ntt_io(V, V, L, N), (int)n, (int)L, c->mapQ(), 1, st));
    RC(launch_dec_finish(c, V, ct, M, (int)n, st));
    return BFHE_OK;
}

}  // namespace

#define CHECK_BATCHING(ctx)                                                                      \
    do {                                                                                         \
        if (!(ctx)->batching)                                                                    \
            return set_error(BFHE_EINVAL, "no slot encoding at t = 2: use the coefficient calls"); \
    } while (0)

extern "C" int bfhe_encrypt(bfhe_ctx* c, const uint64_t* slots, size_t n, uint64_t seed, uint64_t* ct_out,
                            void* stream) {
    CHECK_CTX(c);
    CHECK_KEYS(c);
    CHECK_BATCHING(c);
    if (n == 0) return BFHE_OK;
    if (!slots || !ct_out) return set_error(BFHE_EINVAL, "null buffer");
    const size_t N = c->N, L = c->L;
    cudaStream_t st = S(stream);
    // scratch: M[n][N], u/e1/e2 [3][n][N], U[n][L][N]
    void* p;
    RC(ctx_scratch(c, (4 * n * N + n * L * N) * sizeof(u64), &p));
    u64* M = (u64*)p;
    RC(launch_permute(c, slots, M, (int)n, 1, st));
    RC(launch_ntt_inv(c, ntt_io(M, M, 1, N), (int)n, 1, c->mapT(), 0, st));
    return encrypt_core(c, M, n, seed, ct_out, M + n * N, st);
}

extern "C" int bfhe_encrypt_poly(bfhe_ctx* c, const uint64_t* coeffs, size_t n, uint64_t seed, uint64_t* ct_out,
                                 void* stream) {
    CHECK_CTX(c);
    CHECK_KEYS(c);
    if (n == 0) return BFHE_OK;
    if (!coeffs || !ct_out) return set_error(BFHE_EINVAL, "null buffer");
    void* p;
    RC(ctx_scratch(c, (3 * n * c->N + n * c->L * c->N) * sizeof(u64), &p));
    return encrypt_core(c, coeffs, n, seed, ct_out, (u64*)p, S(stream));
}

extern "C" int bfhe_decrypt(bfhe_ctx* c, const uint64_t* ct, size_t n, uint64_t* slots_out, void* stream) {
    CHECK_CTX(c);
    CHECK_KEYS(c);
    CHECK_BATCHING(c);
    if (n == 0) return BFHE_OK;
    if (!ct || !slots_out) return set_error(BFHE_EINVAL, "null buffer");
    const size_t N = c->N, L = c->L;
    cudaStream_t st = S(stream);
    void* p;
    RC(ctx_scratch(c, (n * L * N + n * N) * sizeof(u64), &p));
    u64* V = (u64*)p;
    u64* M = V + n * L * N;
    RC(decrypt_core(c, ct, n, M, V, st));
    RC(launch_ntt_fwd(c, ntt_io(M, M, 1, N), (int)n, 1, c->mapT(), st));
    RC(launch_permute(c, M, slots_out, (int)n, 0, st));
    return BFHE_OK;
}

extern "C" int bfhe_decrypt_poly(bfhe_ctx* c, const uint64_t* ct, size_t n, uint64_t* coeffs_out, void* stream) {
    CHECK_CTX(c);
    CHECK_KEYS(c);
    if (n == 0) return BFHE_OK;
    if (!ct || !coeffs_out) return set_error(BFHE_EINVAL, "null buffer");
    void* p;
    RC(ctx_scratch(c, n * c->L * c->N * sizeof(u64), &p));
    return decrypt_core(c, ct, n, coeffs_out, (u64*)p, S(stream));
}

static int lin(bfhe_ctx* c, u64* out, const u64* x, const u64* y, LinCoef cf, u64 cval, size_t n, void* stream) {
    CHECK_CTX(c);
    if (n == 0) return BFHE_OK;
    if (!out || (cf.cx && !x) || (cf.cy && !y)) return set_error(BFHE_EINVAL, "null buffer");
    if (cval >= c->t) return set_error(BFHE_EINVAL, "constant must be < t");
    return launch_lincomb(c, out, x, y, nullptr, nullptr, cf, cval, n, S(stream));
}

extern "C" int bfhe_add(bfhe_ctx* c, const uint64_t* a, const uint64_t* b, uint64_t* out, size_t n, void* st) {
    RC(lin(c, out, a, b, LinCoef{0, 1, 1, 0, 0}, 0, n, st));
    c->counts[0] += n;
    return BFHE_OK;
}
extern "C" int bfhe_sub(bfhe_ctx* c, const uint64_t* a, const uint64_t* b, uint64_t* out, size_t n, void* st) {
    RC(lin(c, out, a, b, LinCoef{0, 1, -1, 0, 0}, 0, n, st));
    c->counts[1] += n;
    return BFHE_OK;
}
extern "C" int bfhe_add_const(bfhe_ctx* c, const uint64_t* a, uint64_t k, uint64_t* out, size_t n, void* st) {
    RC(lin(c, out, a, nullptr, LinCoef{1, 1, 0, 0, 0}, k, n, st));
    c->counts[0] += n;
    return BFHE_OK;
}
extern "C" int bfhe_sub_const(bfhe_ctx* c, const uint64_t* a, uint64_t k, uint64_t* out, size_t n, void* st) {
    RC(lin(c, out, a, nullptr, LinCoef{-1, 1, 0, 0, 0}, k, n, st));
    c->counts[1] += n;
    return BFHE_OK;
}
extern "C" int bfhe_const_sub(bfhe_ctx* c, uint64_t k, const uint64_t* a, uint64_t* out, size_t n, void* st) {
    RC(lin(c, out, a, nullptr, LinCoef{1, -1, 0, 0, 0}, k, n, st));
    c->counts[1] += n;
    return BFHE_OK;
}

extern "C" int bfhe_mul_scalar(bfhe_ctx* c, const uint64_t* a, uint64_t k, uint64_t* out, size_t n, void* stream) {
    CHECK_CTX(c);
    if (n == 0) return BFHE_OK;
    if (!a || !out) return set_error(BFHE_EINVAL, "null buffer");
    if (k >= c->t) return set_error(BFHE_EINVAL, "scalar must be < t");
    RC(launch_mul_scalar(c, a, k, out, n, S(stream)));
    c->counts[3] += n;
    return BFHE_OK;
}

extern "C" int bfhe_mul_plain(bfhe_ctx* c, const uint64_t* a, const uint64_t* plain, uint64_t* out, size_t n,
                              void* stream) {
    CHECK_CTX(c);
    CHECK_BATCHING(c);
    if (n == 0) return BFHE_OK;
    if (!a || !plain || !out) return set_error(BFHE_EINVAL, "null buffer");
    const size_t N = c->N, L = c->L;
    cudaStream_t st = S(stream);
    void* p;
    RC(ctx_scratch(c, (n * N + n * L * N + 2 * n * L * N) * sizeof(u64), &p));
    u64* M = (u64*)p;
    u64* PT = M + n * N;
    u64* CT = PT + n * L * N;
    RC(launch_permute(c, plain, M, (int)n, 1, st));
    RC(launch_ntt_inv(c, ntt_io(M, M, 1, N), (int)n, 1, c->mapT(), 0, st));
    RC(launch_spread(c, (const i64*)M, PT, (int)n, (int)L, c->mapQ(), st));
    RC(launch_ntt_fwd(c, ntt_io(PT, PT, L, N), (int)n, (int)L, c->mapQ(), st));
    RC(launch_ntt_fwd(c, ntt_io(a, CT, L, N), (int)(2 * n), (int)L, c->mapQ(), st));
    PwStrides s{2 * L * N, L * N, L * N, 0, 2 * L * N, L * N};
    RC(launch_pointwise(c, CT, PT, out, (int)n, 2, (int)L, c->mapQ(), s, st));
    RC(launch_ntt_inv(c, ntt_io(out, out, L, N), (int)(2 * n), (int)L, c->mapQ(), 1, st));
    c->counts[3] += n;
    return BFHE_OK;
}

extern "C" int bfhe_mul_relin(bfhe_ctx* c, const uint64_t* a, const uint64_t* b, uint64_t* out, size_t n,
                              void* stream) {
    CHECK_CTX(c);
    CHECK_KEYS(c);
    if (n == 0) return BFHE_OK;
    if (!a || !b || !out) return set_error(BFHE_EINVAL, "null buffer");
    if (out == a || out == b) return set_error(BFHE_EINVAL, "out must not alias an input");
    u64 *fixed, *mul;
    size_t mw;
    RC(scratch_for(c, 0, n, &fixed, &mul, &mw));
    RC(mul_relin_impl(c, a, b, out, n, mul, mw, S(stream)));
    c->counts[2] += n;
    return BFHE_OK;
}

static const LinCoef kGate[8] = {
    {0, 0, 0, 0, 1}, {0, 1, 1, 0, -1}, {0, 1, 1, 0, -2}, {1, 0, 0, 0, -1},
    {1, -1, -1, 0, 1}, {1, -1, -1, 0, 2}, {1, -1, 0, 0, 0}, {0, 0, 0, 1, 1},
};
// (add, sub) per gate with the gate equations written as in Sec. 3.1
static const int kGateAddSub[8][2] = {{0, 0}, {1, 1}, {2, 1}, {0, 1}, {1, 2}, {2, 2}, {0, 1}, {1, 1}};

extern "C" int bfhe_bit_gate(bfhe_ctx* c, int gate, const uint64_t* x, const uint64_t* y, const uint64_t* z,
                             uint64_t* out, size_t n, void* stream) {
    CHECK_CTX(c);
    if (gate < 0 || gate > 7) return set_error(BFHE_EINVAL, "unknown gate");
    if (n == 0) return BFHE_OK;
    if (!x || !out || (gate != BFHE_NOT && !y) || (gate == BFHE_MUX && !z))
        return set_error(BFHE_EINVAL, "null buffer");
    cudaStream_t st = S(stream);
    const size_t ctw = c->ct_words();
    if (gate == BFHE_NOT) {
        RC(launch_lincomb(c, out, x, nullptr, nullptr, nullptr, kGate[gate], 1, n, st));
    } else if (c->t == 2 && (gate == BFHE_XOR || gate == BFHE_XNOR)) {
        // mod 2 the XOR equation is x + y; XNOR = 1 - (x + y)
        const bool xnor = gate == BFHE_XNOR;
        RC(launch_lincomb(c, out, x, y, nullptr, nullptr,
                          xnor ? LinCoef{1, -1, -1, 0, 0} : LinCoef{0, 1, 1, 0, 0}, 1, n, st));
        c->counts[0] += n;
        if (xnor) c->counts[1] += n;
        return BFHE_OK;
    } else {
        CHECK_KEYS(c);
        if (out == x || out == y || out == z) return set_error(BFHE_EINVAL, "out must not alias an input");
        u64 *fixed, *mul;
        size_t mw;
        const bool mux = gate == BFHE_MUX;
        RC(scratch_for(c, (mux ? 2 : 1) * n * ctw, n, &fixed, &mul, &mw));
        u64* P = fixed;
        const u64* rhs = y;
        if (mux) {
            u64* D = fixed + n * ctw;
            RC(launch_lincomb(c, D, y, z, nullptr, nullptr, LinCoef{0, 1, -1, 0, 0}, 0, n, st));
            rhs = D;
        }
        RC(mul_relin_impl(c, x, rhs, P, n, mul, mw, st));
        RC(launch_lincomb(c, out, x, y, z, P, kGate[gate], 1, n, st));
        c->counts[2] += n;
    }
    c->counts[0] += n * kGateAddSub[gate][0];
    c->counts[1] += n * kGateAddSub[gate][1];
    return BFHE_OK;
}

extern "C" int bfhe_gate_level(bfhe_ctx* c, uint64_t* wires, size_t n_wires, size_t n, const int32_t* table,
                               size_t n_gates, size_t n_mul, void* stream) {
    CHECK_CTX(c);
    if (n == 0 || n_gates == 0) return BFHE_OK;
    if (!wires || !table || n_mul > n_gates || n_wires == 0) return set_error(BFHE_EINVAL, "bad gate level");
    cudaStream_t st = S(stream);
    const size_t ctw = n * c->ct_words();
    if (n_mul) {
        CHECK_KEYS(c);
        u64 *fixed, *mul;
        size_t mw;
        RC(scratch_for(c, 3 * n_mul * ctw, n_mul * n, &fixed, &mul, &mw));
        u64* AB = fixed;
        u64* P = fixed + 2 * n_mul * ctw;
        RC(launch_gather(c, AB, wires, n, table, (int)n_mul, 0, 0, st));
        RC(mul_relin_impl(c, AB, AB + n_mul * ctw, P, n_mul * n, mul, mw, st));
        RC(launch_gate_epilogue(c, wires, n, table, (int)n_gates, P, (int)n_mul, st));
        c->counts[2] += n_mul * n;
    } else {
        RC(launch_gate_epilogue(c, wires, n, table, (int)n_gates, nullptr, 0, st));
    }
    return BFHE_OK;
}

extern "C" int bfhe_bits_to_mod(bfhe_ctx* c, const uint64_t* bits, uint32_t s, uint64_t* out, size_t n,
                                void* stream) {
    CHECK_CTX(c);
    if (n == 0) return BFHE_OK;
    if (!bits || !out || s == 0) return set_error(BFHE_EINVAL, "bad arguments");
    RC(launch_horner(c, bits, s, out, n, S(stream)));
    c->counts[0] += (uint64_t)2 * (s - 1) * n;
    return BFHE_OK;
}

extern "C" int bfhe_pow(bfhe_ctx* c, const uint64_t* x, uint64_t e, uint64_t* out, size_t n, void* stream) {
    CHECK_CTX(c);
    CHECK_KEYS(c);
    if (n == 0) return BFHE_OK;
    if (!x || !out || e == 0) return set_error(BFHE_EINVAL, "bad arguments");
    if (out == x) return set_error(BFHE_EINVAL, "out must not alias x");
    cudaStream_t st = S(stream);
    if (e == 1) {
        BFHE_CUDA(cudaMemcpyAsync(out, x, n * c->ct_words() * sizeof(u64), cudaMemcpyDeviceToDevice, st));
        return BFHE_OK;
    }
    u64 *fixed, *mul;
    size_t mw;
    RC(scratch_for(c, pow_buf_words(c, e, n), n, &fixed, &mul, &mw));
    return pow_impl(c, x, e, out, n, fixed, mul, mw, st);
}

namespace {

// Scratch plan of one SecureMod -> SecureUint conversion: candidates per tile and the words it takes
// after `reserve` words that the caller keeps at the front of the arena.
struct M2BPlan {
    size_t C, fixed_words, n_mul;
};
M2BPlan m2b_plan(const bfhe_ctx* c, uint32_t s, size_t total, int mode, size_t n, size_t reserve) {
    const size_t ctw = c->ct_words();
    const u64 e = c->t - 1;
    // candidates per tile: chain buffers (2 + popcount(e)) + PAPER's trivial bits, eq copies and products (3s),
    // and the multiply scratch of the tile's squarings in one launch (PAPER's s ANDs per candidate then run
    // in s chunks of the same size)
    const size_t per_cand = n * ctw * (pow_buf_words(c, e, 1) / ctw + (mode == BFHE_PAPER ? 3 * s : 0) + 2);
    const size_t mul_per_cand = n * mul_words_per_ct(c);
    const size_t budget = g_scratch_budget / sizeof(u64);
    const size_t room = budget > reserve ? budget - reserve : 0;
    size_t C = room / (per_cand + mul_per_cand);
    if (C == 0) C = 1;
    if (C > total) C = total;
    return {C, reserve + C * per_cand, C * n};
}

bool m2b_args_ok(const bfhe_ctx* c, uint32_t s, u64 c_lo, u64 c_hi, int mode) {
    return s != 0 && s <= 63 && c_hi >= c_lo && c_hi < c->t && (mode == BFHE_PAPER || mode == BFHE_SELECT);
}

// One tile of Ct candidates c_base .. c_base + Ct - 1 (Eq. 2, Listings 7-8): d_c = x - c, eq_c = 1 - d_c^(t-1),
// then PAPER: s products of eq_c with the trivially encrypted bits of c, summed into the bits; SELECT: eq_c
// added to bit k when bit k of c is 1.  cbp, when not null, is a device word holding c_base (graph replay).
int m2b_tile(bfhe_ctx* c, const u64* x, uint32_t s, u64 c_base, const u64* cbp, int Ct, int mode, u64* bits_out,
             size_t n, u64* fixed, u64* mul, size_t mw, cudaStream_t st) {
    const size_t ctw = c->ct_words();
    const u64 e = c->t - 1;
    const size_t m = (size_t)Ct * n;   // chains in this tile
    u64* D = fixed;                     // [Ct][n]
    u64* bufs = D + m * ctw;            // pow buffers
    u64* EQ = bufs + pow_buf_words(c, e, m);
    RC(launch_sub_const_chains(c, x, D, c_base, cbp, Ct, n, st));
    c->counts[1] += m;
    RC(pow_impl(c, D, e, EQ, m, bufs, mul, mw, st));
    RC(launch_lincomb(c, EQ, EQ, nullptr, nullptr, nullptr, LinCoef{1, -1, 0, 0, 0}, 1, m, st));
    c->counts[1] += m;
    if (mode == BFHE_PAPER) {
        u64* TR = EQ + m * ctw;              // [s][Ct][n] trivial bits
        u64* RP = TR + (size_t)s * m * ctw;  // [s][Ct][n] copies of eq
        u64* PR = RP + (size_t)s * m * ctw;  // products
        RC(launch_trivial_bits(c, TR, s, c_base, cbp, Ct, n, st));
        for (uint32_t k = 0; k < s; ++k)
            BFHE_CUDA(cudaMemcpyAsync(RP + (size_t)k * m * ctw, EQ, m * ctw * sizeof(u64), cudaMemcpyDeviceToDevice,
                                      st));
        RC(mul_relin_impl(c, TR, RP, PR, (size_t)s * m, mul, mw, st));
        c->counts[2] += (uint64_t)s * m;
        RC(launch_accumulate(c, bits_out, PR, s, c_base, cbp, Ct, n, 0, st));
    } else {
        RC(launch_accumulate(c, bits_out, EQ, s, c_base, cbp, Ct, n, 1, st));
    }
    return BFHE_OK;
}

// Captures one full tile on the context's capture stream (candidate base read from c->d_cbase) and keeps the
// instantiated graph with its key; records the op counts and kernel launches of one tile.
int m2b_capture(bfhe_ctx* c, const std::vector<u64>& key, const u64* x, uint32_t s, int C, int mode, u64* bits_out,
                size_t n, u64* fixed, u64* mul, size_t mw) {
    cudaStream_t cs = c->cap_stream;
    if (c->tile_exec) {
        BFHE_CUDA(cudaStreamSynchronize(cs));   // the old graph may still be running
        cudaGraphExecDestroy(c->tile_exec);
        c->tile_exec = nullptr;
        c->tile_key.clear();
    }
    uint64_t counts0[4];
    for (int k = 0; k < 4; ++k) counts0[k] = c->counts[k];
    const uint64_t l0 = bfhe_launch_count();
    BFHE_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    c->capturing = true;
    const int rc = m2b_tile(c, x, s, 0, c->d_cbase, C, mode, bits_out, n, fixed, mul, mw, cs);
    c->capturing = false;
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(cs, &g);
    if (rc != BFHE_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (ec != cudaSuccess) return cuda_check(ec, "cudaStreamEndCapture (mod_to_bits tile)");
    const cudaError_t ei = cudaGraphInstantiate(&c->tile_exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        c->tile_exec = nullptr;
        return cuda_check(ei, "cudaGraphInstantiate (mod_to_bits tile)");
    }
    // the capture recorded the tile without running it: its counts are those of one tile
    for (int k = 0; k < 4; ++k) {
        c->tile_counts[k] = c->counts[k] - counts0[k];
        c->counts[k] = counts0[k];
    }
    c->tile_launches = bfhe_launch_count() - l0;
    count_launches((uint64_t)0 - c->tile_launches);
    c->tile_key = key;
    return BFHE_OK;
}

// Sec. 3.2.3, Eq. 2, Listings 7-8; the first `reserve` words of the arena are left to the caller
// (the arena must already hold them if they carry data: it is grown only when it is too small).
// With graph tiles on and at least two full tiles, the first tile runs eagerly and the other full tiles
// replay one captured tile, all on the context's capture stream (joined to `st` by events); the ragged
// last tile runs eagerly.
int mod_to_bits_impl(bfhe_ctx* c, const u64* x, uint32_t s, u64 c_lo, u64 c_hi, int mode, u64* bits_out,
                     size_t n, size_t reserve, cudaStream_t st) {
    const size_t ctw = c->ct_words();
    const size_t total = c_hi - c_lo + 1;
    const M2BPlan pl = m2b_plan(c, s, total, mode, n, reserve);
    const size_t C = pl.C;
    u64 *fixed, *mul;
    size_t mw;
    RC(scratch_for(c, pl.fixed_words, pl.n_mul, &fixed, &mul, &mw));
    fixed += reserve;
    const size_t full = total / C;
    const bool graph = c->graph_tiles && full >= 2 && !c->prof_on;
    cudaStream_t ws = st;
    if (graph) {
        if (!c->cap_stream) BFHE_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        if (!c->cap_in) BFHE_CUDA(cudaEventCreateWithFlags(&c->cap_in, cudaEventDisableTiming));
        if (!c->cap_out) BFHE_CUDA(cudaEventCreateWithFlags(&c->cap_out, cudaEventDisableTiming));
        if (!c->d_cbase) BFHE_CUDA(cudaMalloc(&c->d_cbase, sizeof(u64)));
        BFHE_CUDA(cudaEventRecord(c->cap_in, st));
        BFHE_CUDA(cudaStreamWaitEvent(c->cap_stream, c->cap_in, 0));
        ws = c->cap_stream;
    }
    BFHE_CUDA(cudaMemsetAsync(bits_out, 0, (size_t)s * n * ctw * sizeof(u64), ws));
    for (size_t cb = 0; cb < total; cb += C) {
        const int Ct = (int)std::min(C, total - cb);
        const u64 c_base = c_lo + cb;
        if (graph && cb > 0 && (size_t)Ct == C) {
            const std::vector<u64> key = {(u64)(uintptr_t)x, (u64)(uintptr_t)bits_out, (u64)(uintptr_t)fixed,
                                          (u64)(uintptr_t)mul, mw, n, s, C, (u64)mode, c->fast_ext ? 1ull : 0ull};
            if (!c->tile_exec || c->tile_key != key)
                RC(m2b_capture(c, key, x, s, (int)C, mode, bits_out, n, fixed, mul, mw));
            RC(launch_set_word(c->d_cbase, c_base, ws));
            BFHE_CUDA(cudaGraphLaunch(c->tile_exec, ws));
            for (int k = 0; k < 4; ++k) c->counts[k] += c->tile_counts[k];
            count_launches(c->tile_launches);
        } else {
            RC(m2b_tile(c, x, s, c_base, nullptr, Ct, mode, bits_out, n, fixed, mul, mw, ws));
        }
    }
    if (graph) {
        BFHE_CUDA(cudaEventRecord(c->cap_out, ws));
        BFHE_CUDA(cudaStreamWaitEvent(st, c->cap_out, 0));
    }
    // the paper's accounting of the final sums: one addition per term after the first, per bit
    for (uint32_t k = 0; k < s; ++k) {
        size_t terms = 0;
        if (mode == BFHE_PAPER) {
            terms = total;
        } else {
            for (size_t j = 0; j < total; ++j)
                if (((c_lo + j) >> k) & 1) terms += 1;
        }
        if (terms > 1) c->counts[0] += (uint64_t)(terms - 1) * n;
    }
    return BFHE_OK;
}

}  // namespace

extern "C" int bfhe_mod_to_bits(bfhe_ctx* c, const uint64_t* x, uint32_t s, uint64_t c_lo, uint64_t c_hi, int mode,
                                uint64_t* bits_out, size_t n, void* stream) {
    CHECK_CTX(c);
    CHECK_KEYS(c);
    if (n == 0) return BFHE_OK;
    if (!x || !bits_out || !m2b_args_ok(c, s, c_lo, c_hi, mode)) return set_error(BFHE_EINVAL, "bad arguments");
    return mod_to_bits_impl(c, x, s, c_lo, c_hi, mode, bits_out, n, 0, S(stream));
}

/* Sec. 3.2.2, Eq. 1, Listing 6.  One batched multiply of 2n: [isNeg; 1 - isNeg] x [neg; pos]. */
extern "C" int bfhe_sint_to_mod(bfhe_ctx* c, const uint64_t* bits, uint32_t s, uint64_t* out, size_t n,
                                void* stream) {
    CHECK_CTX(c);
    CHECK_KEYS(c);
    if (n == 0) return BFHE_OK;
    if (!bits || !out || s == 0 || s > 63 || ((u64)1 << s) > c->t)
        return set_error(BFHE_EINVAL, "bad arguments (need 1 <= s and 2^s <= t)");
    cudaStream_t st = S(stream);
    const size_t ctw = c->ct_words(), nw = n * ctw;
    u64 *fixed, *mul;
    size_t mw;
    RC(scratch_for(c, 6 * nw, 2 * n, &fixed, &mul, &mw));
    u64* A = fixed;       // [isNeg (n); 1 - isNeg (n)]
    u64* B = A + 2 * nw;  // [neg (n); pos (n)]
    u64* P = B + 2 * nw;  // the two products
    const u64* is_neg = bits + (size_t)(s - 1) * nw;
    RC(launch_horner(c, bits, s, B + nw, n, st));
    RC(launch_lincomb(c, B, B + nw, nullptr, nullptr, nullptr, LinCoef{1, 1, 0, 0, 0},
                      (c->t - ((u64)1 << s)) % c->t, n, st));
    BFHE_CUDA(cudaMemcpyAsync(A, is_neg, nw * sizeof(u64), cudaMemcpyDeviceToDevice, st));
    RC(launch_lincomb(c, A + nw, is_neg, nullptr, nullptr, nullptr, LinCoef{1, -1, 0, 0, 0}, 1, n, st));
    RC(mul_relin_impl(c, A, B, P, 2 * n, mul, mw, st));
    RC(launch_lincomb(c, out, P, P + nw, nullptr, nullptr, LinCoef{0, 1, 1, 0, 0}, 0, n, st));
    c->counts[0] += (uint64_t)(2 * (s - 1) + 2) * n;
    c->counts[1] += n;
    c->counts[2] += 2 * n;
    return BFHE_OK;
}

/* Sec. 3.2.4, Listing 9: two SecureMod -> SecureUint conversions (of x and of (2^s - t) + x) and a
 * multiplexer on the sign bit of the first, batched as one multiply of 2sn. */
extern "C" int bfhe_mod_to_sint(bfhe_ctx* c, const uint64_t* x, uint32_t s, uint64_t pos_lo, uint64_t pos_hi,
                                uint64_t neg_lo, uint64_t neg_hi, int mode, uint64_t* bits_out, size_t n,
                                void* stream) {
    CHECK_CTX(c);
    CHECK_KEYS(c);
    if (n == 0) return BFHE_OK;
    if (!x || !bits_out || !m2b_args_ok(c, s, pos_lo, pos_hi, mode) || !m2b_args_ok(c, s, neg_lo, neg_hi, mode))
        return set_error(BFHE_EINVAL, "bad arguments");
    if (((u64)1 << s) < c->t) return set_error(BFHE_EINVAL, "bad arguments (need 2^s >= t)");
    cudaStream_t st = S(stream);
    const size_t ctw = c->ct_words(), nw = n * ctw, sn = (size_t)s * n;
    // kept across the stages: BITS = [neg (s n); pos (s n)] and the shifted input (n)
    const size_t reserve = 2 * sn * ctw + nw;
    const size_t mux_fixed = reserve + 4 * sn * ctw;
    // size the arena once for the largest stage, so that no stage regrows it under kept data
    const M2BPlan p1 = m2b_plan(c, s, pos_hi - pos_lo + 1, mode, n, reserve);
    const M2BPlan p2 = m2b_plan(c, s, neg_hi - neg_lo + 1, mode, n, reserve);
    size_t need = mux_fixed + mul_words_for(c, mux_fixed, 2 * sn);
    need = std::max(need, p1.fixed_words + mul_words_for(c, p1.fixed_words, p1.n_mul));
    need = std::max(need, p2.fixed_words + mul_words_for(c, p2.fixed_words, p2.n_mul));
    void* base;
    RC(ctx_scratch(c, need * sizeof(u64), &base));
    u64* NEG = (u64*)base;
    u64* POS = NEG + sn * ctw;
    u64* XS = POS + sn * ctw;
    RC(mod_to_bits_impl(c, x, s, pos_lo, pos_hi, mode, POS, n, reserve, st));
    RC(launch_lincomb(c, XS, x, nullptr, nullptr, nullptr, LinCoef{1, 1, 0, 0, 0}, (((u64)1 << s) - c->t) % c->t,
                      n, st));
    c->counts[0] += n;
    RC(mod_to_bits_impl(c, XS, s, neg_lo, neg_hi, mode, NEG, n, reserve, st));
    u64 *fixed, *mul;
    size_t mw;
    RC(scratch_for(c, mux_fixed, 2 * sn, &fixed, &mul, &mw));
    if (fixed != (u64*)base) return set_error(BFHE_ESTATE, "scratch moved between stages");
    u64* A = fixed + reserve;   // [isNeg x s; (1 - isNeg) x s] against [neg; pos]
    u64* P = A + 2 * sn * ctw;  // products
    const u64* is_neg = POS + (size_t)(s - 1) * nw;
    RC(launch_lincomb(c, A + sn * ctw, is_neg, nullptr, nullptr, nullptr, LinCoef{1, -1, 0, 0, 0}, 1, n, st));
    c->counts[1] += n;
    for (uint32_t k = 0; k < s; ++k) {
        BFHE_CUDA(cudaMemcpyAsync(A + (size_t)k * nw, is_neg, nw * sizeof(u64), cudaMemcpyDeviceToDevice, st));
        if (k)
            BFHE_CUDA(cudaMemcpyAsync(A + (s + k) * nw, A + sn * ctw, nw * sizeof(u64), cudaMemcpyDeviceToDevice,
                                      st));
    }
    RC(mul_relin_impl(c, A, NEG, P, 2 * sn, mul, mw, st));
    c->counts[2] += 2 * sn;
    RC(launch_lincomb(c, bits_out, P, P + sn * ctw, nullptr, nullptr, LinCoef{0, 1, 1, 0, 0}, 0, sn, st));
    c->counts[0] += sn;
    return BFHE_OK;
}

extern "C" int bfhe_ntt(bfhe_ctx* c, uint64_t* data, size_t n_polys, uint32_t n_limbs, int inverse, void* stream) {
    CHECK_CTX(c);
    if (!data || n_limbs == 0 || n_limbs > c->L) return set_error(BFHE_EINVAL, "bad arguments");
    if (n_polys == 0) return BFHE_OK;
    NttIO io = ntt_io(data, data, n_limbs, c->N);
    if (inverse) return launch_ntt_inv(c, io, (int)n_polys, (int)n_limbs, c->mapQ(), 0, S(stream));
    return launch_ntt_fwd(c, io, (int)n_polys, (int)n_limbs, c->mapQ(), S(stream));
}

extern "C" int bfhe_probe_modmul(int device, uint32_t iters, double* modmul_per_s, void* stream) {
    if (!modmul_per_s || iters == 0) return set_error(BFHE_EINVAL, "bad arguments");
    BFHE_CUDA(cudaSetDevice(device));
    cudaDeviceProp prop;
    BFHE_CUDA(cudaGetDeviceProperties(&prop, device));
    const int threads = 256, blocks = prop.multiProcessorCount * 4;
    u64* buf = nullptr;
    BFHE_CUDA(cudaMalloc(&buf, (size_t)blocks * threads * sizeof(u64)));
    const u64 q = 1125899906826241ull;   // a 50-bit prime = 1 mod 2^16
    const u64 w = 123456789012345ull % q, ws = (u64)(((u128)w << 64) / q);
    cudaStream_t st = S(stream);
    cudaEvent_t e0, e1;
    BFHE_CUDA(cudaEventCreate(&e0));
    BFHE_CUDA(cudaEventCreate(&e1));
    int rc = launch_probe_modmul(buf, blocks, threads, iters / 8 + 1, q, w, ws, st);   // warm-up
    if (rc == BFHE_OK) {
        cudaEventRecord(e0, st);
        rc = launch_probe_modmul(buf, blocks, threads, iters, q, w, ws, st);
        cudaEventRecord(e1, st);
    }
    float ms = 0;
    if (rc == BFHE_OK) {
        cudaError_t e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) rc = cuda_check(e, "probe events");
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (rc == BFHE_OK) *modmul_per_s = (double)blocks * threads * 8.0 * iters / (ms * 1e-3);
    return rc;
}

// ------------------------------------------------------------------ allocation-free multiply
// Scratch for bfhe_mul_relin_noalloc: a fixed file-scope device array, so the
// call itself never allocates.  Every GPU that loads this module holds it until
// the process exits.  Host code must not pass `g_noalloc_scratch` itself to a
// kernel (in host code the name is only a stand-in for the symbol); the device
// address comes from cudaGetSymbolAddress, taken once per device.
#define BFHE_NOALLOC_WORDS ((size_t)BFHE_NOALLOC_SCRATCH_BYTES / sizeof(u64))
static __device__ __align__(256) u64 g_noalloc_scratch[BFHE_NOALLOC_WORDS];

namespace {
std::mutex g_noalloc_mu;
u64* g_noalloc_ptr[BFHE_MAX_DEVICES] = {};

// device address of the static scratch on the current device (set-up on first use)
int noalloc_scratch(int device, u64** out) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_check(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_noalloc_ptr[device] = (u64*)p;
    }
    *out = g_noalloc_ptr[device];
    return BFHE_OK;
}
}  // namespace

extern "C" int bfhe_mul_relin_noalloc(bfhe_ctx* c, const uint64_t* a, const uint64_t* b, uint64_t* out, size_t n,
                                      void* stream) {
    CHECK_CTX(c);
    CHECK_KEYS(c);
    if (n == 0) return BFHE_OK;
    if (!a || !b || !out) return set_error(BFHE_EINVAL, "null buffer");
    if (out == a || out == b) return set_error(BFHE_EINVAL, "out must not alias an input");
    int dev = -1;
    BFHE_CUDA(cudaGetDevice(&dev));
    if (dev != c->device || dev < 0 || dev >= BFHE_MAX_DEVICES)
        return set_error(BFHE_EINVAL, "the context's device must be the current device");
    const size_t per = mul_words_per_ct(c);
    const size_t max_n = BFHE_NOALLOC_WORDS / per;
    if (n > max_n) {
        return set_error(BFHE_EINVAL, "bfhe_mul_relin_noalloc: " + std::to_string(n) + " ciphertexts need " +
                                          std::to_string(n * per * sizeof(u64) >> 20) + " MiB of scratch; the static "
                                          "scratch holds " + std::to_string(BFHE_NOALLOC_SCRATCH_BYTES >> 20) +
                                          " MiB, i.e. at most " + std::to_string(max_n) +
                                          " ciphertexts per call at these parameters");
    }
    u64* scratch = nullptr;
    RC(noalloc_scratch(dev, &scratch));
    RC(mul_relin_impl(c, a, b, out, n, scratch, BFHE_NOALLOC_WORDS, S(stream)));
    c->counts[2] += n;
    return BFHE_OK;
}
