// common.cuh -- shared definitions of the bfhe CUDA library (sm_103a).
//
// Exact 64-bit modular arithmetic for RNS BFV on the integer pipe: Shoup
// products for multiplications by precomputed constants (twiddles, CRT
// constants), Montgomery reduction (REDC) for products of two runtime values
// and for lazily accumulated sums of them.  Every modulus is an odd prime
// below 2^60; the NTT keeps values lazily in [0, 4q).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/bfhe.h"

typedef uint64_t u64;
typedef int64_t i64;
typedef unsigned __int128 u128;

// up to 16 data primes every kernel has a compiled instance per size; 17..32 (insecure, test-only
// parameter sets for deep circuits) run runtime-size variants of the base extensions and the inner product
#define BFHE_MAX_L 32
#define BFHE_MAX_L_UNROLLED 16
#define BFHE_MAX_ALPHA 2
#define BFHE_MAX_PRIMES 80
#define BFHE_MAX_DEVICES 64

// ------------------------------------------------------------------ device modular arithmetic
__host__ __device__ __forceinline__ u64 mulhi64(u64 a, u64 b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (u64)(((u128)a * b) >> 64);
#endif
}

__host__ __device__ __forceinline__ u64 add_mod(u64 a, u64 b, u64 q) {
    u64 s = a + b;
    return s >= q ? s - q : s;
}

__host__ __device__ __forceinline__ u64 sub_mod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }

// a * w mod q in [0, 2q) for any a < 2^64, w < q, ws = floor(w 2^64 / q) (Shoup).
__host__ __device__ __forceinline__ u64 shoup_lazy(u64 a, u64 w, u64 ws, u64 q) {
    return a * w - mulhi64(a, ws) * q;
}

// a * w mod q in [0, 4q) for a < 2^64: the quotient estimate keeps a1 w1 and the high
// halves of the two cross products a1 w0, a0 w1 (their low halves and a0 w0 together are
// below 3 2^64), so it is floor(a ws / 2^64) minus 0, 1 or 2, and Shoup's own estimate
// is the true quotient or one less.
__host__ __device__ __forceinline__ u64 shoup_lazy4(u64 a, u64 w, u64 ws, u64 q) {
    const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32), w0 = (uint32_t)ws, w1 = (uint32_t)(ws >> 32);
    const u64 hi = (u64)a1 * w1 + (((u64)a1 * w0) >> 32) + (((u64)a0 * w1) >> 32);
    return a * w - hi * q;
}

// The same product with the modulus passed negated (nq = 2^64 - q): r = a w + h nq mod 2^64, written
// in 32-bit pieces so that each partial product is one multiply-add (the low word of a0 w0 + h0 nq0 as
// one wide multiply-add, the high word as four narrow ones).
__device__ __forceinline__ u64 shoup_lazy4n(u64 a, u64 w, u64 ws, u64 nq) {
    const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32), s0 = (uint32_t)ws, s1 = (uint32_t)(ws >> 32);
    u64 h = (u64)a1 * s1 + __umulhi(a1, s0);
    h += __umulhi(a0, s1);
    const uint32_t h0 = (uint32_t)h, h1 = (uint32_t)(h >> 32);
    const uint32_t w0 = (uint32_t)w, w1 = (uint32_t)(w >> 32), n0 = (uint32_t)nq, n1 = (uint32_t)(nq >> 32);
    u64 r = (u64)a0 * w0;
    r += (u64)h0 * n0;
    const uint32_t rh = (uint32_t)(r >> 32) + a0 * w1 + a1 * w0 + h0 * n1 + h1 * n0;
    return ((u64)rh << 32) | (uint32_t)r;
}

__host__ __device__ __forceinline__ u64 shoup(u64 a, u64 w, u64 ws, u64 q) {
    u64 r = shoup_lazy(a, w, ws, q);
    return r >= q ? r - q : r;
}

// Montgomery reduction: z = hi 2^64 + lo < q 2^64, qinv = -q^-1 mod 2^64;
// returns z 2^-64 mod q in [0, q).
__host__ __device__ __forceinline__ u64 redc(u64 hi, u64 lo, u64 q, u64 qinv) {
    u64 m = lo * qinv;
    u64 t = hi + mulhi64(m, q) + (lo != 0 ? 1ull : 0ull);
    return t >= q ? t - q : t;
}

// 128-bit accumulate of a * b
__host__ __device__ __forceinline__ void mac128(u64& hi, u64& lo, u64 a, u64 b) {
    u64 l = a * b;
    u64 h = mulhi64(a, b);
    lo += l;
    hi += h + (lo < l ? 1ull : 0ull);
}

// x mod q for any 64-bit x, mu = floor(2^64 / q).
__host__ __device__ __forceinline__ u64 reduce64(u64 x, u64 q, u64 mu) {
    u64 r = x - mulhi64(x, mu) * q;
    return r >= q ? r - q : r;
}

// ------------------------------------------------------------------ exact base extension tables
// Centred extension of an integer given by residues modulo the source primes
// s_0..s_{n-1} (S = prod s_i) to target primes T_0..T_{m-1}: Garner's mixed
// radix digits v_i, a lexicographic compare of (v_{n-1}..v_0) against the
// digits of (S-1)/2 to decide x > S/2, Horner evaluation mod T_j and a
// subtraction of [S]_{T_j} for the negative half.
struct ExtDesc {
    int n_src, n_dst;
    const u64* src_q;    // [n_src]
    const u64* ginv;     // [n_src][n_src]: (i, j<i) -> s_j^-1 mod s_i   (Shoup pair w, ws)
    const u64* ginv_s;
    const u64* hdig;     // [n_src] mixed-radix digits of (S-1)/2
    const u64* dst_q;    // [n_dst]
    const u64* dst_mu;   // [n_dst] floor(2^64 / T_j)
    const u64* radix;    // [n_dst][n_src]: [s_i]_{T_j} (Shoup pair)
    const u64* radix_s;
    const u64* smod;     // [n_dst]: [S]_{T_j}
    // guarded fast path (all moduli < 2^50): x = sum_i y_i (S/s_i) - v S with y_i = [x_i (S/s_i)^-1]_{s_i}
    // and v = round(sum_i y_i / s_i) from a 64.64 fixed-point sum, unless that sum lies within
    // 2 n_src + 2 units of 1/2 (then the exact mixed-radix path decides)
    const u64* qhinv;    // [n_src] [(S/s_i)^-1]_{s_i} (Shoup pair)
    const u64* qhinv_s;
    const u64* g_hi;     // [n_src] floor(2^128 / s_i) >> 64
    const u64* g_lo;     // [n_src] floor(2^128 / s_i) mod 2^64
    const uint32_t* c26; // [n_dst][n_src][2] 26-bit limbs (low, high) of [(S/s_i) 2^64]_{T_j}
    const u64* dst_qinv; // [n_dst] -T_j^-1 mod 2^64
    const u64* vS;       // [n_dst][n_src + 1] [v S]_{T_j}
    int fast_ok;         // all moduli < 2^50: the fast path's tables are valid
};

// Host copies of the guarded fast extension's per-source tables and 26-bit limb pairs: the kernels take them
// as a kernel parameter (constant bank), so that the inner products read their factors without a load
struct ExtHost {
    int n = 0, m = 0;
    std::vector<uint32_t> c26;                       // [m][n][2]
    std::vector<u64> qhinv, qhinv_s, g_hi, g_lo;     // [n]
};

// Device-side prime tables of a context, by prime index
// (0..L-1 data, L..L+alpha-1 special, L+alpha..L+alpha+K-1 auxiliary, last: t).
struct PrimeTab {
    const u64* q;        // modulus
    const u64* qinv;     // -q^-1 mod 2^64
    const u64* mu;       // floor(2^64 / q)
    const u64* tw;       // [nP][N][2] (psi^brv(k), Shoup companion)      forward twiddles
    const u64* twl;      // [nP][3][N][2] the same, stages b < le regrouped per le = 3, 4, 5 (forward last pass)
    const u64* itw;      // [nP][N][2] inverse (DIT) twiddles: entry 2^b + j = omega^-(N/2^(b+1)) j, omega = psi^2
    const u64* twist;    // [nP][3][N][2] output twist N^-1 psi^-m (plain; times R = 2^64; times t R), mod q
};

// limb -> prime index map of a polynomial base: limb < split ? limb : limb + off
struct LimbMap {
    int split, off;
    __host__ __device__ __forceinline__ int operator()(int limb) const { return limb < split ? limb : limb + off; }
};

// ------------------------------------------------------------------ context
struct bfhe_ctx {
    int device = 0;
    uint32_t N = 0, logN = 0, L = 0, alpha = 0, K = 0, nP = 0, prime_bits = 0;
    u64 t = 0;
    bool batching = true;   // t = 1 mod 2N: slot encoding; t = 2: coefficient encoding only
    std::vector<u64> primes;     // nP: Q, P, B, t
    std::vector<uint32_t> brv;   // host copy of bit reversal (N)

    void* d_arena = nullptr;     // all constant tables
    size_t arena_bytes = 0;
    PrimeTab tab{};
    uint32_t* d_brv = nullptr;   // [N]
    ExtDesc ext_QB{}, ext_BQ{}, ext_PQ{}, ext_Qt{};
    ExtHost exth_QB, exth_BQ;
    // Shoup pair tables: p[i] = w_i, p[n + i] = ws_i
    const u64* d_tmod = nullptr;    // [nP] [t]_{prime}
    const u64* d_delta_q = nullptr; // [L]  [Delta]_{q_i}
    const u64* d_Qinv_b = nullptr;  // [K]  [Q^-1]_{b_j}
    const u64* d_Pinv_q = nullptr;  // [L]  [P^-1]_{q_i}
    const u64* d_P_q = nullptr;     // [L]  [P]_{q_i}
    const u64* d_R2 = nullptr;      // [nP] 2^128 mod prime (Montgomery R^2)
    u64 Qinv_t = 0;                 // [Q^-1]_t
    u64 delta_t = 0;

    // keys
    bool have_keys = false;
    i64* d_sk = nullptr;         // [N]
    u64* d_sk_ntt = nullptr;     // [L+alpha][N]
    u64* d_pk = nullptr;         // [2][L][N] coefficient form
    u64* d_pk_ntt = nullptr;     // [2][L][N]
    u64* d_rlk_ntt = nullptr;    // [L][2][L+alpha][N]

    // input-range flags raised by kernels (BFHE_FLAG_*), read and cleared by bfhe_check
    uint32_t* d_flags = nullptr;

    // scratch
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    size_t reserve_n = 0;

    uint64_t counts[4] = {0, 0, 0, 0};
    bool fast_ext = false;       // guarded fast base extension in the multiply (bfhe_set_fast_extension)

    // mod_to_bits tiles replayed from a CUDA graph (bfhe_set_graph_tiles): the tile is captured once on a
    // context-owned stream and replayed with its candidate base in the device word d_cbase; the
    // instantiated graph is kept for later calls with the same buffers and shape (key)
    bool graph_tiles = false;
    bool capturing = false;      // inside a stream capture: no profiling events
    cudaStream_t cap_stream = nullptr;
    cudaEvent_t cap_in = nullptr, cap_out = nullptr;
    u64* d_cbase = nullptr;
    cudaGraphExec_t tile_exec = nullptr;
    std::vector<u64> tile_key;
    uint64_t tile_counts[4] = {0, 0, 0, 0};   // op counts of one captured tile
    uint64_t tile_launches = 0;                // kernels in the captured tile

    // launch timing (measurement only): pending (class, start, stop) event triples
    struct ProfRec {
        int cls;
        double work, bytes;
        cudaEvent_t a, b;
    };
    mutable bool prof_on = false;
    mutable std::vector<ProfRec> prof_pending;
    mutable std::vector<cudaEvent_t> prof_pool;

    LimbMap mapQ() const { return LimbMap{(int)L, 0}; }
    LimbMap mapQP() const { return LimbMap{(int)(L + alpha), 0}; }
    LimbMap mapQB() const { return LimbMap{(int)L, (int)alpha}; }
    LimbMap mapT() const { return LimbMap{0, (int)(L + alpha + K)}; }
    size_t ct_words() const { return (size_t)2 * L * N; }
};

// ------------------------------------------------------------------ host helpers (host.cu)
int set_error(int code, const std::string& msg);
// process-wide count of kernel launches made by this library (measurement)
void count_launch();
void count_launches(uint64_t n);   // kernels launched by a graph replay
int cuda_check(cudaError_t e, const char* where);
#define BFHE_CUDA(call)                                          \
    do {                                                         \
        cudaError_t _e = (call);                                 \
        if (_e != cudaSuccess) return cuda_check(_e, #call);     \
    } while (0)
#define BFHE_LAUNCH_CHECK(where)                                 \
    do {                                                         \
        count_launch();                                          \
        cudaError_t _e = cudaGetLastError();                     \
        if (_e != cudaSuccess) return cuda_check(_e, where);     \
    } while (0)

// scratch arena: returns a pointer to at least `bytes` bytes (grows, syncing the device)
int ctx_scratch(bfhe_ctx* ctx, size_t bytes, void** out);
// bytes of scratch one mul_relin of n ciphertexts needs
size_t mul_scratch_bytes(const bfhe_ctx* ctx, size_t n);

// RAII bracket of one launcher's kernels by CUDA events when profiling is on
// (work = the launch's algorithmic 64-bit modular multiplies)
// work: algorithmic modmuls of the launch; bytes: its algorithmic DRAM bytes (each operand read and each
// result written once; tables that stay in L2 not counted)
struct ProfScope {
    const bfhe_ctx* c;
    int cls;
    double work, bytes;
    cudaStream_t st;
    cudaEvent_t a = nullptr, b = nullptr;
    ProfScope(const bfhe_ctx* ctx, int k, cudaStream_t s, double w, double by);
    ~ProfScope();
};

// ------------------------------------------------------------------ kernel launchers (ntt.cu)
// In/out-of-place negacyclic NTT over n_polys x n_limbs limbs.
// Poly p of a launch is (outer, inner) = (p / n_inner, p % n_inner); a limb's
// words start at base + outer*os + inner*is + limb*ls (strides in words).
struct NttIO {
    const u64* in;
    u64* out;
    int n_inner;
    size_t in_os, in_is, in_ls;
    size_t out_os, out_is, out_ls;
};
// contiguous [n_polys][n_limbs][N] in and out
inline NttIO ntt_io(const u64* in, u64* out, size_t n_limbs, size_t N) {
    NttIO io;
    io.in = in;
    io.out = out;
    io.n_inner = 1;
    io.in_os = io.out_os = n_limbs * N;
    io.in_is = io.out_is = 0;
    io.in_ls = io.out_ls = N;
    return io;
}
// lazy_out: outputs left below 64q (only taken when every prime is below 2^50) for consumers that
// multiply them in Montgomery form; otherwise canonical
int launch_ntt_fwd(const bfhe_ctx* ctx, NttIO io, int n_polys, int n_limbs, LimbMap map, cudaStream_t st,
                   int lazy_out = 0);
// mont != 0: the final scale is N^-1 R (undoes one Montgomery factor R^-1 of the inputs)
// lazy_out: 0 canonical; 1 outputs below 2q (the twist product without its final subtraction) for consumers
// that take lazy words; 2 no twist at all (words below 61q, from inputs below q) for consumers that fold the
// twist into a product of their own (scale-and-round, mod-down)
int launch_ntt_inv(const bfhe_ctx* ctx, NttIO io, int n_polys, int n_limbs, LimbMap map, int mont,
                   cudaStream_t st, int lazy_out = 0);
int ntt_config(int logN, int inverse, int* log_m, int* log_e);
void ntt_set_log_e(int log_e);   // tuning override (0 = default)
