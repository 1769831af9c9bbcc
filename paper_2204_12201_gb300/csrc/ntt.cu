// ntt.cu -- negacyclic NTT / INTT over Z_q[X]/(X^N + 1) per RNS prime.
//
// Forward: Cooley-Tukey with merged psi twiddles (natural order in, bit-
// reversed evaluation order out); butterfly on bit b of the index with
// twiddle psi^brv((N + j) >> (b + 1)) and one Shoup product.  The forward
// butterfly (X, Y) -> (X + T, X - T + 4q), T = Shoup(Y) in [0, 4q) (the
// quotient estimate may be up to three short, see shoup_lazy4n), grows the
// bound by 4q per stage and is never reduced in between: from inputs < 4q,
// 15 stages stay below 64q <= 2^64 for q < 2^58, and one Barrett-style
// reduction at the end makes the output canonical.  Inverse: a_m = N^-1 psi^-m sum_k a^_k
// omega^-km (omega = psi^2) -- a cyclic decimation-in-time transform on the
// bit-reversed input with the same reduction-free butterfly, then one twist
// product by N^-1 psi^-m per word (times R = 2^64 when the inputs carry a
// Montgomery factor), which also makes the output canonical.  Twiddles are
// stored as (w, Shoup(w)) pairs and fetched as one 16-byte load; the forward's
// last pass reads a copy regrouped so that a warp's loads are contiguous.
//
// One CTA transforms a block of M = 2^LOG_M words of a limb held in shared
// memory; each thread keeps E = 2^LOG_E words in registers and runs up to
// LOG_E radix-2 stages on them per pass, with one padded shared-memory
// exchange (one pad word per 16, conflict-free for every window) and one
// barrier between passes.  The first pass reads global memory directly
// (coalesced: lanes differ in the low index bits) and the last pass writes it
// directly (forward: E consecutive words per thread as 16-byte stores;
// inverse: coalesced).
//
// When N = 2M a limb is split over two CTAs (so that two of them share an SM
// at N = 16384), launched as a thread-block cluster of two so they are always
// co-resident.  Forward: the outermost stage pairs word j of the first half
// with word j of the second; each CTA reads both halves in its first pass and
// keeps the output of its own half, so the stage costs no extra pass; a
// cluster barrier after those reads keeps an in-place transform from
// overwriting words the partner has not read yet.
// Inverse: the two CTAs form a thread-block cluster; after the inner stages
// the outermost stage pairs word j of the first half with word j of the
// second: CTA 0 takes the pairs with j < M/2, CTA 1 the others, each reading
// the partner's word of its pairs through distributed shared memory, making
// the pair's one product and writing both outputs (and the twist).
#include <cooperative_groups.h>

#include <atomic>
#include <cstdlib>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace {

__device__ __forceinline__ int phys(int j) { return j + (j >> 4); }

// padded offset of word base + (e << W_LO) relative to phys(base): no carry crosses bit 4
// when e << W_LO is added to a pass's base (checked for every shape on the host), so the
// offset is a compile-time constant per e
template <int W_LO>
__device__ __forceinline__ constexpr int poff(int e) { return (e << W_LO) + ((e << W_LO) >> 4); }

struct NttArgs {
    const u64* in;
    u64* out;
    int n_inner;
    size_t in_os, in_is, in_ls, out_os, out_is, out_ls;
    int n_limbs;
    LimbMap map;
    PrimeTab tab;
    int N, logN;
    int mont;   // inverse: inputs carry a Montgomery factor
    int lazy;   // host side only: forward outputs < 64q / inverse outputs < 2q (selects the template)
    int device; // host side only: the context's device (function attributes are per device)
};

struct LimbPtrs {
    const u64* in;   // limb start
    u64* out;        // limb start
    int p;
};

__device__ __forceinline__ LimbPtrs limb_ptrs(const NttArgs& a, int bx) {
    const int limb = bx % a.n_limbs;
    const int poly = bx / a.n_limbs;
    const int outer = poly / a.n_inner, inner = poly % a.n_inner;
    LimbPtrs r;
    r.in = a.in + outer * a.in_os + inner * a.in_is + limb * a.in_ls;
    r.out = a.out + outer * a.out_os + inner * a.out_is + limb * a.out_ls;
    r.p = a.map(limb);
    return r;
}

// ---------------------------------------------------------------- forward stages
// The last pass (W_LO = 0: E consecutive words per thread) takes its twiddles from the regrouped table:
// twc is this thread's column there, and its g-th twiddle of stage b sits (N >> (b+1)) + g (N / E) entries
// further, so lanes read consecutive 16-byte entries (the standard table gives each lane its own run of
// E >> (b+1) entries: 32 sectors per warp load instead of 16 contiguous).
template <int LOG_N, int LOG_E, int W_LO, int HI, int LO>
__device__ __forceinline__ void fwd_stages(u64 (&x)[1 << LOG_E], u64 jb, const ulonglong2* __restrict__ tw,
                                           const ulonglong2* __restrict__ twc, u64 q) {
    constexpr int E = 1 << LOG_E;
    const u64 q4 = 4 * q, nq = 0 - q;
#pragma unroll
    for (int st = 0; st <= HI - LO; ++st) {
        const int b = HI - st;
        const int h = b - W_LO;
        const u64 base = jb >> (b + 1);
#pragma unroll
        for (int g = 0; g < (E >> (h + 1)); ++g) {
            const ulonglong2 wp = W_LO == 0 ? __ldg(twc + ((1 << LOG_N) >> (b + 1)) + g * (1 << (LOG_N - LOG_E)))
                                            : __ldg(tw + base + g);
#pragma unroll
            for (int r = 0; r < (1 << h); ++r) {
                const int e = (g << (h + 1)) | r;
                const int e2 = e | (1 << h);
                const u64 X = x[e];
                const u64 T = shoup_lazy4n(x[e2], wp.x, wp.y, nq);
                x[e] = X + T;
                x[e2] = X + q4 - T;
            }
        }
    }
}

// TOP: this CTA is half `half` of a limb of N = 2M words and first applies the
// outermost stage (twiddle psi^brv(1)) to the pairs (j, j + M) it reads.
template <int LOG_M, int LOG_E, int P, bool TOP, bool LAZY>
__device__ __forceinline__ void fwd_pass(u64 (&x)[1 << LOG_E], u64* sm, int tid, u64 jglob, const ulonglong2* tw,
                                         const ulonglong2* twl, u64 q, u64 mu, const u64* in, u64* out, int half) {
    constexpr int E = 1 << LOG_E;
    constexpr int M = 1 << LOG_M;
    constexpr int NPASS = (LOG_M + LOG_E - 1) / LOG_E;
    constexpr int HI = LOG_M - 1 - P * LOG_E;
    constexpr int LO = (HI - LOG_E + 1) > 0 ? (HI - LOG_E + 1) : 0;
    constexpr int W_LO = LO;
    const int base = (tid & ((1 << W_LO) - 1)) | ((tid >> W_LO) << (W_LO + LOG_E));
    const int pb = phys(base);
    if (P == 0) {
        if (TOP) {
            const ulonglong2 w1 = __ldg(tw + 1);
            const u64 q4 = 4 * q;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const u64 X = in[base + (e << W_LO)];
                const u64 T = shoup_lazy4n(in[M + base + (e << W_LO)], w1.x, w1.y, 0 - q);
                x[e] = half ? X + q4 - T : X + T;
            }
            // both halves of the limb are read before either CTA writes (in-place transforms)
            cg::this_cluster().sync();
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) x[e] = in[base + (e << W_LO)];
        }
    } else {
#pragma unroll
        for (int e = 0; e < E; ++e) x[e] = sm[pb + poff<W_LO>(e)];
    }
    constexpr int LOG_N = TOP ? LOG_M + 1 : LOG_M;
    // thread index over the whole limb (last pass): (jglob - N + base) / E
    const ulonglong2* twc = W_LO == 0 ? twl + ((((u64)half << LOG_M) + base) >> LOG_E) : twl;
    fwd_stages<LOG_N, LOG_E, W_LO, HI, LO>(x, jglob + base, tw, twc, q);
    if constexpr (P + 1 < NPASS) {
#pragma unroll
        for (int e = 0; e < E; ++e) sm[pb + poff<W_LO>(e)] = x[e];
        __syncthreads();
        fwd_pass<LOG_M, LOG_E, P + 1, TOP, LAZY>(x, sm, tid, jglob, tw, twl, q, mu, in, out, half);
    } else {
        // W_LO == 0 here: E consecutive words per thread; values < 64q -> canonical unless the
        // consumer takes lazy words (Montgomery products of operands < 64q, q < 2^50)
        if constexpr (!LAZY) {
#pragma unroll
            for (int e = 0; e < E; ++e) x[e] = reduce64(x[e], q, mu);
        }
        ulonglong2* o2 = reinterpret_cast<ulonglong2*>(out + base);
#pragma unroll
        for (int e = 0; e < E / 2; ++e) o2[e] = make_ulonglong2(x[2 * e], x[2 * e + 1]);
    }
}

template <int LOG_M, int LOG_E, bool TOP, bool LAZY>
__global__ void __launch_bounds__(1 << (LOG_M - LOG_E), (LOG_M < 14 && LOG_M - LOG_E <= 8 ? 2 : 1)) k_ntt_fwd(NttArgs a) {
    extern __shared__ u64 sm[];
    const LimbPtrs lp = limb_ptrs(a, blockIdx.x);
    const int half = blockIdx.y;
    const u64 q = a.tab.q[lp.p], mu = a.tab.mu[lp.p];
    const ulonglong2* tw = reinterpret_cast<const ulonglong2*>(a.tab.tw) + (size_t)lp.p * a.N;
    const ulonglong2* twl = reinterpret_cast<const ulonglong2*>(a.tab.twl) + ((size_t)lp.p * 3 + (LOG_E - 3)) * a.N;
    const u64 jglob = (u64)a.N + ((u64)half << LOG_M);
    const u64* in = TOP ? lp.in : lp.in + ((size_t)half << LOG_M);
    u64 x[1 << LOG_E];
    fwd_pass<LOG_M, LOG_E, 0, TOP, LAZY>(x, sm, threadIdx.x, jglob, tw, twl, q, mu, in,
                                         lp.out + ((size_t)half << LOG_M), half);
}

// ---------------------------------------------------------------- inverse stages
// Decimation in time on the bit-reversed input with inverse roots: the butterfly on
// bit b at lower index x is (U, V) -> (U + T, U - T + 4q), T = V omega^-(N/2^(b+1)) (x mod 2^b)
// (table entry 2^b + (x mod 2^b)); bounds grow by 4q per stage, as in the forward.
// The natural-order output is then multiplied by the twist N^-1 psi^-m.
template <int LOG_E, int W_LO, int LO, int HI>
__device__ __forceinline__ void inv_stages(u64 (&x)[1 << LOG_E], int base, const ulonglong2* __restrict__ itw, u64 q) {
    constexpr int E = 1 << LOG_E;
    const u64 q4 = 4 * q, nq = 0 - q;
#pragma unroll
    for (int st = 0; st <= HI - LO; ++st) {
        const int b = LO + st;
        const int h = b - W_LO;
        const int tbase = (1 << b) + (base & ((1 << b) - 1));
#pragma unroll
        for (int r = 0; r < (1 << h); ++r) {
            const ulonglong2 wp = __ldg(itw + tbase + (r << W_LO));
#pragma unroll
            for (int g = 0; g < (E >> (h + 1)); ++g) {
                const int e = (g << (h + 1)) | r;
                const int e2 = e | (1 << h);
                const u64 U = x[e];
                const u64 T = shoup_lazy4n(x[e2], wp.x, wp.y, nq);
                x[e] = U + T;
                x[e2] = U + q4 - T;
            }
        }
    }
}

// MODE 1: the block is the whole limb; MODE 2: half `half` of a limb of N = 2M words,
// whose outermost stage pairs with the partner CTA of the cluster.
// OUT 0: twisted, canonical; 1: twisted, below 2q; 2: not twisted (the consumer multiplies by the twist,
// folded into a product it makes anyway): from inputs below q, 15 stages leave words below 61q < 2^64.
template <int LOG_M, int LOG_E, int P, int MODE, int OUT>
__device__ __forceinline__ void inv_pass(u64 (&x)[1 << LOG_E], u64* sm, int tid, const ulonglong2* itw,
                                         const ulonglong2* twist, u64 q, const u64* in, u64* out, int half) {
    constexpr int E = 1 << LOG_E;
    constexpr int M = 1 << LOG_M;
    constexpr int NPASS = (LOG_M + LOG_E - 1) / LOG_E;
    constexpr int LO = P * LOG_E;
    constexpr int HI = (LO + LOG_E - 1) < (LOG_M - 1) ? (LO + LOG_E - 1) : (LOG_M - 1);
    constexpr int W_LO = (HI - LO + 1 == LOG_E) ? LO : (LOG_M - LOG_E);
    const int base = (tid & ((1 << W_LO) - 1)) | ((tid >> W_LO) << (W_LO + LOG_E));
    const int pb = phys(base);
    if (P == 0) {
        // W_LO == 0: E consecutive words per thread
        const ulonglong2* i2 = reinterpret_cast<const ulonglong2*>(in + base);
#pragma unroll
        for (int e = 0; e < E / 2; ++e) {
            const ulonglong2 v = i2[e];
            x[2 * e] = v.x;
            x[2 * e + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int e = 0; e < E; ++e) x[e] = sm[pb + poff<W_LO>(e)];
    }
    constexpr bool LAST = (P + 1 == NPASS);
    inv_stages<LOG_E, W_LO, LO, HI>(x, base, itw, q);
    if constexpr (!LAST) {
#pragma unroll
        for (int e = 0; e < E; ++e) sm[pb + poff<W_LO>(e)] = x[e];
        __syncthreads();
        inv_pass<LOG_M, LOG_E, P + 1, MODE, OUT>(x, sm, tid, itw, twist, q, in, out, half);
    } else if constexpr (MODE == 2) {
        // outermost stage across the halves, pairs (j, j + M): the top bit of e is bit LOG_M - 1 of j, so
        // CTA 0 takes the pairs with j < M/2 and CTA 1 those with j >= M/2; each publishes the words of the
        // other set, reads the partner's word of each pair it takes through distributed shared memory,
        // makes the pair's one product and writes both outputs (the limb's positions j and j + M)
        cg::cluster_group cl = cg::this_cluster();
        constexpr int EH = E / 2;
        // (register indices stay compile-time: the half selects between two words)
#pragma unroll
        for (int e = 0; e < EH; ++e) {
            const u64 v = half ? x[e] : x[e + EH];   // the set the partner takes
            sm[pb + (half ? poff<W_LO>(e) : poff<W_LO>(e + EH))] = v;
        }
        cl.sync();
        const u64* peer = cl.map_shared_rank(sm, cl.block_rank() ^ 1u);
        const u64 q4 = 4 * q;
        u64* o = out - (size_t)half * M;        // limb start
#pragma unroll
        for (int e = 0; e < EH; ++e) {
            const u64 mine = half ? x[e + EH] : x[e];
            const int off = half ? poff<W_LO>(e + EH) : poff<W_LO>(e);
            const int j = base + ((half ? e + EH : e) << W_LO);
            const u64 other = peer[pb + off];
            const u64 U = half ? other : mine, V = half ? mine : other;
            const ulonglong2 wp = __ldg(itw + M + j);
            const u64 T = shoup_lazy4n(V, wp.x, wp.y, 0 - q);
            const u64 y0 = U + T, y1 = U + q4 - T;
            if constexpr (OUT == 2) {
                o[j] = y0;
                o[j + M] = y1;
            } else {
                const ulonglong2 t0 = __ldg(twist + j), t1 = __ldg(twist + j + M);
                o[j] = OUT == 1 ? shoup_lazy(y0, t0.x, t0.y, q) : shoup(y0, t0.x, t0.y, q);
                o[j + M] = OUT == 1 ? shoup_lazy(y1, t1.x, t1.y, q) : shoup(y1, t1.x, t1.y, q);
            }
        }
        cl.sync();   // the partner has finished reading this CTA's shared memory
    } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int j = base + (e << W_LO);
            if constexpr (OUT == 2) {
                out[j] = x[e];
            } else {
                const ulonglong2 tw = __ldg(twist + j);
                out[j] = OUT == 1 ? shoup_lazy(x[e], tw.x, tw.y, q) : shoup(x[e], tw.x, tw.y, q);
            }
        }
    }
}

template <int LOG_M, int LOG_E, int MODE, int OUT>
__global__ void __launch_bounds__(1 << (LOG_M - LOG_E), (MODE == 2 && LOG_M < 14 && LOG_M - LOG_E <= 8 ? 2 : 1)) k_ntt_inv(NttArgs a) {
    extern __shared__ u64 sm[];
    const LimbPtrs lp = limb_ptrs(a, blockIdx.x);
    const int half = blockIdx.y;
    const u64 q = a.tab.q[lp.p];
    const ulonglong2* itw = reinterpret_cast<const ulonglong2*>(a.tab.itw) + (size_t)lp.p * a.N;
    const ulonglong2* twist = reinterpret_cast<const ulonglong2*>(a.tab.twist) + ((size_t)lp.p * 3 + (a.mont ? 1 : 0)) * a.N;
    u64 x[1 << LOG_E];
    inv_pass<LOG_M, LOG_E, 0, MODE, OUT>(x, sm, threadIdx.x, itw, twist, q, lp.in + ((size_t)half << LOG_M),
                                    lp.out + ((size_t)half << LOG_M), half);
}

int g_log_e_override = 0;

template <int LOG_M, int LOG_E>
constexpr size_t smem_bytes() {
    return (LOG_M + LOG_E - 1) / LOG_E > 1 ? (size_t)((1 << LOG_M) + ((1 << LOG_M) >> 4)) * 8 : 0;
}

template <int LOG_M, int LOG_E, bool TOP, bool LAZY>
int run_fwd(const NttArgs& a, int blocks, cudaStream_t st) {
    constexpr int T = 1 << (LOG_M - LOG_E);
    const size_t smem = smem_bytes<LOG_M, LOG_E>();
    static std::atomic<uint64_t> attr{0};   // devices whose function attribute is set
    const int dev = a.device;
    if (!(attr.load() >> dev & 1)) {
        BFHE_CUDA(cudaFuncSetAttribute(k_ntt_fwd<LOG_M, LOG_E, TOP, LAZY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
        attr.fetch_or(1ull << dev);
    }
    if (TOP) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(blocks, 2, 1);
        cfg.blockDim = dim3(T, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 1;
        at[0].val.clusterDim.y = 2;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        BFHE_CUDA(cudaLaunchKernelEx(&cfg, k_ntt_fwd<LOG_M, LOG_E, TOP, LAZY>, a));
        BFHE_LAUNCH_CHECK("k_ntt_fwd (cluster)");
    } else {
        k_ntt_fwd<LOG_M, LOG_E, TOP, LAZY><<<dim3(blocks, 1), T, smem, st>>>(a);
        BFHE_LAUNCH_CHECK("k_ntt_fwd");
    }
    return BFHE_OK;
}

template <int LOG_M, int LOG_E, int MODE, int OUT>
int run_inv(const NttArgs& a, int blocks, cudaStream_t st) {
    constexpr int T = 1 << (LOG_M - LOG_E);
    // the cluster exchange needs the shared buffer even for a single pass
    const size_t smem = MODE == 2 ? (size_t)((1 << LOG_M) + ((1 << LOG_M) >> 4)) * 8 : smem_bytes<LOG_M, LOG_E>();
    static std::atomic<uint64_t> attr{0};   // devices whose function attribute is set
    const int dev = a.device;
    if (!(attr.load() >> dev & 1)) {
        BFHE_CUDA(cudaFuncSetAttribute(k_ntt_inv<LOG_M, LOG_E, MODE, OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
        attr.fetch_or(1ull << dev);
    }
    if (MODE == 2) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(blocks, 2, 1);
        cfg.blockDim = dim3(T, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 1;
        at[0].val.clusterDim.y = 2;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        BFHE_CUDA(cudaLaunchKernelEx(&cfg, k_ntt_inv<LOG_M, LOG_E, MODE, OUT>, a));
        BFHE_LAUNCH_CHECK("k_ntt_inv (cluster)");
    } else {
        k_ntt_inv<LOG_M, LOG_E, MODE, OUT><<<dim3(blocks, 1), T, smem, st>>>(a);
        BFHE_LAUNCH_CHECK("k_ntt_inv");
    }
    return BFHE_OK;
}

NttArgs make_args(const bfhe_ctx* ctx, const NttIO& io, int n_limbs, LimbMap map, int mont, int lazy) {
    NttArgs a;
    a.in = io.in;
    a.out = io.out;
    a.n_inner = io.n_inner > 0 ? io.n_inner : 1;
    a.in_os = io.in_os;
    a.in_is = io.in_is;
    a.in_ls = io.in_ls;
    a.out_os = io.out_os;
    a.out_is = io.out_is;
    a.out_ls = io.out_ls;
    a.n_limbs = n_limbs;
    a.map = map;
    a.tab = ctx->tab;
    a.N = (int)ctx->N;
    a.logN = (int)ctx->logN;
    a.mont = mont;
    a.lazy = lazy;
    a.device = ctx->device < 64 ? ctx->device : 63;
    return a;
}

int env_int(const char* name) {
    const char* s = getenv(name);
    return s ? atoi(s) : 0;
}

}  // namespace

void ntt_set_log_e(int log_e) { g_log_e_override = log_e; }

// Block size and registers per thread.  Defaults (measured on GB300): N <= 8192
// in one block; N = 16384 forward as two 8192-word halves (two CTAs per SM) and
// inverse in one block; N = 32768 as two 16384-word halves.  bfhe_ntt_config
// (the autotuner) or BFHE_NTT_LOG_M / BFHE_NTT_LOG_E override them.
int g_cfg[16][2][2] = {};   // [logN][inverse] -> (log_m, log_e), 0 = default

int ntt_config(int logN, int inverse, int* log_m, int* log_e) {
    static const int env_m = env_int("BFHE_NTT_LOG_M");
    static const int env_e = env_int("BFHE_NTT_LOG_E");
    int m = logN <= 13 ? logN : logN - 1;
    if (inverse && logN == 14) m = 14;
    if (env_m >= logN - 1 && env_m <= logN && env_m >= 10 && env_m <= 14) m = env_m;
    int e = (m == 14 || (m == 13 && logN == 14)) ? 5 : 4;
    if (env_e >= 3 && env_e <= 5) e = env_e;
    if (g_log_e_override >= 3 && g_log_e_override <= 5) e = g_log_e_override;
    if (logN >= 0 && logN < 16 && g_cfg[logN][inverse ? 1 : 0][0]) {
        m = g_cfg[logN][inverse ? 1 : 0][0];
        e = g_cfg[logN][inverse ? 1 : 0][1];
    }
    if (m == 14 && e < 4) e = 4;
    *log_m = m;
    *log_e = e;
    return BFHE_OK;
}

extern "C" int bfhe_ntt_config(uint32_t logN, int inverse, uint32_t log_m, uint32_t log_e, uint32_t* cur_m,
                               uint32_t* cur_e) {
    if (logN < 10 || logN > 15) return set_error(BFHE_EINVAL, "logN must be in [10, 15]");
    if (log_m != 0) {
        if (log_m > logN || log_m + 1 < logN || log_m < 10 || log_m > 14 || log_e < 3 || log_e > 5 ||
            (log_m == 14 && log_e < 4))
            return set_error(BFHE_EINVAL, "unsupported NTT block configuration");
        g_cfg[logN][inverse ? 1 : 0][0] = (int)log_m;
        g_cfg[logN][inverse ? 1 : 0][1] = (int)log_e;
    }
    int m, e;
    ntt_config((int)logN, inverse, &m, &e);
    if (cur_m) *cur_m = (uint32_t)m;
    if (cur_e) *cur_e = (uint32_t)e;
    return BFHE_OK;
}

template <int LM, int LE>
int run_fwd_any(const NttArgs& a, int blocks, cudaStream_t st, bool top, bool lazy) {
    if (top) return lazy ? run_fwd<LM, LE, true, true>(a, blocks, st) : run_fwd<LM, LE, true, false>(a, blocks, st);
    return lazy ? run_fwd<LM, LE, false, true>(a, blocks, st) : run_fwd<LM, LE, false, false>(a, blocks, st);
}

#define FWD_CASE(LM, LE)                                                                                   \
    if (log_m == LM && log_e == LE)                                                                         \
        return run_fwd_any<LM, LE>(a, blocks, st, top, lazy);
template <int LM, int LE, int MODE>
int run_inv_out(const NttArgs& a, int blocks, cudaStream_t st, int out) {
    if (out == 2) return run_inv<LM, LE, MODE, 2>(a, blocks, st);
    return out == 1 ? run_inv<LM, LE, MODE, 1>(a, blocks, st) : run_inv<LM, LE, MODE, 0>(a, blocks, st);
}

template <int LM, int LE>
int run_inv_any(const NttArgs& a, int blocks, cudaStream_t st, bool split, int out) {
    return split ? run_inv_out<LM, LE, 2>(a, blocks, st, out) : run_inv_out<LM, LE, 1>(a, blocks, st, out);
}

#define INV_CASE(LM, LE)                                                                                   \
    if (log_m == LM && log_e == LE)                                                                         \
        return run_inv_any<LM, LE>(a, blocks, st, split, out);

int launch_ntt_fwd(const bfhe_ctx* ctx, NttIO io, int n_polys, int n_limbs, LimbMap map, cudaStream_t st,
                   int lazy_out) {
    if (n_polys <= 0 || n_limbs <= 0) return BFHE_OK;
    ProfScope ps(ctx, BFHE_K_NTT_FWD, st, (double)n_polys * n_limbs * (ctx->N / 2) * ctx->logN,
                 16.0 * n_polys * n_limbs * ctx->N);
    int log_m, log_e;
    ntt_config((int)ctx->logN, 0, &log_m, &log_e);
    NttArgs a = make_args(ctx, io, n_limbs, map, 0, lazy_out && ctx->prime_bits <= 50 ? 1 : 0);
    const int blocks = n_polys * n_limbs;
    const int subs = (int)(ctx->N >> log_m);
    if (subs != 1 && subs != 2) return set_error(BFHE_EINVAL, "unsupported ring degree");
    const bool top = subs == 2;
    const bool lazy = a.lazy != 0;
    FWD_CASE(10, 3) FWD_CASE(10, 4) FWD_CASE(10, 5)
    FWD_CASE(11, 3) FWD_CASE(11, 4) FWD_CASE(11, 5)
    FWD_CASE(12, 3) FWD_CASE(12, 4) FWD_CASE(12, 5)
    FWD_CASE(13, 3) FWD_CASE(13, 4) FWD_CASE(13, 5)
    FWD_CASE(14, 4) FWD_CASE(14, 5)
    return set_error(BFHE_EINVAL, "no NTT configuration for this ring degree");
}

int launch_ntt_inv(const bfhe_ctx* ctx, NttIO io, int n_polys, int n_limbs, LimbMap map, int mont,
                   cudaStream_t st, int lazy_out) {
    if (n_polys <= 0 || n_limbs <= 0) return BFHE_OK;
    ProfScope ps(ctx, BFHE_K_NTT_INV, st, (double)n_polys * n_limbs * (ctx->N / 2) * ctx->logN,
                 16.0 * n_polys * n_limbs * ctx->N);
    int log_m, log_e;
    ntt_config((int)ctx->logN, 1, &log_m, &log_e);
    NttArgs a = make_args(ctx, io, n_limbs, map, mont, lazy_out);
    const int blocks = n_polys * n_limbs;
    const int subs = (int)(ctx->N >> log_m);
    if (subs != 1 && subs != 2) return set_error(BFHE_EINVAL, "unsupported ring degree");
    if (lazy_out < 0 || lazy_out > 2) return set_error(BFHE_EINVAL, "bad inverse output form");
    const bool split = subs == 2;
    const int out = lazy_out;
    INV_CASE(10, 3) INV_CASE(10, 4) INV_CASE(10, 5)
    INV_CASE(11, 3) INV_CASE(11, 4) INV_CASE(11, 5)
    INV_CASE(12, 3) INV_CASE(12, 4) INV_CASE(12, 5)
    INV_CASE(13, 3) INV_CASE(13, 4) INV_CASE(13, 5)
    INV_CASE(14, 4) INV_CASE(14, 5)
    return set_error(BFHE_EINVAL, "no NTT configuration for this ring degree");
}
