/*
 * bfhe.h -- C ABI of the GB300 library for bridged BFV arithmetic.
 *
 * The paper (Chielle, Mazonka, Gamil, Maniatakos, "Accelerating Fully
 * Homomorphic Encryption by Bridging Modular and Bit-Level Arithmetic",
 * ICCAD'22) mixes two secure types on one BFV key set (Sec. 3.2): SecureMod,
 * a native ciphertext mod t, and SecureUint/SecureBool, arrays of ciphertexts
 * that each encrypt a bit.  This library computes the ciphertext kernels both
 * reduce to, on one GPU: the gate equations of Sec. 3.1, the bit -> mod
 * conversion of Listing 5 and the mod -> bit conversion of Eq. 2 / Listings
 * 7-8, over an RNS BFV (Fan-Vercauteren) evaluator.
 *
 * Conventions (every function below):
 *  - All ciphertext, plaintext and slot buffers are caller-owned DEVICE
 *    memory on the context's device.  A ciphertext is uint64 [2][L][N]: two
 *    polynomials, each L RNS limbs of N coefficients, coefficient form,
 *    residues canonical in [0, q_i).  A batch of n ciphertexts is n of those
 *    back to back ([n][2][L][N]).  Slot vectors are uint64 [n][N], values < t.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream) of the context's device, which must be the calling thread's
 *    current CUDA device.  Calls enqueue work and return without
 *    synchronising; outputs are ready when the stream reaches that point.
 *  - The context owns keys, tables and a scratch arena (device memory it
 *    allocates itself with cudaMalloc, grown on demand; growth synchronises
 *    the device, so reserve with bfhe_reserve before capturing a CUDA graph).
 *  - Return value: BFHE_OK (0) or a negative BFHE_E* code; no call aborts,
 *    traps or throws.  Shapes, parameters and pointers are checked at the
 *    call; value ranges (residues < q_i, plaintext values < t) are checked by
 *    the kernels that read them and reported by bfhe_check (below).
 *  - A context is used by one host thread at a time (its scratch arena and
 *    operation counters are not locked); different contexts are independent.
 *    Calls on one context with different streams are ordered only by the
 *    caller: the arena is shared, so put one context's calls on one stream
 *    or synchronise between streams.
 *  - Outputs may alias inputs only where stated.
 *  - Deterministic: the same seeds and inputs give bit-identical outputs.
 */
#ifndef BFHE_H
#define BFHE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BFHE_OK 0
#define BFHE_EINVAL (-1)   /* bad shape, size, parameter or NULL pointer   */
#define BFHE_ENOMEM (-2)   /* device allocation failed                     */
#define BFHE_ECUDA (-3)    /* a CUDA call failed (bfhe_last_error names it) */
#define BFHE_ETIMEOUT (-4) /* a device-side wait gave up (reserved: this     */
                           /* build has no device-side waits)                */
#define BFHE_ESTATE (-5)   /* call out of order (e.g. encrypt before keygen) */

/* Input-range flags.  Calls are asynchronous, so values are not checked on
 * the host; kernels that read a plaintext value (encrypt, encrypt_poly,
 * mul_plain) or a ciphertext residue (mul_relin and everything built on it,
 * decrypt) raise a flag in the context when one is out of range, and compute
 * on regardless (a wrong but in-bounds result: no fault).  bfhe_check
 * synchronises `stream`, returns the flags raised since the previous check in
 * *flags_out (may be NULL), clears them, and returns BFHE_EINVAL if any was
 * raised.  Linear ops (add, sub, ...) do not check. */
#define BFHE_FLAG_PLAINTEXT 1u   /* a slot value or plaintext coefficient >= t */
#define BFHE_FLAG_RESIDUE 2u     /* a ciphertext residue >= its prime q_i      */

typedef struct bfhe_ctx bfhe_ctx;

/* Parameters.  The moduli follow one rule (the paper fixes only n, t and the
 * security level and lets SEAL pick the rest, Sec. 4.1): every modulus is a
 * prime q = 1 (mod 2N) below 2^prime_bits taken from one downward scan over
 * q = 2N k + 1 skipping t; the first L are the data primes (Q), the next
 * alpha the special primes of relinearisation (P), the next K the auxiliary
 * base of the exact multiply, K being the least count with B > 2 t N Q. */
typedef struct {
    uint32_t N;          /* ring degree, power of two, 1024 .. 32768          */
    uint32_t L;          /* data primes, 1 .. 32; above 16 the base extensions */
                         /* and the key-switch inner product run runtime-size */
                         /* kernels (slower; meant for insecure, test-only    */
                         /* moduli that hold deep circuits)                   */
    uint32_t alpha;      /* special primes, 1 or 2                             */
    uint32_t prime_bits; /* bit size of every modulus, 30 .. 58 (default 50)   */
    uint64_t t;          /* plaintext modulus: a prime = 1 (mod 2N), < 2^32,   */
                         /* or 2 (no batching: coefficient encoding only,      */
                         /* Sec. 4.1 and 4.3 run bit-level arithmetic at t = 2) */
} bfhe_params;

/* The parameter rule alone, on the host (no device is touched): the moduli
 * a context with these parameters would use, in library order (data,
 * special, auxiliary; at least L + alpha + K entries in primes_out: 64 are
 * enough up to 16 data primes, 80 always), and K.  Same validation and errors as bfhe_ctx_create. */
int bfhe_param_primes(const bfhe_params* prm, uint64_t* primes_out, uint32_t* K_out);

/* Create a context on CUDA device `device`.  Builds the moduli, NTT twiddles
 * and RNS constants on the host and uploads them.  *out is set on success. */
int bfhe_ctx_create(const bfhe_params* prm, int device, bfhe_ctx** out);
void bfhe_ctx_destroy(bfhe_ctx* ctx);

/* Moduli in library order: primes_out[0 .. L+alpha+K-1] = q_0..q_{L-1},
 * p_0..p_{alpha-1}, b_0..b_{K-1} (host buffer of at least L + alpha + K entries:
 * 64 are enough up to 16 data primes, 80 always);
 * *K_out = K.  Also usable before keygen. */
int bfhe_ctx_primes(const bfhe_ctx* ctx, uint64_t* primes_out, uint32_t* K_out);

/* Read and clear the input-range flags (see BFHE_FLAG_* above). */
int bfhe_check(bfhe_ctx* ctx, void* stream, uint32_t* flags_out);

/* Reserve scratch for batches of up to n ciphertexts in every call (avoids
 * growth, hence device synchronisation, inside later calls). */
int bfhe_reserve(bfhe_ctx* ctx, size_t n);

/* Device memory the context holds, in bytes (host buffer of 4): out[0] the
 * constant tables (moduli, twiddles, twists, extension tables), out[1] the
 * keys (0 before keygen), out[2] the scratch arena (it grows to the largest
 * call and does not shrink), out[3] other small buffers.  For admission
 * control by device memory (serving); the paper has no counterpart. */
int bfhe_ctx_device_bytes(const bfhe_ctx* ctx, size_t* out);

/* Scratch bytes one mul_relin of n ciphertexts uses (its arena share; calls
 * beyond the scratch budget run in tiles of this size); 0 for a NULL context. */
size_t bfhe_mul_scratch_bytes(const bfhe_ctx* ctx, size_t n);

/* Guarded fast base extension inside the multiply.  The
 * exact extensions of the lift (Q -> B) and of the scale-and-round (Q -> B,
 * B -> Q) normally run Garner's mixed-radix digits.  With this on they first
 * try y_i = [x_i (S/s_i)^-1]_{s_i}, x = sum_i y_i (S/s_i) - v S with v =
 * round(sum_i y_i / s_i) from a 64.64 fixed-point sum, and fall back to the
 * mixed-radix path when that sum is within 2n + 2 units of 1/2, where the
 * fixed-point rounding could pick the wrong v.  Results are identical
 * either way (bit for bit); only the speed differs.  Needs every modulus
 * below 2^50 and at most 16 data primes (BFHE_EINVAL otherwise).  Default: on
 * from 8 to 16 data primes (where it measured faster on GB300), off
 * otherwise.  bfhe_fast_extension
 * returns the current setting (1 or 0; BFHE_EINVAL for a NULL context).  The
 * paper has no counterpart: SEAL, which it runs on, uses approximate fast
 * conversions of this family. */
int bfhe_set_fast_extension(bfhe_ctx* ctx, int on);
int bfhe_fast_extension(const bfhe_ctx* ctx);

/* mod_to_bits (and the two conversions inside mod_to_sint) runs its candidates
 * c in tiles (Sec. 3.2.3, Eq. 2: one Fermat chain d_c^(t-1) per candidate,
 * then the s products of Listing 8).  With graph tiles on, a call with at
 * least two full tiles runs the first tile eagerly, captures the next one as
 * a CUDA graph (its candidate base read from a context-owned device word)
 * and replays that graph for every further full tile; the ragged last tile
 * runs eagerly.  The work moves to a context-owned stream joined to the
 * caller's stream by events, so the call stays asynchronous and ordered on
 * the caller's stream.  The instantiated graph is kept for later calls with
 * the same buffers and tile shape.  Results and op counts are identical
 * either way; the first use allocates a word of device memory, a stream and
 * two events.  With profiling on (bfhe_profile) tiles run eagerly.  Default:
 * off.  bfhe_graph_tiles returns the setting (1 or 0; BFHE_EINVAL for a NULL
 * context). */
int bfhe_set_graph_tiles(bfhe_ctx* ctx, int on);
int bfhe_graph_tiles(const bfhe_ctx* ctx);

/* Process-wide device-memory budget for one call's scratch (default 16 GiB).
 * Calls whose batch needs more are tiled: the multiplies run in chunks that
 * fit, mod_to_bits runs its candidates in groups; results do not depend on
 * the budget.  A smaller budget bounds the arena for memory-constrained
 * serving (and lets tests run the tiled paths at small sizes).  It is a
 * target, not a cap: a call always gets its fixed buffers and the scratch of
 * one multiply.  Budgets below 1 MiB are rejected (BFHE_EINVAL).  Not
 * synchronised with calls in flight on other host threads: set it before
 * using the library. */
int bfhe_set_scratch_budget(size_t bytes);
size_t bfhe_scratch_budget(void);

/* Most ciphertexts one multiply launch sequence takes at ring degree 2^logN
 * (process-wide; 0, the default, means as many as the scratch budget holds).
 * Larger batches run in tiles of this size; results do not depend on it.
 * The autotuner sets it (paper_2204_12201_gb300/autotune.py).  BFHE_EINVAL
 * for logN outside [10, 15]; bfhe_mul_tile returns the setting. */
int bfhe_set_mul_tile(uint32_t logN, size_t max_ct);
size_t bfhe_mul_tile(uint32_t logN);

/* Key generation from `seed` (keys stay resident on the device): secret s
 * ternary, pk = ([-(a s + e)]_Q, a), relinearisation keys for the RNS digits
 * j = 0..L-1: ([-(a_j s + e_j) + P g_j s^2]_{PQ}, a_j), g_j = (Q/q_j)
 * [(Q/q_j)^-1]_{q_j}; randomness from Philox4x64-10 keyed by (seed, purpose).
 * Same key set for SecureMod and bit-level types (Sec. 3.2). */
int bfhe_keygen(bfhe_ctx* ctx, uint64_t seed, void* stream);

/* Copy keys out (device buffers), in coefficient form:
 *   sk : int64 [N] in {-1, 0, 1}
 *   pk : uint64 [2][L][N]
 *   rlk: uint64 [L][2][L+alpha][N]  (digit j, component (b_j, a_j), limbs
 *        over q_0..q_{L-1}, p_0..p_{alpha-1})
 * Any pointer may be NULL to skip that key. */
int bfhe_export_keys(bfhe_ctx* ctx, int64_t* sk, uint64_t* pk, uint64_t* rlk, void* stream);

/* Encrypt n slot vectors (slots uint64 [n][N], each < t) into ct_out
 * [n][2][L][N]: (Delta m + pk0 u + e1, pk1 u + e2) mod Q with m the batch
 * encoding (slot j = m(zeta^(2j+1)) mod t, Sec. 2.3) and u, e1, e2 drawn
 * from Philox4x64-10 with key (seed, purpose) and poly index = batch index.
 * BFHE_EINVAL at t = 2 (no slots). */
int bfhe_encrypt(bfhe_ctx* ctx, const uint64_t* slots, size_t n, uint64_t seed,
                 uint64_t* ct_out, void* stream);

/* Decrypt n ciphertexts into slots uint64 [n][N]: m = [round(t [c0 + c1 s]_Q
 * / Q)]_t computed exactly, then decoded.  BFHE_EINVAL at t = 2. */
int bfhe_decrypt(bfhe_ctx* ctx, const uint64_t* ct, size_t n, uint64_t* slots_out, void* stream);

/* Coefficient encoding (any t; the only encoding at t = 2): encrypt n
 * plaintext polynomials coeffs uint64 [n][N] (coefficient k of polynomial
 * i at [i][k], each < t; larger values are a precondition violation that
 * encrypts the unreduced value, not an error) with the same randomness as
 * bfhe_encrypt; a product of two such ciphertexts encrypts the negacyclic
 * product of the polynomials mod t.  Decrypt returns the coefficients
 * [round(t [c0 + c1 s]_Q / Q)]_t into coeffs_out [n][N]. */
int bfhe_encrypt_poly(bfhe_ctx* ctx, const uint64_t* coeffs, size_t n, uint64_t seed, uint64_t* ct_out,
                      void* stream);
int bfhe_decrypt_poly(bfhe_ctx* ctx, const uint64_t* ct, size_t n, uint64_t* coeffs_out, void* stream);

/* Linear operations (Sec. 3.1 uses them in every gate; Listing 5 is only
 * additions).  out may alias a or b.  A public constant c (< t) enters as
 * the trivial ciphertext (Delta c, 0). */
int bfhe_add(bfhe_ctx* ctx, const uint64_t* a, const uint64_t* b, uint64_t* out, size_t n, void* stream);
int bfhe_sub(bfhe_ctx* ctx, const uint64_t* a, const uint64_t* b, uint64_t* out, size_t n, void* stream);
int bfhe_add_const(bfhe_ctx* ctx, const uint64_t* a, uint64_t c, uint64_t* out, size_t n, void* stream);
int bfhe_sub_const(bfhe_ctx* ctx, const uint64_t* a, uint64_t c, uint64_t* out, size_t n, void* stream);
int bfhe_const_sub(bfhe_ctx* ctx, uint64_t c, const uint64_t* a, uint64_t* out, size_t n, void* stream);
/* Multiply both components by the integer c (< t). */
int bfhe_mul_scalar(bfhe_ctx* ctx, const uint64_t* a, uint64_t c, uint64_t* out, size_t n, void* stream);
/* Slot-wise product with public vectors: plain uint64 [n][N] slot values
 * (< t), encoded to [0, t)^N coefficients; out = (c0 pt, c1 pt) mod Q. */
int bfhe_mul_plain(bfhe_ctx* ctx, const uint64_t* a, const uint64_t* plain, uint64_t* out, size_t n,
                   void* stream);

/* Ciphertext product with relinearisation, exact FV: lift inputs to the
 * centred range, tensor over Z (computed in RNS over Q and the auxiliary
 * base), round(t d / Q) mod Q, then key switching of d2 with the digit
 * gadget and rounding division by P.  out must not alias a or b.
 * a[i] * b[i] for i < n. */
int bfhe_mul_relin(bfhe_ctx* ctx, const uint64_t* a, const uint64_t* b, uint64_t* out, size_t n,
                   void* stream);

/* Homomorphic gates over encrypted bits (Sec. 3.1): AND = xy,
 * NAND = 1 - xy, OR = x + y - xy, NOR = 1 - OR, XOR = x + y - 2xy,
 * XNOR = 1 - XOR, NOT = 1 - x, MUX(x, y, z) = x (y - z) + z.
 * y is ignored for NOT; z is used by MUX only.  One multiply per gate
 * (none for NOT).  At t = 2 XOR = x + y and XNOR = 1 - (x + y), without a
 * multiply (Sec. 3.1).  out must not alias the inputs of a multiplying
 * gate. */
enum { BFHE_AND = 0, BFHE_OR = 1, BFHE_XOR = 2, BFHE_NAND = 3, BFHE_NOR = 4, BFHE_XNOR = 5,
       BFHE_NOT = 6, BFHE_MUX = 7 };
int bfhe_bit_gate(bfhe_ctx* ctx, int gate, const uint64_t* x, const uint64_t* y, const uint64_t* z,
                  uint64_t* out, size_t n, void* stream);

/* A levelised gate list over one wire array: all multiplying entries of one
 * circuit depth level share one batched multiply.  Gate entries run the
 * Sec. 3.1 equations as written at every t (a netlist for t = 2 writes its
 * XORs as linear entries).  wires: uint64
 * [n_wires][n][2][L][N] (n slot-packed ciphertexts per wire); table: DEVICE
 * int32 [n_gates][5] = (op, x, y, z, out) wire indices, the n_mul entries
 * with a multiply first.  op is a gate above (BFHE_AND .. BFHE_MUX, with the
 * Sec. 3.1 equation), BFHE_OP_MUL (out = x * y, relinearised) or
 * BFHE_OP_LIN | code << 8, a linear node out = cc Delta + cx x + cy y + cz z
 * with code = ((cc+2) 5 + (cx+2)) 25 + (cy+2) 5 + (cz+2), coefficients in
 * -2..2 (no multiply; place after the n_mul entries).  No entry may read a
 * wire that another entry of the same call writes; wire indices must be
 * < n_wires (not checked on the device).  Counts only the multiplies.
 * Needs no host synchronisation: capturable in a CUDA graph once scratch is
 * reserved (bfhe_reserve) and one call of the same shape has run. */
enum { BFHE_OP_MUL = 8, BFHE_OP_LIN = 9 };
int bfhe_gate_level(bfhe_ctx* ctx, uint64_t* wires, size_t n_wires, size_t n, const int32_t* table,
                    size_t n_gates, size_t n_mul, void* stream);

/* SecureUint<s> -> SecureMod (Sec. 3.2.1, Listing 5): Horner's scheme
 * r = v[s-1]; r += r + v[i] for i = s-2 .. 0, i.e. sum_i 2^i v[i] mod Q.
 * bits: uint64 [s][n][2][L][N] (bit 0 first); out [n][2][L][N].
 * 2(s-1) additions, no multiplies. */
int bfhe_bits_to_mod(bfhe_ctx* ctx, const uint64_t* bits, uint32_t s, uint64_t* out, size_t n,
                     void* stream);

/* SecureMod -> SecureUint<s> (Sec. 3.2.3, Eq. 2, Listings 7-8): for every
 * candidate c in [c_lo, c_hi], eq_c = 1 - (x - c)^(t-1) by the square-and-
 * multiply recursion of Listing 7; then
 *   mode BFHE_PAPER : bit k += AND(trivial(bit k of c), eq_c)  (s multiplies
 *                     per candidate: the count the paper states),
 *   mode BFHE_SELECT: bit k += eq_c where bit k of c is 1 (no multiply).
 * x: [n][2][L][N]; bits_out: [s][n][2][L][N].  Chains of all candidates run
 * batched. */
enum { BFHE_PAPER = 0, BFHE_SELECT = 1 };
int bfhe_mod_to_bits(bfhe_ctx* ctx, const uint64_t* x, uint32_t s, uint64_t c_lo, uint64_t c_hi, int mode,
                     uint64_t* bits_out, size_t n, void* stream);

/* SecureInt<s> -> SecureMod (Sec. 3.2.2, Eq. 1, Listing 6): bits hold the
 * two's complement of v (bit s-1 the sign); pos = Horner(bits) as in
 * bfhe_bits_to_mod, neg = pos + (t - 2^s), and
 *   out = isNeg * neg + (1 - isNeg) * pos,   isNeg = bits[s-1],
 * an encryption of v mod t.  Needs 1 <= s and 2^s <= t, else BFHE_EINVAL.
 * bits: uint64 [s][n][2][L][N] (bit 0 first); out: [n][2][L][N] (may alias
 * bits).  2 multiplies (run as one batched multiply of 2n) and 2s + 1
 * additions/subtractions per ciphertext; scratch from the context arena. */
int bfhe_sint_to_mod(bfhe_ctx* ctx, const uint64_t* bits, uint32_t s, uint64_t* out, size_t n, void* stream);

/* SecureMod -> SecureInt<s> (Sec. 3.2.4, Listing 9): pos = the conversion
 * of bfhe_mod_to_bits applied to x over candidates [pos_lo, pos_hi];
 * neg = the same conversion of (2^s - t) + x (SecureMod addition, mod t)
 * over [neg_lo, neg_hi]; isNeg = pos[s-1]; bit k of the result is
 *   isNeg * neg[k] + (1 - isNeg) * pos[k].
 * This is the listing's arithmetic: where (2^s - t) + x wraps mod t the
 * result is not the two's complement of x - t (Eq. 3 adds in bit-level
 * arithmetic instead).  Needs 2^s >= t, s <= 63, both ranges inside
 * [0, t), mode BFHE_PAPER or BFHE_SELECT, else BFHE_EINVAL.
 * x: [n][2][L][N]; bits_out: [s][n][2][L][N] (may alias x).
 * Multiplies: the two conversions' plus 2s per ciphertext (one batched
 * multiply of 2sn). */
int bfhe_mod_to_sint(bfhe_ctx* ctx, const uint64_t* x, uint32_t s, uint64_t pos_lo, uint64_t pos_hi,
                     uint64_t neg_lo, uint64_t neg_hi, int mode, uint64_t* bits_out, size_t n, void* stream);

/* Allocation-free variant of bfhe_mul_relin.  The paper has no counterpart:
 * this is for callers that cannot allocate device memory at call time --
 * deployments that reserve all device memory at start-up and forbid
 * allocation afterwards, and host code whose hot path must not enter an
 * allocator or wait for the device-wide synchronisation that growing the
 * context's scratch arena takes.  Same arguments and result as bfhe_mul_relin (bit
 * identical), but the multiply's scratch is a fixed static device array of
 * BFHE_NOALLOC_SCRATCH_BYTES (32 MiB) instead of the context's arena; the
 * call makes no cudaMalloc, cudaFree or other allocating call.
 *  - Size limit: n ciphertexts need n x (4(L+K) + 3L + L(L+alpha) +
 *    2(L+alpha)) N x 8 bytes of scratch; larger n is rejected with
 *    BFHE_EINVAL and a message giving the maximum (at N = 16384, L = 8 one
 *    ciphertext per call; at N = 4096, L = 2, 26).
 *  - The context's device must be the current device.  The first call on a
 *    device looks up the array's device address (cudaGetSymbolAddress) and
 *    caches it; make that first call before any stream capture.
 *  - Every call on a device shares the one array and leaves its contents
 *    behind; no part of it needs to start at zero (every word is written
 *    before it is read).  Calls that overlap on the GPU (other streams, other
 *    threads) race on it: serialise them.
 *  - Every GPU that loads this library keeps the array until the process
 *    exits. */
#define BFHE_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
int bfhe_mul_relin_noalloc(bfhe_ctx* ctx, const uint64_t* a, const uint64_t* b, uint64_t* out, size_t n,
                           void* stream);

/* Power by the recursion of Listing 7 (floor(log2 e) + w(e) - 1 multiplies):
 * out[i] = x[i]^e, e >= 1.  out must not alias x. */
int bfhe_pow(bfhe_ctx* ctx, const uint64_t* x, uint64_t e, uint64_t* out, size_t n, void* stream);

/* Operation counters kept with the paper's accounting (Table 1 counts
 * ciphertext add / mul / sub): out[0] = additions, out[1] = subtractions,
 * out[2] = ciphertext multiplies, out[3] = plaintext multiplies.  Reset
 * when reset != 0 (after reading). */
int bfhe_op_counts(bfhe_ctx* ctx, uint64_t out[4], int reset);

/* Negacyclic NTT of a batch of polynomials in place, for tests and tools:
 * data uint64 [n_polys][n_limbs][N] over the first n_limbs data primes
 * (n_limbs <= L); forward maps coefficients to the library's internal
 * evaluation order, inverse maps back (inputs canonical). */
int bfhe_ntt(bfhe_ctx* ctx, uint64_t* data, size_t n_polys, uint32_t n_limbs, int inverse, void* stream);

/* NTT block shape for ring degree 2^logN and one direction (inverse != 0): a
 * CTA transforms 2^log_m words (log_m = logN, or logN - 1 with the limb split
 * over two CTAs), each thread holding 2^log_e of them.  log_m = 0 only reads
 * the current shape into *cur_m, *cur_e (may be NULL).  Process-wide; used
 * by the autotuner.  Shapes: log_m in [10, 14], log_e in [3, 5] (>= 4 at
 * log_m = 14). */
int bfhe_ntt_config(uint32_t logN, int inverse, uint32_t log_m, uint32_t log_e, uint32_t* cur_m, uint32_t* cur_e);

/* Measurement support.  While profiling is on, every launch of the kernel
 * classes below is bracketed by CUDA events on its own stream;
 * bfhe_profile_read synchronises on the last event and returns, per class,
 * the summed device time in ms, the number of launches, (work_out, may be
 * NULL) the algorithmic 64-bit modular multiplies those launches performed
 * and (bytes_out, may be NULL) their algorithmic DRAM bytes, every operand
 * read and every result written once (arrays of BFHE_K_COUNT), then clears
 * the record.  Modmul counts: NTT (N/2) log2 N per limb; modup per
 * coefficient L(L-1)/2 + K(L-1); scale per coefficient of each of 3 polys
 * 2L + 3K + L(L-1)/2 + K(L-1) + K(K-1)/2 + L(K-1) (both the exact
 * algorithm's count, also when the fast extension ran); tensor 4 per limb
 * word; inner 2L per word of the Q u P limbs; moddown per coefficient of
 * each of 2 polys alpha(alpha-1)/2 + L alpha + L + alpha (with the inverse
 * transform's twist).  Bytes: NTT 16N per limb; modup 8(2L + K) per
 * coefficient of an input poly; scale 8(2L + K) per coefficient of each of
 * 3 polys; tensor 56 (squaring 40) per limb word of Q u B; inner 8(L + 2)
 * per word of Q u P per ciphertext plus the key's 16L once per launch;
 * moddown 8(3L + alpha) per coefficient of each of 2 polys. */
enum { BFHE_K_NTT_FWD = 0, BFHE_K_NTT_INV = 1, BFHE_K_MODUP = 2, BFHE_K_TENSOR = 3, BFHE_K_SCALE = 4,
       BFHE_K_INNER = 5, BFHE_K_MODDOWN = 6, BFHE_K_COUNT = 7 };
int bfhe_profile(bfhe_ctx* ctx, int enable);
int bfhe_profile_read(bfhe_ctx* ctx, double* ms_out, uint64_t* launches_out, double* work_out, double* bytes_out);

/* Number of kernels this library has launched in this process so far. */
uint64_t bfhe_launch_count(void);

/* Integer-pipe probe: a kernel of independent 64-bit Shoup modular-multiply
 * chains on every SM (grid = SMs x 4 CTAs of 256 threads, 8 chains per
 * thread, `iters` steps each).  *modmul_per_s = modmuls / device time. */
int bfhe_probe_modmul(int device, uint32_t iters, double* modmul_per_s, void* stream);

/* Message of the last failed call on this thread (static storage). */
const char* bfhe_strerror(int code);
const char* bfhe_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* BFHE_H */
