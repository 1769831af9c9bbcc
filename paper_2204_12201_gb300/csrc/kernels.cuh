// kernels.cuh -- launchers of the elementwise, sampling and RNS kernels (kernels.cu).
#pragma once
#include "common.cuh"

// Philox4x64-10 samplers (see kernels.cu for the counter layout)
int launch_sample_uniform(const bfhe_ctx* ctx, u64* out, int n_polys, int n_limbs, LimbMap map, u64 seed,
                          u64 purpose, u64 poly_base, cudaStream_t st);
int launch_sample_small(const bfhe_ctx* ctx, i64* out, int n_polys, u64 seed, u64 purpose, u64 poly_base,
                        int cbd, cudaStream_t st);
// signed small polys [n][N] -> residues [n][n_limbs][N]
int launch_spread(const bfhe_ctx* ctx, const i64* in, u64* out, int n_polys, int n_limbs, LimbMap map,
                  cudaStream_t st);

// out[c][p][l][k] = A[..] * B[..] * 2^-64 mod q (REDC), strides in words (0 = broadcast)
struct PwStrides {
    size_t a_cs, a_ps, b_cs, b_ps, o_cs, o_ps;
};
int launch_pointwise(const bfhe_ctx* ctx, const u64* A, const u64* B, u64* out, int n, int polys, int n_limbs,
                     LimbMap map, PwStrides s, cudaStream_t st);

// exact multiply pipeline pieces
// slots = 4 (a0 a1 b0 b1) or 2 (squaring: a0 a1 only)
int launch_modup(const bfhe_ctx* ctx, const u64* A, const u64* B, u64* X, int n, int slots, cudaStream_t st);
int launch_tensor(const bfhe_ctx* ctx, u64* X, int n, int square, cudaStream_t st);
// tmp: [n][3][K][N] words for the two-pass form (10 or more data primes), or null for one pass
int launch_scale(const bfhe_ctx* ctx, const u64* X, u64* C3, int n, cudaStream_t st, u64* tmp = nullptr);
int launch_inner(const bfhe_ctx* ctx, const u64* Dg, u64* W, int n, cudaStream_t st);
int launch_moddown(const bfhe_ctx* ctx, const u64* W, const u64* C3, u64* out, int n, cudaStream_t st);

// decrypt: V = [c1 s]_Q (coefficient form), ct -> M = [round(t (c0 + c1 s) / Q)]_t
int launch_dec_finish(const bfhe_ctx* ctx, const u64* V, const u64* ct, u64* M, int n, cudaStream_t st);
// encode / decode permutations (slot j <-> evaluation position brv(j))
int launch_permute(const bfhe_ctx* ctx, const u64* in, u64* out, int n, int scatter, cudaStream_t st);
// encrypt epilogue: ct[c][0] += Delta m + e1, ct[c][1] += e2
int launch_enc_finish(const bfhe_ctx* ctx, u64* ct, const u64* M, const i64* e1, const i64* e2, int n,
                      cudaStream_t st);
// keygen epilogues
int launch_neg_add_small(const bfhe_ctx* ctx, const u64* as, const i64* e, u64* out, int n_polys, int n_limbs,
                         LimbMap map, const u64* s2, int gadget, cudaStream_t st);

// linear combination: out = cc*Delta*[c0, coeff 0] + cx x + cy y + cz z + cp p (coefficients in -2..2)
struct LinCoef {
    int cc, cx, cy, cz, cp;
};
int launch_lincomb(const bfhe_ctx* ctx, u64* out, const u64* x, const u64* y, const u64* z, const u64* p,
                   LinCoef cf, u64 cval, size_t n, cudaStream_t st);
int launch_mul_scalar(const bfhe_ctx* ctx, const u64* a, u64 c, u64* out, size_t n, cudaStream_t st);
int launch_horner(const bfhe_ctx* ctx, const u64* bits, uint32_t s, u64* out, size_t n, cudaStream_t st);
// gate table helpers
int launch_gather(const bfhe_ctx* ctx, u64* dst, const u64* wires, size_t n, const int32_t* table, int n_gates,
                  int field, int sub_field, cudaStream_t st);
int launch_gate_epilogue(const bfhe_ctx* ctx, u64* wires, size_t n, const int32_t* table, int n_gates,
                         const u64* prod, int n_mul, cudaStream_t st);
// mod_to_bits helpers; the candidate base is c_base, or the device word *cbp when cbp is not null
// (a tile replayed from a CUDA graph reads its base from device memory)
int launch_trivial_bits(const bfhe_ctx* ctx, u64* out, uint32_t s, u64 c_base, const u64* cbp, int C, size_t n,
                        cudaStream_t st);
int launch_accumulate(const bfhe_ctx* ctx, u64* bits, const u64* src, uint32_t s, u64 c_base, const u64* cbp, int C,
                      size_t n, int select, cudaStream_t st);
int launch_sub_const_chains(const bfhe_ctx* ctx, const u64* x, u64* out, u64 c_base, const u64* cbp, int C, size_t n,
                            cudaStream_t st);
int launch_set_word(u64* w, u64 v, cudaStream_t st);
int launch_probe_modmul(u64* out, int blocks, int threads, uint32_t iters, u64 q, u64 w, u64 ws, cudaStream_t st);
