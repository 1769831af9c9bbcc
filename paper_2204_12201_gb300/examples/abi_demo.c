/* The C ABI used from plain C, with no Python and no PyTorch: key generation,
 * encryption of two slot vectors, one relinearised multiply, the SecureMod ->
 * SecureUint -> SecureMod round trip of the bridge (Eq. 2, Listings 5 and 8)
 * on small values, decryption, and a check against plain arithmetic mod t.
 * Device memory comes from cudaMalloc; everything runs on one stream.
 *
 * Build (what paper_2204_12201_gb300.build.build_demo() runs):
 *   gcc -O2 -I include -I /usr/local/cuda/include abi_demo.c
 *       -L paper_2204_12201_gb300/_lib -lbfhe -L /usr/local/cuda/lib64 -lcudart
 * Prints "abi demo ok" and exits 0 on success, prints the failure and exits 1
 * otherwise. */
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "bfhe.h"

#define CK(x)                                                                            \
    do {                                                                                 \
        int rc_ = (x);                                                                   \
        if (rc_ != BFHE_OK) {                                                            \
            fprintf(stderr, "%s failed: %s (%s)\n", #x, bfhe_strerror(rc_), bfhe_last_error()); \
            return 1;                                                                    \
        }                                                                                \
    } while (0)
#define CU(x)                                                                            \
    do {                                                                                 \
        cudaError_t e_ = (x);                                                            \
        if (e_ != cudaSuccess) {                                                         \
            fprintf(stderr, "%s failed: %s\n", #x, cudaGetErrorString(e_));              \
            return 1;                                                                    \
        }                                                                                \
    } while (0)

int main(void) {
    /* the bridge's Fermat chains are 16 squarings deep: 16 data primes keep them decryptable */
    const uint32_t N = 32768, L = 16, S_BITS = 4;
    const uint64_t t = 65537;
    bfhe_params prm = {N, L, 2, 50, t};
    bfhe_ctx* ctx = NULL;
    CU(cudaSetDevice(0));
    CK(bfhe_ctx_create(&prm, 0, &ctx));
    cudaStream_t st;
    CU(cudaStreamCreate(&st));
    CK(bfhe_keygen(ctx, 1, st));

    const size_t ct_words = 2 * (size_t)L * N;
    uint64_t* h_slots = (uint64_t*)malloc(3 * N * sizeof(uint64_t));
    uint64_t* h_out = (uint64_t*)malloc(3 * N * sizeof(uint64_t));
    for (uint32_t j = 0; j < N; ++j) {
        h_slots[j] = (j * 2654435761u) % t;                  /* a */
        h_slots[N + j] = (j * 40503u + 17) % t;              /* b */
        h_slots[2 * N + j] = j % (1u << S_BITS);             /* x < 2^s for the bridge */
    }
    uint64_t *d_slots, *d_ct, *d_prod, *d_bits, *d_back, *d_out;
    CU(cudaMalloc((void**)&d_slots, 3 * N * sizeof(uint64_t)));
    CU(cudaMalloc((void**)&d_ct, 3 * ct_words * sizeof(uint64_t)));
    CU(cudaMalloc((void**)&d_prod, ct_words * sizeof(uint64_t)));
    CU(cudaMalloc((void**)&d_bits, S_BITS * ct_words * sizeof(uint64_t)));
    CU(cudaMalloc((void**)&d_back, ct_words * sizeof(uint64_t)));
    CU(cudaMalloc((void**)&d_out, 3 * N * sizeof(uint64_t)));
    CU(cudaMemcpyAsync(d_slots, h_slots, 3 * N * sizeof(uint64_t), cudaMemcpyHostToDevice, st));

    CK(bfhe_encrypt(ctx, d_slots, 3, 7, d_ct, st));                         /* three ciphertexts */
    CK(bfhe_mul_relin(ctx, d_ct, d_ct + ct_words, d_prod, 1, st));           /* a * b */
    CK(bfhe_mod_to_bits(ctx, d_ct + 2 * ct_words, S_BITS, 0, (1u << S_BITS) - 1, BFHE_SELECT, d_bits, 1, st));
    CK(bfhe_bits_to_mod(ctx, d_bits, S_BITS, d_back, 1, st));               /* back to SecureMod */
    CK(bfhe_decrypt(ctx, d_prod, 1, d_out, st));
    CK(bfhe_decrypt(ctx, d_back, 1, d_out + N, st));
    CK(bfhe_decrypt(ctx, d_bits + 2 * ct_words, 1, d_out + 2 * N, st));     /* bit 2 of x */
    CU(cudaMemcpyAsync(h_out, d_out, 3 * N * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    CK(bfhe_check(ctx, st, NULL));                                          /* synchronises */

    int bad = 0;
    for (uint32_t j = 0; j < N && bad < 5; ++j) {
        const uint64_t want_prod = (h_slots[j] * h_slots[N + j]) % t;
        const uint64_t x = h_slots[2 * N + j];
        if (h_out[j] != want_prod || h_out[N + j] != x || h_out[2 * N + j] != ((x >> 2) & 1)) {
            fprintf(stderr, "slot %u: got %llu %llu %llu\n", j, (unsigned long long)h_out[j],
                    (unsigned long long)h_out[N + j], (unsigned long long)h_out[2 * N + j]);
            ++bad;
        }
    }
    cudaFree(d_slots);
    cudaFree(d_ct);
    cudaFree(d_prod);
    cudaFree(d_bits);
    cudaFree(d_back);
    cudaFree(d_out);
    free(h_slots);
    free(h_out);
    cudaStreamDestroy(st);
    bfhe_ctx_destroy(ctx);
    if (bad) return 1;
    printf("abi demo ok\n");
    return 0;
}
