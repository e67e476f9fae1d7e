/* A plain C program on the C ABI alone (no Python): embed a message into a
 * cover in device memory with fused statistics, extract it back, and check
 * the round trip, the untouched high bits and the changed-byte count on the
 * host.  Built and run by tests/test_gpu_c_abi.py. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime_api.h>

#include "stego.h"

#define CHECK(x)                                                               \
    do {                                                                       \
        if (!(x)) {                                                            \
            fprintf(stderr, "check failed: %s (line %d)\n", #x, __LINE__);    \
            return 1;                                                          \
        }                                                                      \
    } while (0)

static uint64_t rng = 0x9E3779B97F4A7C15ull;
static uint8_t next_byte(void)
{
    rng ^= rng << 13;
    rng ^= rng >> 7;
    rng ^= rng << 17;
    return (uint8_t)(rng >> 32);
}

int main(void)
{
    const uint64_t C = 3u * 1024u * 1024u + 40u;
    uint64_t cap = 0;
    CHECK(stego_capacity(C, NULL, STEGO_HEADER_BE32, &cap) == STEGO_OK);
    const uint64_t m = cap - 3u;
    uint8_t *cover = malloc(C), *stego = malloc(C), *msg = malloc(m), *out = malloc(cap);
    CHECK(cover && stego && msg && out);
    for (uint64_t i = 0; i < C; ++i)
        cover[i] = next_byte();
    for (uint64_t i = 0; i < m; ++i)
        msg[i] = next_byte();

    uint8_t *d_cover, *d_stego, *d_msg, *d_out;
    stego_result *d_res, *d_res2;
    CHECK(cudaMalloc((void **)&d_cover, C) == cudaSuccess);
    CHECK(cudaMalloc((void **)&d_stego, C) == cudaSuccess);
    CHECK(cudaMalloc((void **)&d_msg, m) == cudaSuccess);
    CHECK(cudaMalloc((void **)&d_out, cap) == cudaSuccess);
    CHECK(cudaMalloc((void **)&d_res, sizeof(stego_result)) == cudaSuccess);
    CHECK(cudaMalloc((void **)&d_res2, sizeof(stego_result)) == cudaSuccess);
    CHECK(cudaMemcpy(d_cover, cover, C, cudaMemcpyHostToDevice) == cudaSuccess);
    CHECK(cudaMemcpy(d_msg, msg, m, cudaMemcpyHostToDevice) == cudaSuccess);

    CHECK(stego_embed(d_cover, d_stego, C, d_msg, m, NULL,
                      STEGO_HEADER_BE32 | STEGO_FUSE_STATS, d_res, NULL) == STEGO_OK);
    CHECK(stego_extract(d_stego, C, d_out, cap, 0, NULL, STEGO_HEADER_BE32, d_res2,
                        NULL) == STEGO_OK);
    /* host-detected errors return at once */
    CHECK(stego_embed(d_cover, d_stego, C, d_msg, cap + 1u, NULL, STEGO_HEADER_BE32, NULL,
                      NULL) == STEGO_E_CAPACITY);
    CHECK(cudaDeviceSynchronize() == cudaSuccess);

    stego_result r, r2;
    CHECK(cudaMemcpy(&r, d_res, sizeof r, cudaMemcpyDeviceToHost) == cudaSuccess);
    CHECK(cudaMemcpy(&r2, d_res2, sizeof r2, cudaMemcpyDeviceToHost) == cudaSuccess);
    CHECK(cudaMemcpy(stego, d_stego, C, cudaMemcpyDeviceToHost) == cudaSuccess);
    CHECK(cudaMemcpy(out, d_out, cap, cudaMemcpyDeviceToHost) == cudaSuccess);

    CHECK(r.status == STEGO_OK && r.msg_bytes == m);
    CHECK(r2.status == STEGO_OK && r2.msg_bytes == m);
    CHECK(memcmp(out, msg, m) == 0);
    uint64_t changed = 0;
    for (uint64_t i = 0; i < C; ++i) {
        CHECK(((stego[i] ^ cover[i]) & 0xFEu) == 0);
        changed += stego[i] != cover[i];
    }
    CHECK(r.changed == changed && r.sse == changed);
    printf("c abi round trip ok: %llu cover bytes, %llu message bytes, %llu changed (%s)\n",
           (unsigned long long)C, (unsigned long long)m, (unsigned long long)changed,
           stego_strerror(STEGO_OK));
    cudaFree(d_cover);
    cudaFree(d_stego);
    cudaFree(d_msg);
    cudaFree(d_out);
    cudaFree(d_res);
    cudaFree(d_res2);
    free(cover);
    free(stego);
    free(msg);
    free(out);
    return 0;
}
