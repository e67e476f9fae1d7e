/* A plain C program on the C ABI alone (no Python): embed a message into a
 * cover in device memory with fused statistics, extract it back, and check
 * the round trip, the untouched high bits and the changed-byte count on the
 * host; then the same cover from pinned host memory through a host
 * pipeline (with a read-back), and a byte-volume partition.  Built and run
 * by tests/test_gpu_c_abi.py. */
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
    /* the same cover from pinned host memory through a host pipeline: two
     * jobs (one with a read-back), results and outputs on the host */
    stego_pipeline_config pc;
    memset(&pc, 0, sizeof pc);
    pc.slots = 2;
    pc.max_descs = 4;
    pc.slot_bytes = C + 2u * m + 4096u;
    pc.mode = STEGO_PIPE_STAGED;
    const uint64_t arena_bytes = stego_pipeline_arena_bytes(&pc);
    CHECK(arena_bytes > 0);
    void *d_arena;
    CHECK(cudaMalloc(&d_arena, arena_bytes) == cudaSuccess);
    stego_pipeline *pipe = NULL;
    CHECK(stego_pipeline_create(&pc, d_arena, arena_bytes, &pipe) == STEGO_OK);
    uint8_t *h_cover, *h_msg, *h_stego0, *h_stego1, *h_back;
    CHECK(cudaHostAlloc((void **)&h_cover, C, cudaHostAllocDefault) == cudaSuccess);
    CHECK(cudaHostAlloc((void **)&h_msg, m, cudaHostAllocDefault) == cudaSuccess);
    CHECK(cudaHostAlloc((void **)&h_stego0, C, cudaHostAllocDefault) == cudaSuccess);
    CHECK(cudaHostAlloc((void **)&h_stego1, C, cudaHostAllocDefault) == cudaSuccess);
    CHECK(cudaHostAlloc((void **)&h_back, m, cudaHostAllocDefault) == cudaSuccess);
    memcpy(h_cover, cover, C);
    memcpy(h_msg, msg, m);
    stego_host_job jobs[2];
    memset(jobs, 0, sizeof jobs);
    for (int j = 0; j < 2; ++j) {
        jobs[j].cover = h_cover;
        jobs[j].stego = j ? h_stego1 : h_stego0;
        jobs[j].msg = h_msg;
        jobs[j].readback = j ? h_back : NULL;
        jobs[j].cover_bytes = C;
        jobs[j].msg_bytes = m;
        jobs[j].flags = STEGO_HEADER_BE32;
    }
    stego_result hr[2], hb[2];
    CHECK(stego_pipeline_embed(pipe, jobs, 2, hr, hb, STEGO_FUSE_STATS) == STEGO_OK);
    for (int j = 0; j < 2; ++j)
        CHECK(hr[j].status == STEGO_OK && hr[j].msg_bytes == m && hr[j].changed == changed);
    CHECK(memcmp(h_stego0, stego, C) == 0 && memcmp(h_stego1, stego, C) == 0);
    CHECK(hb[1].status == STEGO_OK && hb[1].msg_bytes == m && memcmp(h_back, msg, m) == 0);
    CHECK(stego_pipeline_destroy(pipe) == STEGO_OK);

    /* a batch split among three GPUs by byte volume (host only) */
    const uint64_t sizes[6] = {5, 9, 1, 7, 3, 3};
    uint32_t rank_of[6];
    uint64_t rank_bytes[3];
    CHECK(stego_partition(sizes, 6, 3, rank_of, rank_bytes) == STEGO_OK);
    CHECK(rank_bytes[0] + rank_bytes[1] + rank_bytes[2] == 28);
    CHECK(rank_of[1] == 0 && rank_of[3] == 1 && rank_of[0] == 2);
    CHECK(stego_partition(sizes, 6, 0, rank_of, NULL) == STEGO_E_INVAL);

    printf("c abi round trip ok: %llu cover bytes, %llu message bytes, %llu changed (%s)\n",
           (unsigned long long)C, (unsigned long long)m, (unsigned long long)changed,
           stego_strerror(STEGO_OK));
    cudaFreeHost(h_cover);
    cudaFreeHost(h_msg);
    cudaFreeHost(h_stego0);
    cudaFreeHost(h_stego1);
    cudaFreeHost(h_back);
    cudaFree(d_arena);
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
