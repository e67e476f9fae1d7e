// ballot.cu -- the one-bit stream extraction (Section VII step 6) with the
// message packed by warp ballots: lane l of a warp loads stego byte
// base + 32w + l, and one __ballot_sync of the 32 LSBs is message word w
// (bit l = stego byte 32w + l; bit-reversed, its bytes are message bytes
// 4w..4w+3 most significant bit first).  The same results as extract_vec
// (stream1.cu), which gives each lane 16 consecutive stego bytes with one
// 128-bit load and packs their LSBs with one multiply per four bytes: a
// ballot gathers across lanes, so its lanes must hold consecutive bytes, and
// byte loads move 32 bytes per warp instruction where 128-bit loads move 512.
// Kept as stego_extract_ballot for that comparison.
#include "s1_device.cuh"

namespace stego {
namespace {

constexpr int kWordsPerWarp = 4; // message words per warp per iteration, loads first

__global__ void __launch_bounds__(512) extract_ballot(s1::ExtractArgs a)
{
    grid_dependency_wait(); // launched dependent: nothing is touched before
    allow_dependents();
    s1::ExtractView x;
    if (s1::extract_prologue(a, x) != STEGO_OK)
        return;
    const uint8_t *src = x.st + x.base;
    const uint64_t nwords = x.len >> 2; // whole message words
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const bool msg_w4 = ((uintptr_t)x.msg & 3u) == 0;
    for (uint64_t w0 = warp * kWordsPerWarp; w0 < nwords; w0 += nwarps * kWordsPerWarp) {
        uint32_t b[kWordsPerWarp];
#pragma unroll
        for (int i = 0; i < kWordsPerWarp; ++i) {
            const uint64_t w = w0 + i;
            b[i] = w < nwords ? (uint32_t)__ldcs(src + 32u * w + lane) : 0u;
        }
        uint32_t bal[kWordsPerWarp];
#pragma unroll
        for (int i = 0; i < kWordsPerWarp; ++i)
            bal[i] = __ballot_sync(0xFFFFFFFFu, b[i] & 1u);
        if (lane < (uint32_t)kWordsPerWarp && w0 + lane < nwords) {
            uint32_t v = bal[0];
#pragma unroll
            for (int i = 1; i < kWordsPerWarp; ++i)
                if (lane == (uint32_t)i)
                    v = bal[i];
            const uint32_t word = __byte_perm(__brev(v), 0u, 0x0123u);
            uint8_t *dst = x.msg + 4u * (w0 + lane);
            if (msg_w4) {
                *reinterpret_cast<uint32_t *>(dst) = word;
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    dst[j] = (uint8_t)(word >> (8 * j));
            }
        }
    }
    // message bytes after the last whole word
    if (blockIdx.x == 0 && threadIdx.x < (uint32_t)(x.len & 3u))
        s1::extract_one(x, (nwords << 2) + threadIdx.x);
}

} // namespace

cudaError_t s1_extract_ballot(const uint8_t *st, uint64_t C, uint8_t *msg, uint64_t cap,
                              uint64_t raw_len, bool header, stego_result *res, const Shape &sh,
                              cudaStream_t s)
{
    s1::ExtractArgs a;
    a.st = st;
    a.C = C;
    a.msg = msg;
    a.cap = cap;
    a.raw_len = raw_len;
    a.header = header ? 1u : 0u;
    a.msg_even = ((uintptr_t)msg & 1u) == 0;
    a.res = res;
    uint64_t max_len = raw_len;
    if (header) {
        const uint64_t fit = C >= 32 ? (C - 32) / 8 : 0;
        max_len = fit < cap ? fit : cap;
    }
    a.max_vec = max_len >> 1;
    const void *k = (const void *)extract_ballot;
    const uint64_t words = max_len >> 2;
    const int T = sh.threads;
    const int grid = persistent_grid(k, T, 0, sh.ctas_per_sm, words ? words : 1,
                                     (uint64_t)(T / 32) * kWordsPerWarp);
    void *args[] = {&a};
    return launch_dependent(k, dim3(grid), dim3(T), args, 0, s);
}

} // namespace stego
