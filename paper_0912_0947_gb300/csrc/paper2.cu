// paper2.cu -- Sections VI and VII as printed: two bits per cover byte in one
// colour plane, the message divided greedily among image rows.
//
// Row r of plane `plane` is A_r[x] = cover[(r*W + x)*channels + plane].  With
// Q = floor(W/4) (Section VI step 5: 4*|B| <= |A|), rows take Q message bytes
// each until fewer than Q remain (Section VII step 4), so message byte o sits
// in row r = o / Q at column j = o % Q, and that row's length is
// L_r = min(Q, N - r*Q).  Block i of the paper's launch writes bit pair i of
// B[j] to A_r[L_r*i + j] (Section VI step 7); extraction ORs the pairs back
// (Section VII step 6).
//
// One thread per message byte computes (r, j, L_r) once and touches its four
// plane bytes; consecutive threads touch consecutive pixels, so each warp's
// accesses are contiguous to within the channel stride.  The out-of-place
// copy of the cover is done beforehand by the STREAM1 vector kernel with no
// carrying bytes (a 128-bit streaming copy).
#include "internal.cuh"

namespace stego {
namespace {

struct P2Args {
    const uint8_t *src; // cover (embed) or stego (extract)
    uint8_t *dst;       // stego (embed)
    const uint8_t *msg_in;
    uint8_t *msg_out;
    uint64_t N;
    uint64_t Q; // bytes per full row, floor(W/4)
    uint64_t W;
    uint32_t channels;
    uint32_t plane;
    stego_result *res;
};

// Position in the cover of bit pair i of message byte o.
struct RowPos {
    uint64_t row_base; // r*W
    uint64_t L;        // L_r
    uint64_t j;        // column of the byte within the row's quarter
};

__device__ __forceinline__ RowPos row_pos(const P2Args &a, uint64_t o)
{
    RowPos p;
    const uint64_t r = o / a.Q;
    p.j = o - r * a.Q;
    const uint64_t rem = a.N - r * a.Q;
    p.L = rem < a.Q ? rem : a.Q;
    p.row_base = r * a.W;
    return p;
}

__device__ __forceinline__ uint64_t byte_index(const P2Args &a, const RowPos &p, int i)
{
    return (p.row_base + p.L * (uint64_t)i + p.j) * a.channels + a.plane;
}

template <bool STATS>
__global__ void __launch_bounds__(512) p2_embed_kernel(P2Args a)
{
    unsigned long long changed = 0, sse = 0;
    if (a.res && blockIdx.x == 0 && threadIdx.x == 0) {
        a.res->msg_bytes = a.N;
        a.res->status = STEGO_OK;
        a.res->reserved = 0;
        if (!STATS) {
            a.res->changed = 0;
            a.res->sse = 0;
        }
    }
    for (uint64_t o = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; o < a.N;
         o += (uint64_t)gridDim.x * blockDim.x) {
        const RowPos p = row_pos(a, o);
        const uint32_t B = __ldg(a.msg_in + o);
        uint64_t x[4];
        uint32_t c[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            x[i] = byte_index(a, p, i);
            c[i] = a.src[x[i]]; // plain load: src may equal dst (in place)
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t v = (c[i] & 0xFCu) | ((B >> (2 * i)) & 3u);
            a.dst[x[i]] = (uint8_t)v;
            if (STATS) {
                const uint32_t d = v > c[i] ? v - c[i] : c[i] - v;
                changed += d != 0;
                sse += d * d;
            }
        }
    }
    if (STATS)
        block_add2(changed, sse, reinterpret_cast<unsigned long long *>(&a.res->changed));
}

__global__ void __launch_bounds__(512) p2_extract_kernel(P2Args a)
{
    if (a.res && blockIdx.x == 0 && threadIdx.x == 0) {
        a.res->changed = 0;
        a.res->sse = 0;
        a.res->msg_bytes = a.N;
        a.res->status = STEGO_OK;
        a.res->reserved = 0;
    }
    for (uint64_t o = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; o < a.N;
         o += (uint64_t)gridDim.x * blockDim.x) {
        const RowPos p = row_pos(a, o);
        uint32_t c[4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
            c[i] = __ldg(a.src + byte_index(a, p, i));
        uint32_t B = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i)
            B |= (c[i] & 3u) << (2 * i);
        a.msg_out[o] = (uint8_t)B;
    }
}

P2Args make_args(const uint8_t *src, uint8_t *dst, const stego_geom &g, const uint8_t *msg_in,
                 uint8_t *msg_out, uint64_t N, stego_result *res)
{
    P2Args a;
    a.src = src;
    a.dst = dst;
    a.msg_in = msg_in;
    a.msg_out = msg_out;
    a.N = N;
    a.Q = g.width / 4u;
    a.W = g.width;
    a.channels = g.channels;
    a.plane = g.plane;
    a.res = res;
    return a;
}

} // namespace

cudaError_t p2_embed(const uint8_t *cover, uint8_t *stego, const stego_geom &g,
                     const uint8_t *msg, uint64_t N, bool stats, stego_result *res,
                     const Shape &sh, cudaStream_t s)
{
    P2Args a = make_args(cover, stego, g, msg, nullptr, N, res);
    const void *k = stats ? (const void *)p2_embed_kernel<true> : (const void *)p2_embed_kernel<false>;
    const int grid = persistent_grid(k, sh.threads, 0, sh.ctas_per_sm, N, (uint64_t)sh.threads);
    void *args[] = {&a};
    return cudaLaunchKernel(k, dim3(grid), dim3(sh.threads), args, 0, s);
}

cudaError_t p2_extract(const uint8_t *st, const stego_geom &g, uint8_t *msg, uint64_t N,
                       stego_result *res, const Shape &sh, cudaStream_t s)
{
    P2Args a = make_args(st, nullptr, g, nullptr, msg, N, res);
    const void *k = (const void *)p2_extract_kernel;
    const int grid = persistent_grid(k, sh.threads, 0, sh.ctas_per_sm, N, (uint64_t)sh.threads);
    void *args[] = {&a};
    return cudaLaunchKernel(k, dim3(grid), dim3(sh.threads), args, 0, s);
}

} // namespace stego
