// stream1.cu -- single-cover kernels of the one-bit stream layout: the
// Section VI substitution rule with one bit per cover byte over the cover in
// memory order, and the Section VII extraction of the same bits.
//
// Data layout and traffic: a 16-byte cover vector v carries stream bytes 2v
// and 2v+1, so one warp's 128-bit load instruction covers 512 contiguous
// cover bytes and its message reads cover 64 contiguous stream bytes.  Out of
// place an embed moves 2C + T/8 bytes, in place 2T + T/8, an extract T + T/8
// (T = carrying bytes).  Each byte is read once and written once, so nothing
// is staged through shared memory: 128-bit streaming loads/stores with V
// vectors in flight per thread over a persistent grid feed HBM directly.
// Misaligned buffers: cover and stego with the same address mod 16 run
// aligned vectors after a head of scalar bytes (the stream cut at the head's
// bit offset); cover and stego at different addresses mod 16 build each
// aligned stego vector from the two aligned cover vectors around its bytes;
// a misaligned stego is read as aligned vectors, each reduced to its 16
// LSBs, a pair's second part coming from the next lane.  Rounds wholly
// inside the buffers and the message run without per-vector checks.
#include "s1_device.cuh"

namespace stego {
namespace {

using s1::EmbedView;
using s1::ExtractView;

struct EmbedArgs {
    EmbedView a;
    stego_result *res;
    uint64_t res_msg_bytes;
    StatSlot *slot;
};

__device__ __forceinline__ void write_res(const EmbedArgs &e, bool stats)
{
    if (e.res && blockIdx.x == 0 && threadIdx.x == 0) {
        e.res->msg_bytes = e.res_msg_bytes;
        e.res->status = STEGO_OK;
        e.res->reserved = 0;
        if (!stats) {
            e.res->changed = 0;
            e.res->sse = 0;
        }
    }
}

// Vector path (cover and stego 16-byte aligned), persistent grid.  Whole
// rounds of V vectors per thread cover the vectors up to the last multiple
// of the grid's round; the remainder is spread one vector per thread over
// the whole grid, so every CTA ends within a fraction of a round of the
// others (with rounds dealt whole, a quarter of the CTAs would run one round
// longer on the 201 MB cover).
template <int V, bool STATS>
__global__ void __launch_bounds__(512) embed_vec(EmbedArgs e)
{
    grid_dependency_wait(); // launched dependent: nothing is touched before
    allow_dependents();
    unsigned long long changed = 0, sse = 0;
    write_res(e, STATS);
    const uint64_t nvec = e.a.n_bytes >> 4;
    const uint64_t round = (uint64_t)gridDim.x * blockDim.x * V;
    const uint64_t whole = nvec / round * round;
    s1::embed_vec_range<V, STATS>(e.a, (uint64_t)blockIdx.x * blockDim.x * V + threadIdx.x,
                                  whole, round, changed, sse);
    s1::embed_vec_range<1, STATS>(e.a, whole + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x,
                                  nvec, (uint64_t)gridDim.x * blockDim.x, changed, sse);
    if (blockIdx.x == 0)
        s1::embed_tail<STATS>(e.a, changed, sse);
    if (STATS)
        block_stats(changed, sse, e.res, e.slot);
}

// The h head bytes and the bytes after the nvb aligned vectors that follow
// them (fewer than 32 in all), one per thread of the calling CTA.
template <bool STATS>
__device__ __forceinline__ void head_tail(const s1::EmbedView &a, uint32_t h, uint64_t nvb,
                                          unsigned long long &changed, unsigned long long &sse)
{
    const uint32_t tail = (uint32_t)(a.n_bytes - h - (nvb << 4));
    if (threadIdx.x < h + tail) {
        const uint64_t k = threadIdx.x < h ? (uint64_t)threadIdx.x
                                           : h + (nvb << 4) + (threadIdx.x - h);
        const uint32_t sb = k < a.t_bytes ? s1::stream_byte(a, k >> 3) : 0u;
        s1::embed_one<STATS>(a, k, sb, changed, sse);
    }
}

// Cover and stego with the same misalignment: aligned vectors after h head
// bytes, the stream cut at bit h % 8; block 0 does the head and the tail
// (fewer than 32 bytes).  Requires n_bytes >= h.
template <int V, bool STATS>
__global__ void __launch_bounds__(512) embed_shift(EmbedArgs e, uint32_t h)
{
    grid_dependency_wait(); // launched dependent: nothing is touched before
    allow_dependents();
    unsigned long long changed = 0, sse = 0;
    write_res(e, STATS);
    const uint64_t nvb = (e.a.n_bytes - h) >> 4;
    s1::embed_shift_range<V, STATS>(e.a, h, (uint64_t)blockIdx.x * blockDim.x * V + threadIdx.x,
                                    nvb, (uint64_t)gridDim.x * blockDim.x * V, changed, sse);
    if (blockIdx.x == 0)
        head_tail<STATS>(e.a, h, nvb, changed, sse);
    if (STATS)
        block_stats(changed, sse, e.res, e.slot);
}

// Cover and stego at different addresses mod 16, out of place: aligned
// stego vectors after h head bytes, each from two aligned cover vectors
// (cover + h is 4Q + b bytes past a 16-byte boundary), the grid's warps
// taking blocks of 32*V consecutive stego vectors; block 0 does the head and
// the tail (fewer than 32 bytes).
// Requires n_bytes >= h.
template <int Q, int V, bool STATS>
__global__ void __launch_bounds__(512) embed_funnel(EmbedArgs e, uint32_t h, uint32_t sel)
{
    grid_dependency_wait(); // launched dependent: nothing is touched before
    allow_dependents();
    unsigned long long changed = 0, sse = 0;
    write_res(e, STATS);
    const uint64_t nvb = (e.a.n_bytes - h) >> 4;
    s1::embed_funnel_warp<Q, STATS, V>(e.a, h, sel, 0, nvb,
                                       ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5,
                                       ((uint64_t)gridDim.x * blockDim.x) >> 5, changed, sse);
    if (blockIdx.x == 0)
        head_tail<STATS>(e.a, h, nvb, changed, sse);
    if (STATS)
        block_stats(changed, sse, e.res, e.slot);
}

// Byte path for cover and stego with different misalignments: one thread
// per stream byte (eight cover bytes).
template <bool STATS>
__global__ void __launch_bounds__(512) embed_bytes(EmbedArgs e)
{
    grid_dependency_wait(); // launched dependent: nothing is touched before
    allow_dependents();
    unsigned long long changed = 0, sse = 0;
    write_res(e, STATS);
    s1::embed_bytes_range<STATS>(e.a, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x,
                                 (e.a.n_bytes + 7) >> 3, (uint64_t)gridDim.x * blockDim.x,
                                 changed, sse);
    if (STATS)
        block_stats(changed, sse, e.res, e.slot);
}

using s1::ExtractArgs;
using s1::extract_prologue;

// Vector path: stego 16-byte aligned.  The first round's loads are issued
// before the header is read (bounded by the longest message the call can
// produce, so they stay inside the stego); the round is then written for the
// header's length.  Later rounds: whole rounds, then the remainder spread
// one vector per thread as in embed_vec.
template <int V>
__global__ void __launch_bounds__(512) extract_vec(ExtractArgs a)
{
    grid_dependency_wait(); // launched dependent: nothing is touched before
    allow_dependents();
    const uint64_t first = (uint64_t)blockIdx.x * blockDim.x * V + threadIdx.x;
    const uint64_t round = (uint64_t)gridDim.x * blockDim.x * V;
    const uint4 *__restrict__ src =
        reinterpret_cast<const uint4 *>(a.st + (a.header ? 32u : 0u));
    uint4 c[V];
#pragma unroll
    for (int u = 0; u < V; ++u) {
        const uint64_t v = first + (uint64_t)u * blockDim.x;
        if (v < a.max_vec)
            c[u] = __ldcs(src + v);
    }
    ExtractView x;
    if (extract_prologue(a, x) != STEGO_OK)
        return;
    const uint64_t nvec = x.len >> 1;
#pragma unroll
    for (int u = 0; u < V; ++u) {
        const uint64_t v = first + (uint64_t)u * blockDim.x;
        if (v >= nvec)
            continue;
        const uint32_t pair = s1::gather16(c[u]);
        if (x.msg_even) {
            *reinterpret_cast<unsigned short *>(x.msg + 2 * v) = (unsigned short)pair;
        } else {
            x.msg[2 * v] = (uint8_t)pair;
            x.msg[2 * v + 1] = (uint8_t)(pair >> 8);
        }
    }
    const uint64_t whole = nvec / round * round;
    s1::extract_vec_range<V>(x, first + round, whole, round);
    const uint64_t rest = whole > round ? whole : round; // vectors below: done above
    s1::extract_vec_range<1>(x, rest + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nvec,
                             (uint64_t)gridDim.x * blockDim.x);
    if ((x.len & 1u) && blockIdx.x == 0 && threadIdx.x == 0)
        s1::extract_one(x, x.len - 1);
}

// A stego that is not 16-byte aligned: the warps of the grid take rounds
// of 32*V message byte pairs; each aligned stego vector is loaded once and
// reduced to its 16 LSBs, a pair's bits cut from its own and the next
// lane's.
template <int V>
__global__ void __launch_bounds__(512) extract_shift(ExtractArgs a)
{
    grid_dependency_wait(); // launched dependent: nothing is touched before
    allow_dependents();
    ExtractView x;
    if (extract_prologue(a, x) != STEGO_OK)
        return;
    const uint64_t wpb = blockDim.x >> 5;
    s1::extract_shift_lsb<V>(x, a.C, 0, x.len >> 1,
                             (uint64_t)blockIdx.x * wpb + (threadIdx.x >> 5),
                             (uint64_t)gridDim.x * wpb);
    if ((x.len & 1u) && blockIdx.x == 0 && threadIdx.x == 0)
        s1::extract_one(x, x.len - 1);
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// Vectors in flight per thread in the misaligned kernels, measured on the
// 201 MB cover at full capacity (with the check-free interior rounds):
// same misalignment embed 69.6 / 69.7 / 69.2 us for 1 / 2 / 4 (83-88 us
// before those rounds), and with the message words' address computed once
// per round 70.0-71.7 / 67.6-68.9 us for 2 / 4; different misalignments, both cover vectors loaded
// per stego vector, 82.7 / 72.4-73.7 / 71.7-84.7 us, and with the second
// vector shuffled from the next lane 71.7-74.5 us at 2 and 4 alike (4 kept:
// the batched kernel shares the routine and gains there); extraction 48.7
// (vector pairs, one per thread) / 43-44 / 36.1-36.9 us (LSB words shuffled
// between lanes).
constexpr int kShiftV = 4;
constexpr int kFunnelV = 4;
constexpr int kExtractShiftV = 4;

int clamp_vec(int v) { return (v == 1 || v == 2 || v == 8) ? v : 4; }

} // namespace

cudaError_t s1_embed(const uint8_t *cover, uint8_t *stego, uint64_t n_bytes, uint64_t t_bytes,
                     const uint8_t *msg, uint64_t slen, bool header, uint32_t nbits, bool stats,
                     stego_result *res, uint64_t res_msg_bytes, const Shape &sh, cudaStream_t s,
                     StatSlot *slot)
{
    EmbedArgs e;
    e.a.cover = cover;
    e.a.stego = stego;
    e.a.msg = msg;
    e.a.n_bytes = n_bytes;
    e.a.t_bytes = t_bytes;
    e.a.slen = slen;
    e.a.header = header ? 1u : 0u;
    e.a.nbits = nbits;
    e.a.msg_even = ((uintptr_t)msg & 1u) == 0;
    e.a.pad = 0;
    e.res = res;
    e.res_msg_bytes = res_msg_bytes;
    e.slot = stats ? slot : nullptr;
    const int T = sh.threads;
    void *args[] = {&e};
    if (aligned16(cover) && aligned16(stego) && bulk_stages(sh))
        return s1_embed_bulk(cover, stego, n_bytes, t_bytes, msg, slen, header, nbits, stats,
                             res, res_msg_bytes, sh, s, slot);
    if (aligned16(cover) && aligned16(stego)) {
        const int vec = clamp_vec(sh.vec);
        const void *k = nullptr;
        switch (vec) {
        case 1: k = stats ? (const void *)embed_vec<1, true> : (const void *)embed_vec<1, false>; break;
        case 2: k = stats ? (const void *)embed_vec<2, true> : (const void *)embed_vec<2, false>; break;
        case 8: k = stats ? (const void *)embed_vec<8, true> : (const void *)embed_vec<8, false>; break;
        default: k = stats ? (const void *)embed_vec<4, true> : (const void *)embed_vec<4, false>; break;
        }
        const uint64_t nvec = n_bytes >> 4;
        const int grid = persistent_grid(k, T, 0, sh.ctas_per_sm, nvec > 0 ? nvec : 1,
                                         (uint64_t)T * vec);
        return launch_dependent(k, dim3(grid), dim3(T), args, 0, s);
    }
    const uint32_t h = (uint32_t)((16u - ((uintptr_t)cover & 15u)) & 15u);
    if ((((uintptr_t)cover ^ (uintptr_t)stego) & 15u) == 0 && n_bytes >= (uint64_t)h + 16u) {
        const void *k = stats ? (const void *)embed_shift<kShiftV, true>
                              : (const void *)embed_shift<kShiftV, false>;
        const uint64_t nvb = (n_bytes - h) >> 4;
        const int grid = persistent_grid(k, T, 0, sh.ctas_per_sm, nvb, (uint64_t)T * kShiftV);
        void *sargs[] = {&e, (void *)&h};
        return launch_dependent(k, dim3(grid), dim3(T), sargs, 0, s);
    }
    const uint32_t hs = (uint32_t)((16u - ((uintptr_t)stego & 15u)) & 15u);
    if (cover != stego && n_bytes >= (uint64_t)hs + 16u) {
        const uint32_t d = (uint32_t)(((uintptr_t)cover + hs) & 15u), b = d & 3u;
        const uint32_t sel = b | ((b + 1) << 4) | ((b + 2) << 8) | ((b + 3) << 12);
        const void *k;
        constexpr int F = kFunnelV;
        switch (d >> 2) {
        case 0: k = stats ? (const void *)embed_funnel<0, F, true> : (const void *)embed_funnel<0, F, false>; break;
        case 1: k = stats ? (const void *)embed_funnel<1, F, true> : (const void *)embed_funnel<1, F, false>; break;
        case 2: k = stats ? (const void *)embed_funnel<2, F, true> : (const void *)embed_funnel<2, F, false>; break;
        default: k = stats ? (const void *)embed_funnel<3, F, true> : (const void *)embed_funnel<3, F, false>; break;
        }
        const uint64_t nvb = (n_bytes - hs) >> 4;
        const int grid = persistent_grid(k, T, 0, sh.ctas_per_sm, nvb, (uint64_t)T * F);
        void *fargs[] = {&e, (void *)&hs, (void *)&sel};
        return launch_dependent(k, dim3(grid), dim3(T), fargs, 0, s);
    }
    const void *k = stats ? (const void *)embed_bytes<true> : (const void *)embed_bytes<false>;
    const uint64_t units = (n_bytes + 7) >> 3;
    const int grid = persistent_grid(k, T, 0, sh.ctas_per_sm, units > 0 ? units : 1, (uint64_t)T);
    return launch_dependent(k, dim3(grid), dim3(T), args, 0, s);
}

cudaError_t s1_extract(const uint8_t *st, uint64_t C, uint8_t *msg, uint64_t cap,
                       uint64_t raw_len, bool header, stego_result *res, const Shape &sh,
                       cudaStream_t s)
{
    ExtractArgs a;
    a.st = st;
    a.C = C;
    a.msg = msg;
    a.cap = cap;
    a.raw_len = raw_len;
    a.header = header ? 1u : 0u;
    a.msg_even = ((uintptr_t)msg & 1u) == 0;
    a.res = res;
    // the longest message the launch may have to produce
    uint64_t max_len = raw_len;
    if (header) {
        const uint64_t fit = C >= 32 ? (C - 32) / 8 : 0;
        max_len = fit < cap ? fit : cap;
    }
    a.max_vec = max_len >> 1;
    const int T = sh.threads;
    void *args[] = {&a};
    if (aligned16(st) && bulk_stages(sh))
        return s1_extract_bulk(st, C, msg, cap, raw_len, header, res, sh, s);
    if (aligned16(st)) {
        const int vec = clamp_vec(sh.vec);
        const void *k;
        switch (vec) {
        case 1: k = (const void *)extract_vec<1>; break;
        case 2: k = (const void *)extract_vec<2>; break;
        case 8: k = (const void *)extract_vec<8>; break;
        default: k = (const void *)extract_vec<4>; break;
        }
        const uint64_t nvec = max_len >> 1;
        const int grid = persistent_grid(k, T, 0, sh.ctas_per_sm, nvec > 0 ? nvec : 1,
                                         (uint64_t)T * vec);
        return launch_dependent(k, dim3(grid), dim3(T), args, 0, s);
    }
    const void *k = (const void *)extract_shift<kExtractShiftV>;
    const uint64_t npairs = max_len >> 1;
    const int grid = persistent_grid(k, T, 0, sh.ctas_per_sm, npairs > 0 ? npairs : 1,
                                     (uint64_t)T * kExtractShiftV);
    return launch_dependent(k, dim3(grid), dim3(T), args, 0, s);
}

} // namespace stego
