// streamk.cu -- the stream layout with k = 1..4 bits per carrying byte, over
// every cover byte or over one colour plane in pixel order (Section VI step
// 2's "separate any one plane").  The variant space between the one-bit
// stream and the paper's two bits per byte (Section VI step 7c-f):
//
//   stream bit b  ->  bit (k - 1 - b mod k) of carrying byte b / k,
//   carrying byte x = cover byte x (all bytes) or x*channels + plane,
//
// S = BE32(8m) || msg (header) or msg.  When 8|S| is not a multiple of k, the
// last carrying byte changes only its top (8|S| mod k) field bits.  k = 1 over
// all bytes is handled by stream1.cu.
//
// Kernels:
//   embedk_vec<K,STATS>  all bytes, 16-byte aligned cover and stego: a
//       16-byte vector carries 16K stream bits = stream bytes [2Kv, 2Kv+2K),
//       assembled big-endian into one 64-bit word and cut into 16 K-bit
//       fields; traffic 2C + 8|S|/8 out of place.
//   embedk_bytes<STATS>  any alignment, any k, either carrying order: one
//       thread per carrying byte (out of place with one plane, after a copy
//       of the cover).
//   extractk_vec<K>  all bytes, 16-byte aligned stego.
//   extractk_bytes  any alignment, any k, either carrying order.
// The header's 32 bits are read by warp 0 of each CTA: lane l loads stream
// bit l from its carrying byte and one ballot gathers them.
#include <cstring>

#include "internal.cuh"

namespace stego {
namespace {

struct KView {
    const uint8_t *cover; // embed: cover; extract: stego
    uint8_t *stego;       // embed output
    const uint8_t *msg;   // embed message
    uint8_t *out;         // extract output
    uint64_t C;           // cover bytes
    uint64_t n_carry;     // carrying bytes processed (embed) / available (extract)
    uint64_t t_bits;      // embed: stream bits 8|S|
    uint64_t slen;        // embed: stream bytes
    uint64_t cap, raw_len;
    uint32_t k, header, nbits, plane_only;
    uint32_t channels, plane;
    stego_result *res;
    uint64_t res_msg_bytes;
};

__device__ __forceinline__ uint64_t carry_pos(const KView &a, uint64_t x)
{
    return a.plane_only ? x * a.channels + a.plane : x;
}

__device__ __forceinline__ uint32_t sbyte(const KView &a, uint64_t q)
{
    if (q >= a.slen)
        return 0u;
    if (a.header) {
        if (q < 4)
            return (a.nbits >> (24u - 8u * (uint32_t)q)) & 0xFFu;
        return __ldg(a.msg + (q - 4));
    }
    return __ldg(a.msg + q);
}

// The k-bit field of carrying byte x and the mask of its bits that carry
// stream data (all k, the top few for the last byte, none past the stream).
__device__ __forceinline__ void field_of(const KView &a, uint64_t x, uint32_t &f, uint32_t &fm)
{
    const uint32_t k = a.k;
    const uint64_t b0 = x * k;
    if (b0 >= a.t_bits) {
        f = fm = 0u;
        return;
    }
    const uint64_t left = a.t_bits - b0;
    const uint32_t valid = left < k ? (uint32_t)left : k;
    const uint32_t w = (sbyte(a, b0 >> 3) << 8) | sbyte(a, (b0 >> 3) + 1);
    const uint32_t off = (uint32_t)(b0 & 7u);
    f = (w >> (16u - off - k)) & ((1u << k) - 1u);
    fm = ((1u << valid) - 1u) << (k - valid);
}

__device__ __forceinline__ void embed_res(const KView &a, bool stats)
{
    if (a.res && blockIdx.x == 0 && threadIdx.x == 0) {
        a.res->msg_bytes = a.res_msg_bytes;
        a.res->status = STEGO_OK;
        a.res->reserved = 0;
        if (!stats) {
            a.res->changed = 0;
            a.res->sse = 0;
        }
    }
}

// Changed bytes and squared error of a word pair that differs only in the
// low four bits of some bytes.
__device__ __forceinline__ void low_stats(uint32_t o, uint32_t c, unsigned long long &changed,
                                          unsigned long long &sse)
{
    const uint32_t x = o ^ c;
    changed += __popc((x | (x >> 1) | (x >> 2) | (x >> 3)) & 0x01010101u);
    const uint32_t d = __vabsdiffu4(o & 0x0F0F0F0Fu, c & 0x0F0F0F0Fu);
    sse += __dp4a(d, d, 0u);
}

// The one vector where the stream ends, field by field (a call of its own
// keeps the hot loop's registers low).
__device__ __noinline__ uint4 stream_end_vector(const KView &a, uint64_t v, uint4 c)
{
    uint32_t ow[4] = {c.x, c.y, c.z, c.w};
    for (int t = 0; t < 16; ++t) {
        uint32_t fv, fm;
        field_of(a, v * 16u + t, fv, fm);
        const uint32_t s = 8 * (t & 3);
        ow[t >> 2] = (ow[t >> 2] & ~(fm << s)) | ((fv & fm) << s);
    }
    return make_uint4(ow[0], ow[1], ow[2], ow[3]);
}

// Stream bytes [2Kv, 2Kv + 2K) as a big-endian 64-bit word (whole vector
// inside the stream): word loads when they are message bytes on a 4-byte
// boundary, byte loads otherwise.
template <int K>
__device__ __forceinline__ uint64_t stream_window(const KView &a, uint64_t v)
{
    uint64_t X = 0;
    const uint64_t q0 = 2u * K * v;
    const uint64_t hb = a.header ? 4u : 0u;
    const uint8_t *mp = a.msg + (q0 - hb);
    if ((K & 1) == 0 && q0 >= hb && (((uintptr_t)mp & 3u) == 0)) {
#pragma unroll
        for (int i = 0; i < K / 2; ++i) {
            const uint32_t w = __ldg(reinterpret_cast<const uint32_t *>(mp) + i);
            X |= (uint64_t)__byte_perm(w, 0u, 0x0123u) << (32 - 32 * i);
        }
    } else {
#pragma unroll
        for (int i = 0; i < 2 * K; ++i)
            X |= (uint64_t)sbyte(a, q0 + i) << (56 - 8 * i);
    }
    return X;
}

// Grid-stride over 16-byte vectors (V per thread per iteration, cover and
// stream loads issued before any arithmetic).
template <int K, bool STATS>
__global__ void __launch_bounds__(512) embedk_vec(KView a)
{
    constexpr int V = 1; // more in flight measured slower (registers)
    constexpr uint32_t MASK = (1u << K) - 1u;
    constexpr uint32_t BYTEMASK = MASK * 0x01010101u;
    unsigned long long changed = 0, sse = 0;
    embed_res(a, STATS);
    const uint64_t nvec = a.n_carry >> 4;
    const uint4 *__restrict__ src = reinterpret_cast<const uint4 *>(a.cover);
    uint4 *dst = reinterpret_cast<uint4 *>(a.stego);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x * V;
    for (uint64_t v0 = (uint64_t)blockIdx.x * blockDim.x * V + threadIdx.x; v0 < nvec;
         v0 += stride) {
        uint4 c[V];
        uint64_t X[V];
#pragma unroll
        for (int u = 0; u < V; ++u) {
            const uint64_t v = v0 + (uint64_t)u * blockDim.x;
            if (v < nvec)
                c[u] = __ldcs(src + v);
        }
#pragma unroll
        for (int u = 0; u < V; ++u) {
            const uint64_t v = v0 + (uint64_t)u * blockDim.x;
            X[u] = 0;
            if (v < nvec && (v + 1) * 16u * K <= a.t_bits)
                X[u] = stream_window<K>(a, v);
        }
#pragma unroll
        for (int u = 0; u < V; ++u) {
            const uint64_t v = v0 + (uint64_t)u * blockDim.x;
            if (v >= nvec)
                continue;
            uint4 o = c[u];
            const uint64_t b0 = v * 16u * K; // first stream bit of the vector
            if (b0 + 16u * K <= a.t_bits) {
                uint32_t f[4];
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    f[w] = 0;
#pragma unroll
                    for (int l = 0; l < 4; ++l) {
                        const int t = 4 * w + l;
                        f[w] |= (uint32_t)((X[u] >> (64 - K * (t + 1))) & MASK) << (8 * l);
                    }
                }
                o.x = (c[u].x & ~BYTEMASK) | f[0];
                o.y = (c[u].y & ~BYTEMASK) | f[1];
                o.z = (c[u].z & ~BYTEMASK) | f[2];
                o.w = (c[u].w & ~BYTEMASK) | f[3];
            } else if (b0 < a.t_bits) {
                o = stream_end_vector(a, v, c[u]);
            }
            __stcs(dst + v, o);
            if (STATS) {
                low_stats(o.x, c[u].x, changed, sse);
                low_stats(o.y, c[u].y, changed, sse);
                low_stats(o.z, c[u].z, changed, sse);
                low_stats(o.w, c[u].w, changed, sse);
            }
        }
    }
    // carrying bytes after the last whole vector
    if (blockIdx.x == 0 && threadIdx.x < (uint32_t)(a.n_carry & 15u)) {
        const uint64_t x = ((a.n_carry >> 4) << 4) + threadIdx.x;
        uint32_t fv, fm;
        field_of(a, x, fv, fm);
        const uint32_t cb = a.cover[x];
        const uint32_t ob = (cb & ~fm) | (fv & fm);
        a.stego[x] = (uint8_t)ob;
        if (STATS) {
            const uint32_t d = ob > cb ? ob - cb : cb - ob;
            changed += d != 0;
            sse += d * d;
        }
    }
    if (STATS)
        block_add2(changed, sse, reinterpret_cast<unsigned long long *>(&a.res->changed));
}

// One thread per carrying byte x < n_carry (all bytes: the bytes past the
// stream are copied; one plane: only plane bytes are written).
template <bool STATS>
__global__ void __launch_bounds__(512) embedk_bytes(KView a)
{
    unsigned long long changed = 0, sse = 0;
    embed_res(a, STATS);
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < a.n_carry;
         x += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t fv, fm;
        field_of(a, x, fv, fm);
        const uint64_t p = carry_pos(a, x);
        const uint32_t cb = a.cover[p]; // plain load: cover may equal stego
        const uint32_t ob = (cb & ~fm) | (fv & fm);
        a.stego[p] = (uint8_t)ob;
        if (STATS) {
            const uint32_t d = ob > cb ? ob - cb : cb - ob;
            changed += d != 0;
            sse += d * d;
        }
    }
    if (STATS)
        block_add2(changed, sse, reinterpret_cast<unsigned long long *>(&a.res->changed));
}

// Stream bit b read back from the stego.
__device__ __forceinline__ uint32_t stream_bit(const KView &a, uint64_t b)
{
    const uint64_t x = b / a.k;
    const uint32_t pos = a.k - 1u - (uint32_t)(b - x * a.k);
    return (a.cover[carry_pos(a, x)] >> pos) & 1u;
}

// Length, status and first message bit of an extraction; block 0 publishes
// the result.  With the header, warp 0 reads stream bits 0..31 (one per lane)
// and one ballot assembles the count.
__device__ __forceinline__ int extractk_prologue(const KView &a, uint64_t &len)
{
    __shared__ int s_status;
    __shared__ unsigned long long s_len;
    const uint64_t avail = a.n_carry * a.k; // stream bits the stego holds
    if (a.header) {
        if (threadIdx.x < 32) {
            const uint32_t l = threadIdx.x;
            const uint32_t bit = (l < avail) ? stream_bit(a, l) : 0u;
            const uint32_t nbits = __brev(__ballot_sync(0xFFFFFFFFu, bit));
            if (l == 0) {
                int st = STEGO_OK;
                if (avail < 32u || (nbits & 7u) || 32ull + nbits > avail)
                    st = STEGO_E_BAD_HEADER;
                else if ((uint64_t)(nbits >> 3) > a.cap)
                    st = STEGO_E_MSG_TOO_SMALL;
                s_status = st;
                s_len = st == STEGO_OK ? (nbits >> 3) : 0u;
            }
        }
    } else if (threadIdx.x == 0) {
        s_status = STEGO_OK;
        s_len = a.raw_len;
    }
    __syncthreads();
    len = s_len;
    const int status = s_status;
    if (a.res && blockIdx.x == 0 && threadIdx.x == 0) {
        a.res->changed = 0;
        a.res->sse = 0;
        a.res->msg_bytes = len;
        a.res->status = status;
        a.res->reserved = 0;
    }
    return status;
}

// All bytes, aligned stego: vector v yields stream bytes [2Kv, 2Kv + 2K).
template <int K>
__global__ void __launch_bounds__(512) extractk_vec(KView a)
{
    constexpr uint32_t MASK = (1u << K) - 1u;
    uint64_t len;
    if (extractk_prologue(a, len) != STEGO_OK)
        return;
    const uint64_t hb = a.header ? 4u : 0u;       // stream bytes before the message
    const uint64_t sbytes = len + hb;              // stream bytes to recover
    // whole 16-byte vectors of the stego only; the stream bytes after them
    // (when the stego's length is not a multiple of 16) go bit by bit
    const uint64_t want = (sbytes + 2 * K - 1) / (2 * K);
    const uint64_t nvec = want < (a.C >> 4) ? want : (a.C >> 4);
    const uint4 *__restrict__ src = reinterpret_cast<const uint4 *>(a.cover);
    for (uint64_t q = 2u * K * nvec + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
         q < sbytes; q += (uint64_t)gridDim.x * blockDim.x) {
        if (q < hb)
            continue;
        uint32_t v = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i)
            v |= stream_bit(a, 8u * q + i) << (7 - i);
        a.out[q - hb] = (uint8_t)v;
    }
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvec;
         v += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 c = __ldcs(src + v);
        const uint32_t w[4] = {c.x, c.y, c.z, c.w};
        uint64_t X = 0;
#pragma unroll
        for (int t = 0; t < 16; ++t)
            X |= (uint64_t)((w[t >> 2] >> (8 * (t & 3))) & MASK) << (64 - K * (t + 1));
        const uint64_t q0 = 2u * K * v; // first stream byte of the vector
        uint8_t *op = a.out + (q0 - hb);
        if ((K & 1) == 0 && q0 >= hb && q0 + 2 * K <= sbytes && (((uintptr_t)op & 3u) == 0)) {
            // message bytes only, 4-byte aligned: K/2 word stores
#pragma unroll
            for (int i = 0; i < K / 2; ++i)
                reinterpret_cast<uint32_t *>(op)[i] =
                    __byte_perm((uint32_t)(X >> (32 - 32 * i)), 0u, 0x0123u);
        } else {
#pragma unroll
            for (int i = 0; i < 2 * K; ++i) {
                const uint64_t q = q0 + i; // stream byte
                if (q >= hb && q < sbytes)
                    a.out[q - hb] = (uint8_t)(X >> (56 - 8 * i));
            }
        }
    }
}

// Any alignment, any k, either carrying order: one thread per message byte.
__global__ void __launch_bounds__(512) extractk_bytes(KView a)
{
    uint64_t len;
    if (extractk_prologue(a, len) != STEGO_OK)
        return;
    const uint64_t first = a.header ? 32u : 0u;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < len;
         s += (uint64_t)gridDim.x * blockDim.x) {
        // walk the message byte's eight stream bits field by field: one
        // division per byte, one load per carrying byte touched
        const uint64_t b0 = first + 8u * s;
        uint64_t x = b0 / a.k;
        uint32_t r = (uint32_t)(b0 - x * a.k);
        uint32_t cb = a.cover[carry_pos(a, x)];
        uint32_t v = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            v |= ((cb >> (a.k - 1u - r)) & 1u) << (7 - i);
            if (++r == a.k && i < 7) {
                r = 0;
                cb = a.cover[carry_pos(a, ++x)];
            }
        }
        a.out[s] = (uint8_t)v;
    }
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

} // namespace

cudaError_t sk_embed(const uint8_t *cover, uint8_t *stego, uint64_t C, uint32_t k, bool plane_only,
                     const stego_geom *g, const uint8_t *msg, uint64_t m, bool header,
                     bool stats, stego_result *res, const Shape &sh, cudaStream_t s)
{
    KView a;
    std::memset(&a, 0, sizeof(a));
    a.cover = cover;
    a.stego = stego;
    a.msg = msg;
    a.C = C;
    a.slen = m + (header ? 4u : 0u);
    a.t_bits = 8u * a.slen;
    a.k = k;
    a.header = header ? 1u : 0u;
    a.nbits = (uint32_t)(8u * m);
    a.plane_only = plane_only ? 1u : 0u;
    a.channels = plane_only ? g->channels : 1u;
    a.plane = plane_only ? g->plane : 0u;
    a.res = res;
    a.res_msg_bytes = m;
    const bool inplace = cover == stego;
    const uint64_t t_carry = (a.t_bits + k - 1) / k; // carrying bytes the stream uses
    const int T = sh.threads;
    void *args[] = {&a};
    if (!plane_only && aligned16(cover) && aligned16(stego)) {
        a.n_carry = inplace ? t_carry : C;
        const void *kern;
        switch (k) {
        case 2: kern = stats ? (const void *)embedk_vec<2, true> : (const void *)embedk_vec<2, false>; break;
        case 3: kern = stats ? (const void *)embedk_vec<3, true> : (const void *)embedk_vec<3, false>; break;
        default: kern = stats ? (const void *)embedk_vec<4, true> : (const void *)embedk_vec<4, false>; break;
        }
        const uint64_t nvec = a.n_carry >> 4;
        const int grid = persistent_grid(kern, T, 0, sh.ctas_per_sm, nvec ? nvec : 1,
                                         (uint64_t)T); // one vector per thread
        return cudaLaunchKernel(kern, dim3(grid), dim3(T), args, 0, s);
    }
    if (plane_only && !inplace) {
        // the non-carrying bytes come from a copy of the cover (a stream
        // embed with nothing to carry), then the plane bytes are rewritten
        cudaError_t e = s1_embed(cover, stego, C, 0, nullptr, 0, false, 0, false, nullptr, 0, sh, s);
        if (e != cudaSuccess)
            return e;
    }
    a.n_carry = plane_only ? t_carry : (inplace ? t_carry : C);
    const void *kern = stats ? (const void *)embedk_bytes<true> : (const void *)embedk_bytes<false>;
    const int grid = persistent_grid(kern, T, 0, sh.ctas_per_sm, a.n_carry ? a.n_carry : 1,
                                     (uint64_t)T * 16);
    return cudaLaunchKernel(kern, dim3(grid), dim3(T), args, 0, s);
}

cudaError_t sk_extract(const uint8_t *st, uint64_t C, uint32_t k, bool plane_only,
                       const stego_geom *g, uint8_t *msg, uint64_t cap, uint64_t raw_len,
                       bool header, stego_result *res, const Shape &sh, cudaStream_t s)
{
    KView a;
    std::memset(&a, 0, sizeof(a));
    a.cover = st;
    a.out = msg;
    a.C = C;
    a.cap = cap;
    a.raw_len = raw_len;
    a.k = k;
    a.header = header ? 1u : 0u;
    a.plane_only = plane_only ? 1u : 0u;
    a.channels = plane_only ? g->channels : 1u;
    a.plane = plane_only ? g->plane : 0u;
    a.n_carry = plane_only ? (uint64_t)g->width * g->height : C;
    a.res = res;
    const uint64_t avail_bits = a.n_carry * k;
    uint64_t max_len = raw_len;
    if (header) {
        const uint64_t fit = avail_bits >= 32 ? (avail_bits - 32) / 8 : 0;
        max_len = fit < cap ? fit : cap;
    }
    const int T = sh.threads;
    void *args[] = {&a};
    if (!plane_only && aligned16(st)) {
        const void *kern;
        switch (k) {
        case 2: kern = (const void *)extractk_vec<2>; break;
        case 3: kern = (const void *)extractk_vec<3>; break;
        default: kern = (const void *)extractk_vec<4>; break;
        }
        const uint64_t nvec = (max_len + 4 + 2 * k - 1) / (2 * k);
        const int grid = persistent_grid(kern, T, 0, sh.ctas_per_sm, nvec ? nvec : 1, (uint64_t)T);
        return cudaLaunchKernel(kern, dim3(grid), dim3(T), args, 0, s);
    }
    const void *kern = (const void *)extractk_bytes;
    const int grid = persistent_grid(kern, T, 0, sh.ctas_per_sm, max_len ? max_len : 1, (uint64_t)T);
    return cudaLaunchKernel(kern, dim3(grid), dim3(T), args, 0, s);
}

} // namespace stego
