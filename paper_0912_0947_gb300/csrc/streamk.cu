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
//   embedk_units<K,CH,PLANE,STATS>  16-byte aligned cover and stego, all
//       bytes (CH = 1) or one plane of 3 or 4 channels: a unit of 16
//       carrying bytes (CH vectors of the cover) carries 16K stream bits =
//       stream bytes [2Ku, 2Ku+2K), assembled big-endian into one 64-bit
//       word and cut into 16 K-bit fields; out of place the whole cover
//       moves once, 2C + |S| bytes.
//   embedk_bytes<STATS>  any alignment, any k, either carrying order: one
//       thread per carrying byte (out of place with one plane, after a copy
//       of the cover).
//   extractk_units<K,CH,PLANE>  16-byte aligned stego, same layouts.
//   extractk_bytes  any alignment, any k, either carrying order.
// The header's 32 bits are read by warp 0 of each CTA: lane l loads stream
// bit l from its carrying byte and one ballot gathers them.
#include <cstring>

#include "async_copy.cuh"
#include "s1_device.cuh"

namespace stego {
namespace {

// The installed launch shapes are tuned for the one-bit kernels; these
// kernels (other register counts) take as many resident CTAs as occupancy
// allows instead of a tuned CTA count.
constexpr int kAnyCtas = 0;

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
    uint64_t full_units;  // embed: units wholly inside the stream, t_bits / 16k
    uint64_t part_units;  // embed: units touching the stream, ceil(t_bits / 16k)
    uint32_t msg_w4;      // embed: msg - (header bytes) is 4-byte aligned
    uint32_t msg_w2;      // embed: msg - (header bytes) is 2-byte aligned
    StatSlot *slot;       // embed: per-stream statistics slot or nullptr
    uint32_t kmul;        // embed: 1 << k (a multiplier the compiler cannot see)
    uint32_t pad;
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

// Changed bytes and squared error of a unit's 16 carrying bytes (c before,
// o after, d = o ^ c, differences in the low K bits only), summed in 32 bits
// per unit.  A byte changed when any of its low K bits did (the packing and
// the per-field test are below).  With K = 1 every change is +-1, so the
// squared error equals the count.
template <int K>
__device__ __forceinline__ void unit_stats(const uint32_t (&o)[4], const uint32_t (&c)[4],
                                           const uint32_t (&d)[4], uint32_t kmul,
                                           unsigned long long &changed,
                                           unsigned long long &sse)
{
    constexpr uint32_t BM = ((1u << K) - 1u) * 0x01010101u;
    uint32_t n, s = 0;
    static_assert(K >= 1 && K <= 4, "one to four bits per byte");
    if constexpr (K <= 2) {
        // the four words' K-bit changes in disjoint bit ranges of each byte
        // (word i at bits K*i), joined by multiply-adds, then one fold
        // Horner in kmul = 1 << K: multiply-adds (FMA pipe), not shifts on
        // the busy ALU pipe; kmul comes from the launch arguments so the
        // compiler keeps the multiplies
        const uint32_t acc0 = ((d[3] * kmul + d[2]) * kmul + d[1]) * kmul + d[0];
        uint32_t acc = acc0;
        if (K == 2)
            acc = (acc | (acc >> 1)) & 0x55555555u;
        n = __popc(acc);
    } else {
        // k = 3, 4: two words per byte (word 2j+1 at bit K), then a field is
        // nonzero when its top bit is set or its low K-1 bits plus all ones
        // carry into the top bit (no carry leaves a field)
        constexpr uint32_t LOW = K == 4 ? 0x77777777u : 0x1B1B1B1Bu;
        constexpr uint32_t TOP = K == 4 ? 0x88888888u : 0x24242424u;
        const uint32_t a01 = d[1] * kmul + d[0], a23 = d[3] * kmul + d[2];
        n = __popc((a01 | ((a01 & LOW) + LOW)) & TOP) + __popc((a23 | ((a23 & LOW) + LOW)) & TOP);
    }
    if (K > 1) {
        uint32_t ab = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) { // sum of (a - b)^2 = a.a + b.b - 2 a.b over the fields
            const uint32_t fa = o[i] & BM, fb = c[i] & BM;
            s = __dp4a(fa, fa, s);
            s = __dp4a(fb, fb, s);
            ab = __dp4a(fa, fb, ab);
        }
        s -= 2u * ab;
    }
    changed += n;
    sse += K > 1 ? s : n;
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
// boundary, byte loads otherwise.  K = 3 packs its 6 bytes as two 24-bit
// halves instead, bytes 0-2 in the high word and 3-5 in the low one, each
// first byte on top (the form unit_fields<3> spreads).
template <int K>
__device__ __forceinline__ uint64_t stream_window(const KView &a, uint64_t v)
{
    uint64_t X = 0;
    const uint64_t q0 = 2u * K * v;
    const uint64_t hb = a.header ? 4u : 0u;
    const uint8_t *mp = a.msg + (q0 - hb);
    // q0 is a multiple of 4 for even K (of 2 for K = 3), so mp's alignment
    // is the launch's
    if constexpr (K == 3) {
        uint32_t v01, v23;
        if (q0 >= hb && a.msg_w2) {
            const unsigned short *hp = reinterpret_cast<const unsigned short *>(mp);
            const uint32_t h0 = __ldg(hp), h1 = __ldg(hp + 1), h2 = __ldg(hp + 2);
            v01 = __byte_perm(h0, h1, 0x2014u); // bytes 0, 1, 2 from the top; byte 3 zero
            v23 = __byte_perm(h1, h2, 0x2145u); // bytes 3, 4, 5
        } else {
            v01 = (sbyte(a, q0) << 16) | (sbyte(a, q0 + 1) << 8) | sbyte(a, q0 + 2);
            v23 = (sbyte(a, q0 + 3) << 16) | (sbyte(a, q0 + 4) << 8) | sbyte(a, q0 + 5);
        }
        return ((uint64_t)v01 << 32) | v23;
    } else if ((K & 1) == 0 && q0 >= hb && a.msg_w4) {
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

// A unit is 16 consecutive carrying bytes: 16 consecutive cover bytes (all
// bytes, CH = 1) or the plane bytes of 16 consecutive pixels (CH = 3 or 4
// channels, plane PLANE), i.e. CH 16-byte vectors of the cover.  Pixel t's
// plane byte is unit byte t*CH + PLANE, a compile-time position, so the 16
// carrying bytes are gathered into one 16-byte value, transformed as one
// vector of the all-bytes layout, and the change is XORed back.
template <int CH>
__device__ __forceinline__ void load_unit(const uint8_t *base, uint64_t u, uint32_t (&w)[4 * CH])
{
    const uint4 *p = reinterpret_cast<const uint4 *>(base) + u * CH;
#pragma unroll
    for (int j = 0; j < CH; ++j) {
        const uint4 c = __ldcs(p + j);
        w[4 * j] = c.x;
        w[4 * j + 1] = c.y;
        w[4 * j + 2] = c.z;
        w[4 * j + 3] = c.w;
    }
}

template <int CH>
__device__ __forceinline__ void store_unit(uint8_t *base, uint64_t u, const uint32_t (&w)[4 * CH])
{
    uint4 *p = reinterpret_cast<uint4 *>(base) + u * CH;
#pragma unroll
    for (int j = 0; j < CH; ++j)
        __stcs(p + j, make_uint4(w[4 * j], w[4 * j + 1], w[4 * j + 2], w[4 * j + 3]));
}

// The unit's 16 carrying bytes, byte t of word t/4 = carrying byte t.
template <int CH, int PLANE>
__device__ __forceinline__ void gather_unit(const uint32_t (&w)[4 * CH], uint32_t (&g)[4])
{
    if constexpr (CH == 1) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
            g[i] = w[i];
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            g[i] = 0;
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const int pos = (4 * i + l) * CH + PLANE; // unit byte of carrying byte 4i+l
                g[i] |= ((w[pos >> 2] >> (8 * (pos & 3))) & 0xFFu) << (8 * l);
            }
        }
    }
}

// XOR of carrying-byte differences d (gathered order) into the unit's words.
template <int CH, int PLANE>
__device__ __forceinline__ void scatter_xor(uint32_t (&w)[4 * CH], const uint32_t (&d)[4])
{
    if constexpr (CH == 1) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
            w[i] ^= d[i];
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const int pos = (4 * i + l) * CH + PLANE;
                w[pos >> 2] ^= ((d[i] >> (8 * l)) & 0xFFu) << (8 * (pos & 3));
            }
        }
    }
}

// Word i (carrying bytes 4i..4i+3, field in each byte's low K bits) of a
// unit whose stream window is X (stream bytes big-endian, the first in bits
// 56..63; for K = 3 two 24-bit halves).  K = 1, 4 fill the four byte lanes
// from replicated stream bytes with fixed per-lane shifts, K = 2 with one
// multiply; K = 3 (fields across byte boundaries) takes the word's 12 bits
// t and multiplies by 2^24 + 4: the two copies of t do not overlap, and
// leave fields 1, 3 at bits 8, 24 and fields 0, 2 at bits 11, 27, which one
// shift by 11 brings to bits 0, 16.
template <int K>
__device__ __forceinline__ uint32_t unit_fields(uint64_t X, int i)
{
    const uint32_t hi = (uint32_t)(X >> 32), lo = (uint32_t)X;
    if constexpr (K == 1) {
        // stream byte i/2; even words take its bits 7..4, odd words 3..0
        const uint32_t r = __byte_perm(hi, 0u, i < 2 ? 0x3333u : 0x2222u);
        return (i & 1) ? s1::spread_lo(r) : s1::spread_hi(r);
    } else if constexpr (K == 2) {
        // stream byte i; lane l takes its bits 7-2l and 6-2l: the products
        // b << 10l occupy disjoint bit ranges, and bits 8l+6, 8l+7 of their
        // sum hold pair l (b's bits 7-2l, 6-2l)
        const uint32_t b = __byte_perm(hi, 0u, 0x4440u | (3 - i)); // (hi >> (24 - 8i)) & 0xFF
        return ((b * 0x40100401u) >> 6) & 0x03030303u;
    } else if constexpr (K == 4) {
        // stream bytes 2i, 2i+1; lanes take high nibble, low nibble, high, low
        const uint32_t r = __byte_perm(i < 2 ? hi : lo, 0u, (i & 1) ? 0x0011u : 0x2233u);
        return ((r >> 4) & 0x000F000Fu) | (r & 0x0F000F00u);
    } else if constexpr (K == 3) {
        const uint32_t h = i < 2 ? hi : lo;
        const uint32_t t = (i & 1) ? (h & 0xFFFu) : (h >> 12);
        const uint32_t p = t * 0x01000004u;
        return (p & 0x07000700u) | ((p & 0x38003800u) >> 11);
    } else {
        constexpr uint32_t MASK = (1u << K) - 1u;
        uint32_t f = 0;
#pragma unroll
        for (int l = 0; l < 4; ++l)
            f |= (uint32_t)((X >> (64 - K * (4 * i + l + 1))) & MASK) << (8 * l);
        return f;
    }
}

// The inverse: a unit's stream window from its 16 carrying bytes g (words
// of four), fields in the low K bits.  K = 1 and 2 gather the four lanes of
// a word with one multiply (the partial products of the wanted bits land in
// disjoint bit ranges of the top byte, all others below it or past bit 31);
// K = 4 joins nibble pairs.
template <int K>
__device__ __forceinline__ uint64_t unit_window(const uint32_t (&g)[4])
{
    if constexpr (K == 1) {
        const uint32_t b0 = (s1::gather4(g[0]) << 4) | s1::gather4(g[1]);
        const uint32_t b1 = (s1::gather4(g[2]) << 4) | s1::gather4(g[3]);
        return (uint64_t)((b0 << 24) | (b1 << 16)) << 32;
    } else if constexpr (K == 2) {
        uint32_t hi = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) // lane l -> bits 30-2l, 31-2l of the product
            hi |= (((g[i] & 0x03030303u) * 0x40100401u) >> 24) << (24 - 8 * i);
        return (uint64_t)hi << 32;
    } else if constexpr (K == 4) {
        uint32_t b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t m = g[i] & 0x0F0F0F0Fu;
            b[i] = ((m << 4) | (m >> 8)) & 0x00FF00FFu; // bytes 2i (lane 0), 2i+1 (lane 2)
        }
        const uint32_t hi = __byte_perm(b[0], b[1], 0x0246u); // b0.l0 b0.l2 b1.l0 b1.l2, first on top
        const uint32_t lo = __byte_perm(b[2], b[3], 0x0246u);
        return ((uint64_t)hi << 32) | lo;
    } else {
        constexpr uint32_t MASK = (1u << K) - 1u;
        uint64_t X = 0;
#pragma unroll
        for (int t = 0; t < 16; ++t)
            X |= (uint64_t)((g[t >> 2] >> (8 * (t & 3))) & MASK) << (64 - K * (t + 1));
        return X;
    }
}

// k = 3: the unit's 48 stream bits as two 24-bit halves (words 0-1, 2-3),
// first bit on top.  Per word, one multiply by 2^11 + 1 joins the fields of
// bytes 0, 1 into bits 8-13 and those of bytes 2, 3 into bits 24-29 (the
// shifted copies do not overlap, so nothing carries); the high half of a
// second product, by 2^30 + 2^8, puts the first pair above the second at
// bits 0-11, with a copy of the second pair at bits 22-27 that the 12-bit
// shift of the first word pushes out and a mask of the second word drops.
// The multiplies run on the FMA pipe, which the k = 3 gather left idle.
__device__ __forceinline__ void unit_window3(const uint32_t (&g)[4], uint32_t &v01, uint32_t &v23)
{
    uint32_t t[4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
        t[i] = __umulhi(((g[i] & 0x07070707u) * 0x801u) & 0x3F003F00u, 0x40000100u);
    v01 = (t[0] << 12) | (t[1] & 0xFFFu);
    v23 = (t[2] << 12) | (t[3] & 0xFFFu);
}

// Units each thread keeps in flight per loop iteration.  A plane unit is
// already CH vectors; all-bytes units are single vectors, of which the
// extract batches four (measured on the 201 MB cover, k = 2: 43.0 us
// against 45.1 us with one, while one is fastest for the embed: 101.4 us
// against 114.7 us with two and 148.5 us with four).
constexpr int kEmbedAllBytesUnits = 1;
constexpr int kExtractAllBytesUnits = 4;
template <int CH, bool EMBED>
__host__ __device__ constexpr int units_per_iter()
{
    return CH == 1 ? (EMBED ? kEmbedAllBytesUnits : kExtractAllBytesUnits) : 1;
}

// Embed over units (cover and stego 16-byte aligned): U units per thread
// per iteration (lane-interleaved), each unit's 16K stream bits = stream
// bytes [2Ku, 2Ku + 2K) loaded as one big-endian word, all loads issued
// before any arithmetic.  Units wholly past the stream are copied.
// Carrying bytes after the last whole unit (fewer than 16) are done by
// block 0 byte by byte.
template <int K, int CH, int PLANE, bool STATS>
__global__ void __launch_bounds__(512, K >= 3 ? 3 : 0) embedk_units(KView a)
{
    grid_dependency_wait(); // launched dependent: nothing is touched before
    allow_dependents();
    constexpr int U = units_per_iter<CH, true>();
    constexpr uint32_t MASK = (1u << K) - 1u;
    constexpr uint32_t BYTEMASK = MASK * 0x01010101u;
    unsigned long long changed = 0, sse = 0;
    embed_res(a, STATS);
    const uint64_t nunits = a.n_carry >> 4;
    for (uint64_t u0 = (uint64_t)blockIdx.x * blockDim.x * U + threadIdx.x; u0 < nunits;
         u0 += (uint64_t)gridDim.x * blockDim.x * U) {
        uint32_t w[U][4 * CH];
        uint64_t X[U];
#pragma unroll
        for (int r = 0; r < U; ++r) {
            const uint64_t u = u0 + (uint64_t)r * blockDim.x;
            if (u < nunits)
                load_unit<CH>(a.cover, u, w[r]);
        }
#pragma unroll
        for (int r = 0; r < U; ++r) {
            const uint64_t u = u0 + (uint64_t)r * blockDim.x;
            X[r] = (u < nunits && u < a.full_units) ? stream_window<K>(a, u) : 0ull;
        }
#pragma unroll
        for (int r = 0; r < U; ++r) {
            const uint64_t u = u0 + (uint64_t)r * blockDim.x;
            if (u >= nunits)
                continue;
            if (u < a.part_units) {
                uint32_t c[4], o[4];
                gather_unit<CH, PLANE>(w[r], c);
                if (u < a.full_units) {
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        o[i] = (c[i] & ~BYTEMASK) | unit_fields<K>(X[r], i);
                } else {
                    const uint4 e = stream_end_vector(a, u, make_uint4(c[0], c[1], c[2], c[3]));
                    o[0] = e.x;
                    o[1] = e.y;
                    o[2] = e.z;
                    o[3] = e.w;
                }
                uint32_t d[4];
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    d[i] = o[i] ^ c[i];
                if (STATS)
                    unit_stats<K>(o, c, d, a.kmul, changed, sse);
                scatter_xor<CH, PLANE>(w[r], d);
            }
            store_unit<CH>(a.stego, u, w[r]);
        }
    }
    // cover bytes of the carrying bytes after the last whole unit: plane
    // bytes take their field, the other bytes of those pixels are copied
    if (blockIdx.x == 0 && threadIdx.x < (uint32_t)(a.n_carry & 15u) * CH) {
        const uint64_t pbyte = ((a.n_carry >> 4) << 4) * CH + threadIdx.x;
        const uint32_t cb = a.cover[pbyte];
        uint32_t ob = cb;
        if (threadIdx.x % CH == PLANE) {
            uint32_t fv, fm;
            field_of(a, pbyte / CH, fv, fm);
            ob = (cb & ~fm) | (fv & fm);
        }
        a.stego[pbyte] = (uint8_t)ob;
        if (STATS) {
            const uint32_t dd = ob > cb ? ob - cb : cb - ob;
            changed += dd != 0;
            sse += dd * dd;
        }
    }
    if (STATS)
        block_stats(changed, sse, a.res, a.slot);
}

// Plane units (CH = 3 or 4) with a two-stage copy pipeline per warp: while
// the warp embeds the units of one iteration from shared memory, the cover
// vectors of its next iteration are on their way there (cp.async, memory
// order, coalesced: a lane's own unit is 16*CH bytes from its neighbour's)
// and the next units' stream windows on their way to registers.  Each lane
// then takes its unit from shared memory, embeds it as embedk_units does and
// writes it back; the warp stores its vectors in memory order.  CTAs of at
// most kAsyncThreads threads (the staging area holds that many warps).
constexpr int kAsyncThreads = 256;
template <int K, int CH, int PLANE, bool STATS>
__global__ void __launch_bounds__(kAsyncThreads) embedk_units_async(KView a)
{
    grid_dependency_wait(); // launched dependent: nothing is touched before
    allow_dependents();
    static_assert(CH > 1, "plane units only");
    constexpr uint32_t MASK = (1u << K) - 1u;
    constexpr uint32_t BYTEMASK = MASK * 0x01010101u;
    constexpr uint32_t SV = unit_stage_slots<CH>();
    __shared__ uint4 stage[(kAsyncThreads / 32) * 2 * SV];
    uint4 *const sw = stage + (threadIdx.x >> 5) * 2 * SV;
    const uint32_t lane = threadIdx.x & 31u;
    unsigned long long changed = 0, sse = 0;
    embed_res(a, STATS);
    const uint64_t nunits = a.n_carry >> 4;
    const uint64_t vend = nunits * CH;
    const uint4 *__restrict__ cv = reinterpret_cast<const uint4 *>(a.cover);
    uint4 *const ov = reinterpret_cast<uint4 *>(a.stego);
    const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
    auto issue = [&](uint64_t ub, uint32_t s) { // the warp's vectors from unit ub -> stage s
        const uint64_t v0 = ub * CH;
#pragma unroll
        for (int j = 0; j < CH; ++j)
            if (v0 + 32u * j + lane < vend)
                cp_async16(sw + s * SV + unit_stage_slot<CH>(32u * j + lane), cv + v0 + 32u * j + lane);
        cp_async_commit();
    };
    auto window = [&](uint64_t u) {
        return (u < nunits && u < a.full_units) ? stream_window<K>(a, u) : 0ull;
    };
    uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; // u - lane: the same for the warp
    if (u - lane < nunits) {
        issue(u - lane, 0);
        uint64_t X = window(u);
        uint32_t s = 0;
        for (;;) {
            const uint64_t un = u + step;
            const bool next = un - lane < nunits;
            uint64_t Xn = 0;
            if (next) {
                issue(un - lane, s ^ 1u);
                Xn = window(un);
                cp_async_wait<1>(); // this iteration's copies landed (the next may be pending)
            } else {
                cp_async_wait<0>();
            }
            __syncwarp(); // every lane's copies visible to the warp
            uint4 *const st = sw + s * SV;
            if (u < nunits && u < a.part_units) {
                uint32_t w[4 * CH];
#pragma unroll
                for (int q = 0; q < CH; ++q) {
                    const uint4 t = st[unit_stage_slot<CH>(CH * lane + q)];
                    w[4 * q] = t.x;
                    w[4 * q + 1] = t.y;
                    w[4 * q + 2] = t.z;
                    w[4 * q + 3] = t.w;
                }
                uint32_t c[4], o[4];
                gather_unit<CH, PLANE>(w, c);
                if (u < a.full_units) {
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        o[i] = (c[i] & ~BYTEMASK) | unit_fields<K>(X, i);
                } else {
                    const uint4 e = stream_end_vector(a, u, make_uint4(c[0], c[1], c[2], c[3]));
                    o[0] = e.x;
                    o[1] = e.y;
                    o[2] = e.z;
                    o[3] = e.w;
                }
                uint32_t d[4];
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    d[i] = o[i] ^ c[i];
                if (STATS)
                    unit_stats<K>(o, c, d, a.kmul, changed, sse);
                scatter_xor<CH, PLANE>(w, d);
#pragma unroll
                for (int q = 0; q < CH; ++q)
                    st[unit_stage_slot<CH>(CH * lane + q)] =
                        make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
            }
            __syncwarp(); // the rewritten units visible to the storing lanes
            const uint64_t v0 = (u - lane) * CH;
#pragma unroll
            for (int j = 0; j < CH; ++j)
                if (v0 + 32u * j + lane < vend)
                    __stcs(ov + v0 + 32u * j + lane, st[unit_stage_slot<CH>(32u * j + lane)]);
            if (!next)
                break;
            // stage s is refilled two iterations on, after this lane's reads
            // of its own memory-order slots above
            X = Xn;
            u = un;
            s ^= 1u;
        }
    }
    // cover bytes of the carrying bytes after the last whole unit: plane
    // bytes take their field, the other bytes of those pixels are copied
    if (blockIdx.x == 0 && threadIdx.x < (uint32_t)(a.n_carry & 15u) * CH) {
        const uint64_t pbyte = ((a.n_carry >> 4) << 4) * CH + threadIdx.x;
        const uint32_t cb = a.cover[pbyte];
        uint32_t ob = cb;
        if (threadIdx.x % CH == PLANE) {
            uint32_t fv, fm;
            field_of(a, pbyte / CH, fv, fm);
            ob = (cb & ~fm) | (fv & fm);
        }
        a.stego[pbyte] = (uint8_t)ob;
        if (STATS) {
            const uint32_t dd = ob > cb ? ob - cb : cb - ob;
            changed += dd != 0;
            sse += dd * dd;
        }
    }
    if (STATS)
        block_stats(changed, sse, a.res, a.slot);
}

// One thread per carrying byte x < n_carry (all bytes: the bytes past the
// stream are copied; one plane: only plane bytes are written).
template <bool STATS>
__global__ void __launch_bounds__(512) embedk_bytes(KView a)
{
    grid_dependency_wait(); // launched dependent: nothing is touched before
    allow_dependents();
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
        block_stats(changed, sse, a.res, a.slot);
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

// k = 3 units of the extract: unit u yields the 6 stream bytes [6u, 6u + 6),
// so a lane pair (units 2j, 2j + 1) holds 12 consecutive message bytes and
// writes them as three aligned words: the even lane its first four bytes
// and its last two joined to the odd lane's first two (one shuffle), the
// odd lane its last four.  The loop runs while the warp's first unit is in
// range, so every lane reaches the shuffle; pairs at the header, at the
// message's end or on an unaligned output store 16-bit halves or bytes.
template <int CH, int PLANE>
__device__ __forceinline__ void extract3_units(const KView &a, uint64_t nunits, uint64_t hb,
                                               uint64_t sbytes)
{
    constexpr int U = units_per_iter<CH, false>();
    const uint32_t lane = threadIdx.x & 31u;
    const bool odd = (lane & 1u) != 0;
    // stream byte 12j lands at out + 12j - hb: word-aligned for every j or none
    const bool words = (((uintptr_t)a.out - hb) & 3u) == 0;
    for (uint64_t u0 = (uint64_t)blockIdx.x * blockDim.x * U + threadIdx.x; u0 - lane < nunits;
         u0 += (uint64_t)gridDim.x * blockDim.x * U) {
        uint32_t w[U][4 * CH];
#pragma unroll
        for (int r = 0; r < U; ++r) {
            const uint64_t u = u0 + (uint64_t)r * blockDim.x;
            if (u < nunits) {
                load_unit<CH>(a.cover, u, w[r]);
            } else {
#pragma unroll
                for (int j = 0; j < 4 * CH; ++j)
                    w[r][j] = 0;
            }
        }
#pragma unroll
        for (int r = 0; r < U; ++r) {
            const uint64_t u = u0 + (uint64_t)r * blockDim.x;
            uint32_t g[4], v01, v23;
            gather_unit<CH, PLANE>(w[r], g);
            unit_window3(g, v01, v23);
            const uint32_t P = __byte_perm(v01, v23, 0x6012u); // stream bytes 0-3, memory order
            const uint32_t Q = __byte_perm(v23, 0u, 0x4401u);  // stream bytes 4-5
            const uint32_t Pn = __shfl_down_sync(0xFFFFFFFFu, P, 1);
            const uint64_t q2 = 6u * (u & ~1ull); // first stream byte of the pair
            if (words && (u | 1u) < nunits && q2 >= hb && q2 + 12 <= sbytes) {
                uint32_t *op = reinterpret_cast<uint32_t *>(a.out + (q2 - hb));
                if (odd) {
                    op[2] = __byte_perm(P, Q, 0x5432u);
                } else {
                    op[0] = P;
                    op[1] = __byte_perm(Q, Pn, 0x5410u);
                }
            } else if (u < nunits) {
                const uint64_t q0 = 6u * u; // first stream byte of the unit
                if (q0 >= hb && q0 + 6 <= sbytes && ((q0 - hb + (uintptr_t)a.out) & 1u) == 0) {
                    unsigned short *op = reinterpret_cast<unsigned short *>(a.out + (q0 - hb));
                    op[0] = (unsigned short)P;
                    op[1] = (unsigned short)(P >> 16);
                    op[2] = (unsigned short)Q;
                } else {
#pragma unroll
                    for (int i = 0; i < 6; ++i) {
                        const uint64_t q = q0 + i;
                        if (q >= hb && q < sbytes)
                            a.out[q - hb] = (uint8_t)(i < 3 ? v01 >> (16 - 8 * i) : v23 >> (40 - 8 * i));
                    }
                }
            }
        }
    }
}

// Extract over units (stego 16-byte aligned): unit u yields stream bytes
// [2Ku, 2Ku + 2K); U units per thread per iteration, loads first.  Stream
// bytes past the last whole unit go bit by bit.
template <int K, int CH, int PLANE>
__global__ void __launch_bounds__(512) extractk_units(KView a)
{
    grid_dependency_wait(); // launched dependent: nothing is touched before
    allow_dependents();
    uint64_t len;
    if (extractk_prologue(a, len) != STEGO_OK)
        return;
    const uint64_t hb = a.header ? 4u : 0u;       // stream bytes before the message
    const uint64_t sbytes = len + hb;              // stream bytes to recover
    const uint64_t want = (sbytes + 2 * K - 1) / (2 * K);
    const uint64_t nunits = want < (a.n_carry >> 4) ? want : (a.n_carry >> 4);
    for (uint64_t q = 2u * K * nunits + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
         q < sbytes; q += (uint64_t)gridDim.x * blockDim.x) {
        if (q < hb)
            continue;
        uint32_t v = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i)
            v |= stream_bit(a, 8u * q + i) << (7 - i);
        a.out[q - hb] = (uint8_t)v;
    }
    if constexpr (K == 3) {
        extract3_units<CH, PLANE>(a, nunits, hb, sbytes);
        return;
    }
    constexpr int U = units_per_iter<CH, false>();
    for (uint64_t u0 = (uint64_t)blockIdx.x * blockDim.x * U + threadIdx.x; u0 < nunits;
         u0 += (uint64_t)gridDim.x * blockDim.x * U) {
        uint32_t w[U][4 * CH];
#pragma unroll
        for (int r = 0; r < U; ++r) {
            const uint64_t u = u0 + (uint64_t)r * blockDim.x;
            if (u < nunits)
                load_unit<CH>(a.cover, u, w[r]);
        }
#pragma unroll
        for (int r = 0; r < U; ++r) {
            const uint64_t u = u0 + (uint64_t)r * blockDim.x;
            if (u >= nunits)
                continue;
            uint32_t g[4];
            gather_unit<CH, PLANE>(w[r], g);
            const uint64_t X = unit_window<K>(g);
            const uint64_t q0 = 2u * K * u; // first stream byte of the unit
            uint8_t *op = a.out + (q0 - hb);
            if ((K & 1) == 0 && q0 >= hb && q0 + 2 * K <= sbytes &&
                (((uintptr_t)op & 3u) == 0)) {
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
}

// Any alignment, any k, either carrying order: one thread per message byte.
__global__ void __launch_bounds__(512) extractk_bytes(KView a)
{
    grid_dependency_wait(); // launched dependent: nothing is touched before
    allow_dependents();
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

// Unit kernels exist for 1, 3 and 4 channels.
bool unit_layout(bool plane_only, const stego_geom *g)
{
    return !plane_only || g->channels == 1 || g->channels == 3 || g->channels == 4;
}

template <int K, bool STATS>
const void *embed_units_for(uint32_t ch, uint32_t plane)
{
    if (ch == 1)
        return (const void *)embedk_units<K, 1, 0, STATS>;
    if (ch == 3) {
        switch (plane) {
        case 0: return (const void *)embedk_units_async<K, 3, 0, STATS>;
        case 1: return (const void *)embedk_units_async<K, 3, 1, STATS>;
        default: return (const void *)embedk_units_async<K, 3, 2, STATS>;
        }
    }
    switch (plane) {
    case 0: return (const void *)embedk_units_async<K, 4, 0, STATS>;
    case 1: return (const void *)embedk_units_async<K, 4, 1, STATS>;
    case 2: return (const void *)embedk_units_async<K, 4, 2, STATS>;
    default: return (const void *)embedk_units_async<K, 4, 3, STATS>;
    }
}

template <bool STATS>
const void *embed_units_kernel(uint32_t k, uint32_t ch, uint32_t plane)
{
    switch (k) {
    case 1: return embed_units_for<1, STATS>(ch, plane);
    case 2: return embed_units_for<2, STATS>(ch, plane);
    case 3: return embed_units_for<3, STATS>(ch, plane);
    default: return embed_units_for<4, STATS>(ch, plane);
    }
}

template <int K>
const void *extract_units_for(uint32_t ch, uint32_t plane)
{
    if (ch == 1)
        return (const void *)extractk_units<K, 1, 0>;
    if (ch == 3) {
        switch (plane) {
        case 0: return (const void *)extractk_units<K, 3, 0>;
        case 1: return (const void *)extractk_units<K, 3, 1>;
        default: return (const void *)extractk_units<K, 3, 2>;
        }
    }
    switch (plane) {
    case 0: return (const void *)extractk_units<K, 4, 0>;
    case 1: return (const void *)extractk_units<K, 4, 1>;
    case 2: return (const void *)extractk_units<K, 4, 2>;
    default: return (const void *)extractk_units<K, 4, 3>;
    }
}

const void *extract_units_kernel(uint32_t k, uint32_t ch, uint32_t plane)
{
    switch (k) {
    case 1: return extract_units_for<1>(ch, plane);
    case 2: return extract_units_for<2>(ch, plane);
    case 3: return extract_units_for<3>(ch, plane);
    default: return extract_units_for<4>(ch, plane);
    }
}

} // namespace

cudaError_t sk_embed(const uint8_t *cover, uint8_t *stego, uint64_t C, uint32_t k, bool plane_only,
                     const stego_geom *g, const uint8_t *msg, uint64_t m, bool header,
                     bool stats, stego_result *res, const Shape &sh, cudaStream_t s,
                     StatSlot *slot)
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
    a.slot = stats ? slot : nullptr;
    a.full_units = a.t_bits / (16u * k);
    a.part_units = (a.t_bits + 16u * k - 1) / (16u * k);
    a.msg_w4 = (((uintptr_t)msg - (header ? 4u : 0u)) & 3u) == 0;
    a.msg_w2 = (((uintptr_t)msg - (header ? 4u : 0u)) & 1u) == 0;
    a.kmul = 1u << k;
    const bool inplace = cover == stego;
    const uint64_t t_carry = (a.t_bits + k - 1) / k; // carrying bytes the stream uses
    const int T = sh.threads;
    void *args[] = {&a};
    if (aligned16(cover) && aligned16(stego) && unit_layout(plane_only, g)) {
        // carrying bytes processed: all of them out of place (the rest of
        // the cover is copied with them), those the stream uses in place
        a.n_carry = inplace ? t_carry : (plane_only ? (uint64_t)g->width * g->height : C);
        const void *kern = stats ? embed_units_kernel<true>(k, a.channels, a.plane)
                                 : embed_units_kernel<false>(k, a.channels, a.plane);
        const uint64_t nunits = a.n_carry >> 4;
        const int per_thread = a.channels == 1 ? kEmbedAllBytesUnits : 1;
        const int TU = a.channels == 1 ? T : kAsyncThreads; // plane units: the pipeline's CTAs
        const int grid = persistent_grid(kern, TU, 0, kAnyCtas, nunits ? nunits : 1,
                                         (uint64_t)TU * per_thread);
        return launch_dependent(kern, dim3(grid), dim3(TU), args, 0, s);
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
    const int grid = persistent_grid(kern, T, 0, kAnyCtas, a.n_carry ? a.n_carry : 1,
                                     (uint64_t)T * 16);
    return launch_dependent(kern, dim3(grid), dim3(T), args, 0, s);
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
    if (aligned16(st) && unit_layout(plane_only, g)) {
        const void *kern = extract_units_kernel(k, a.channels, a.plane);
        const uint64_t nunits = (max_len + 4 + 2 * k - 1) / (2 * k);
        const int per_thread = a.channels == 1 ? kExtractAllBytesUnits : 1;
        const int grid = persistent_grid(kern, T, 0, kAnyCtas, nunits ? nunits : 1,
                                         (uint64_t)T * per_thread);
        return launch_dependent(kern, dim3(grid), dim3(T), args, 0, s);
    }
    const void *kern = (const void *)extractk_bytes;
    const int grid = persistent_grid(kern, T, 0, kAnyCtas, max_len ? max_len : 1, (uint64_t)T);
    return launch_dependent(kern, dim3(grid), dim3(T), args, 0, s);
}

} // namespace stego
