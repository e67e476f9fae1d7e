// s1_device.cuh -- device routines of the one-bit stream layout, shared by
// the single-cover kernels (stream1.cu) and the persistent batched kernels
// (batched.cu), so both run exactly the same per-vector code.
//
//   stego[k] = (cover[k] & 0xFE) | ((S[k/8] >> (7 - k%8)) & 1)   for k < T,
//   stego[k] = cover[k]                                           for k >= T,
//   S = BE32(8m) || msg (header) or S = msg,  T = 8|S|,
//   msg[s] = sum_b (stego[base + 8s + b] & 1) << (7 - b),  base = 32 or 0.
#pragma once

#include "internal.cuh"

namespace stego {
namespace s1 {

// One embedding job: cover/stego bytes [0, n_bytes) are written, bytes
// below t_bytes carry stream bits.
struct EmbedView {
    const uint8_t *cover;
    uint8_t *stego;
    const uint8_t *msg;
    uint64_t n_bytes; // bytes written (C out of place, T in place)
    uint64_t t_bytes; // carrying bytes, 8 * slen
    uint64_t slen;    // stream bytes
    uint32_t header;  // S starts with BE32(nbits)
    uint32_t nbits;
    uint32_t msg_even; // msg pointer is 2-byte aligned
    uint32_t pad;
};

// One extraction job: message bytes [0, len) from stego bytes starting at
// `base` (32 behind a header, 0 otherwise).
struct ExtractView {
    const uint8_t *st;
    uint8_t *msg;
    uint64_t len;
    uint64_t base;
    uint32_t msg_even;
    uint32_t pad;
};

// Byte q < slen of the stream S.
__device__ __forceinline__ uint32_t stream_byte(const EmbedView &a, uint64_t q)
{
    if (a.header) {
        if (q < 4)
            return (a.nbits >> (24u - 8u * (uint32_t)q)) & 0xFFu;
        return __ldg(a.msg + (q - 4));
    }
    return __ldg(a.msg + q);
}

// Stream bytes q and q+1 (q even) as S[q] | S[q+1] << 8; bytes at or past
// slen read as 0.
__device__ __forceinline__ uint32_t stream_pair(const EmbedView &a, uint64_t q)
{
    if (q + 1 < a.slen && (!a.header || q >= 4) && a.msg_even)
        return __ldg(reinterpret_cast<const unsigned short *>(a.msg + (a.header ? q - 4 : q)));
    uint32_t r = 0;
    if (q < a.slen)
        r = stream_byte(a, q);
    if (q + 1 < a.slen)
        r |= stream_byte(a, q + 1) << 8;
    return r;
}

// The eight bits of a stream byte, most significant first, moved to bit 0 of
// eight consecutive bytes.  `rep` holds the stream byte in all four byte
// lanes (one __byte_perm).  Selecting bit 7-i in lane i and adding 0x7F to
// every lane sets the lane's bit 7 exactly when the selected bit was set (no
// carry leaves a lane); >> 7 brings it to bit 0.
__device__ __forceinline__ uint32_t spread_hi(uint32_t rep)
{ // cover bytes 0..3 <- bits 7..4
    return (((rep & 0x10204080u) + 0x7F7F7F7Fu) >> 7) & 0x01010101u;
}
__device__ __forceinline__ uint32_t spread_lo(uint32_t rep)
{ // cover bytes 4..7 <- bits 3..0
    return (((rep & 0x01020408u) + 0x7F7F7F7Fu) >> 7) & 0x01010101u;
}

// Changed bytes of one embedded vector.  Only bit 0 of a byte can differ
// between cover and stego in this layout, so each word of (stego ^ cover)
// has at most the four bits 0, 8, 16, 24 set; the four words shifted by 0..3
// bits never overlap, and one population count of their OR is the number
// of changed bytes.  Each changed byte moves by exactly one, so the same
// count is also the vector's squared error.
__device__ __forceinline__ uint32_t vec_changes(const uint4 &o, const uint4 &c)
{
    return __popc((o.x ^ c.x) | ((o.y ^ c.y) << 1) | ((o.z ^ c.z) << 2) | ((o.w ^ c.w) << 3));
}

// Cover vector v (bytes 16v..16v+15) with its stream bytes p = S[2v] |
// S[2v+1] << 8 -> stego vector; n += changed bytes when STATS.
template <bool STATS>
__device__ __forceinline__ uint4 embed_vec16(const EmbedView &a, uint64_t v, const uint4 &c,
                                             uint32_t p, uint32_t &n)
{
    uint4 o = c;
    const uint64_t k0 = v << 4;
    if (k0 < a.t_bytes) {
        const uint32_t r0 = __byte_perm(p, 0u, 0x0000u);
        o.x = (c.x & 0xFEFEFEFEu) | spread_hi(r0);
        o.y = (c.y & 0xFEFEFEFEu) | spread_lo(r0);
        if (k0 + 8 < a.t_bytes) { // T is a multiple of 8
            const uint32_t r1 = __byte_perm(p, 0u, 0x1111u);
            o.z = (c.z & 0xFEFEFEFEu) | spread_hi(r1);
            o.w = (c.w & 0xFEFEFEFEu) | spread_lo(r1);
        }
        if (STATS)
            n += vec_changes(o, c);
    }
    return o;
}

// 16-byte vectors v = v_first + i*step (+ u*blockDim.x for u < V), v < v_end,
// of a job whose cover and stego are 16-byte aligned.  Each warp's 128-bit
// load and store instructions cover 512 contiguous bytes.  With STATS the
// changed-byte count (= squared error, see vec_changes) is added to both
// accumulators.
template <int V, bool STATS>
__device__ __forceinline__ void embed_vec_range(const EmbedView &a, uint64_t v_first,
                                                uint64_t v_end, uint64_t step,
                                                unsigned long long &changed,
                                                unsigned long long &sse)
{
    const uint4 *__restrict__ src = reinterpret_cast<const uint4 *>(a.cover);
    uint4 *dst = reinterpret_cast<uint4 *>(a.stego);
    // changed bytes of this call in 32 bits: a thread covers at most
    // (bytes / threads) bytes, far below 2^32 for any cover in device memory
    uint32_t n = 0;
    // vectors [fast_lo, fast_hi) carry message bytes only (two per vector, a
    // 16-bit load when the message is 2-byte aligned) in all 16 bytes
    const uint64_t fast_lo = a.header ? 2u : 0u;
    const uint64_t fast_hi = a.msg_even ? (a.t_bytes >> 4) : 0u;
    const unsigned short *__restrict__ mw =
        reinterpret_cast<const unsigned short *>(a.msg) - fast_lo;
    for (uint64_t v0 = v_first; v0 < v_end; v0 += step) {
        uint4 c[V];
        uint32_t p[V];
        const uint64_t vlast = v0 + (uint64_t)(V - 1) * blockDim.x;
        if (v0 >= fast_lo && vlast < fast_hi && vlast < v_end) {
            // the whole round inside the message: no per-vector checks
#pragma unroll
            for (int u = 0; u < V; ++u)
                c[u] = __ldcs(src + v0 + (uint64_t)u * blockDim.x);
#pragma unroll
            for (int u = 0; u < V; ++u)
                p[u] = __ldg(mw + v0 + (uint64_t)u * blockDim.x);
#pragma unroll
            for (int u = 0; u < V; ++u) {
                const uint32_t r0 = __byte_perm(p[u], 0u, 0x0000u);
                const uint32_t r1 = __byte_perm(p[u], 0u, 0x1111u);
                uint4 o;
                o.x = (c[u].x & 0xFEFEFEFEu) | spread_hi(r0);
                o.y = (c[u].y & 0xFEFEFEFEu) | spread_lo(r0);
                o.z = (c[u].z & 0xFEFEFEFEu) | spread_hi(r1);
                o.w = (c[u].w & 0xFEFEFEFEu) | spread_lo(r1);
                if (STATS)
                    n += vec_changes(o, c[u]);
                __stcs(dst + v0 + (uint64_t)u * blockDim.x, o);
            }
            continue;
        }
#pragma unroll
        for (int u = 0; u < V; ++u) {
            const uint64_t v = v0 + (uint64_t)u * blockDim.x;
            if (v < v_end)
                c[u] = __ldcs(src + v);
        }
#pragma unroll
        for (int u = 0; u < V; ++u) {
            const uint64_t v = v0 + (uint64_t)u * blockDim.x;
            p[u] = 0;
            if (v < v_end && (v << 4) < a.t_bytes)
                p[u] = stream_pair(a, v << 1);
        }
#pragma unroll
        for (int u = 0; u < V; ++u) {
            const uint64_t v = v0 + (uint64_t)u * blockDim.x;
            if (v >= v_end)
                continue;
            __stcs(dst + v, embed_vec16<STATS>(a, v, c[u], p[u], n));
        }
    }
    if (STATS) {
        changed += n;
        sse += n;
    }
}

// ---------------------------------------------------------------------------
// Misaligned buffers
// ---------------------------------------------------------------------------

// Byte q of the stream, 0 at or past its end.
__device__ __forceinline__ uint32_t stream_byte_or0(const EmbedView &a, uint64_t q)
{
    return q < a.slen ? stream_byte(a, q) : 0u;
}

// The stream bits of cover bytes k0..k0+15 for any k0, as S[2v] | S[2v+1]
// << 8 would give them for k0 = 16v: three stream bytes, cut at bit k0 % 8.
// Inside the message (stream bytes q-3 .. q+7 all message bytes) the three
// come from the two aligned 32-bit words around them, joined by a funnel
// shift; elsewhere byte by byte.
__device__ __forceinline__ uint32_t stream_bits16(const EmbedView &a, uint64_t k0)
{
    const uint64_t q = k0 >> 3;
    const uint64_t hdr = a.header ? 4u : 0u;
    uint32_t w;
    if (q >= hdr + 3 && q + 7 < a.slen) {
        const uintptr_t pa = (uintptr_t)(a.msg + (q - hdr));
        const uint32_t *wp = reinterpret_cast<const uint32_t *>(pa & ~(uintptr_t)3u);
        const uint32_t b = __funnelshift_r(__ldg(wp), __ldg(wp + 1), 8u * (uint32_t)(pa & 3u));
        w = __byte_perm(b, 0u, 0x4012u); // S[q] << 16 | S[q+1] << 8 | S[q+2]
    } else {
        w = (stream_byte_or0(a, q) << 16) | (stream_byte_or0(a, q + 1) << 8) |
            stream_byte_or0(a, q + 2);
    }
    const uint32_t bits = (w >> (8u - (uint32_t)(k0 & 7u))) & 0xFFFFu; // byte k0's bit on top
    return (bits >> 8) | ((bits & 0xFFu) << 8);
}

// The 16 stream bits of a vector from the stream bytes b = S[q] | S[q+1] << 8
// | S[q+2] << 16 (little-endian word) cut at bit s of S[q], as S[2v] |
// S[2v+1] << 8 would give them for an aligned vector.
__device__ __forceinline__ uint32_t bits16_from(uint32_t b, uint32_t s)
{
    const uint32_t w = __byte_perm(b, 0u, 0x4012u); // S[q] << 16 | S[q+1] << 8 | S[q+2]
    const uint32_t bits = (w >> (8u - s)) & 0xFFFFu;
    return (bits >> 8) | ((bits & 0xFFu) << 8);
}

// Cover vector c with its 16 stream bits p (as S[2v] | S[2v+1] << 8) ->
// stego vector, all 16 bytes carrying.
__device__ __forceinline__ uint4 spread16(const uint4 &c, uint32_t p)
{
    const uint32_t r0 = __byte_perm(p, 0u, 0x0000u);
    const uint32_t r1 = __byte_perm(p, 0u, 0x1111u);
    uint4 o;
    o.x = (c.x & 0xFEFEFEFEu) | spread_hi(r0);
    o.y = (c.y & 0xFEFEFEFEu) | spread_lo(r0);
    o.z = (c.z & 0xFEFEFEFEu) | spread_hi(r1);
    o.w = (c.w & 0xFEFEFEFEu) | spread_lo(r1);
    return o;
}

// Whether the vectors at cover bytes k_first .. k_last + 15 (k = h + 16j)
// all carry stream bits in every byte and have their stream windows inside
// the message (the fast paths' condition).
__device__ __forceinline__ bool window_inner(const EmbedView &a, uint64_t k_first, uint64_t k_last)
{
    const uint64_t hdr = a.header ? 4u : 0u;
    return k_last + 16u <= a.t_bytes && (k_first >> 3) >= hdr + 3u && (k_last >> 3) + 7u < a.slen;
}

// A vector that holds the end of the carrying bytes: bytes from t on keep
// the cover.
static __device__ __noinline__ uint4 keep_past_end(uint4 o, const uint4 &c, uint32_t carrying)
{
    uint32_t ow[4] = {o.x, o.y, o.z, o.w};
    const uint32_t cw[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int n = (int)carrying - 4 * i; // carrying bytes in word i
        const uint32_t m = n >= 4 ? 0xFFFFFFFFu : (n <= 0 ? 0u : (1u << (8 * n)) - 1u);
        ow[i] = (ow[i] & m) | (cw[i] & ~m);
    }
    return make_uint4(ow[0], ow[1], ow[2], ow[3]);
}

// Cover bytes k0..k0+15 (any k0, the vector itself 16-byte aligned) with
// their stream bits p -> stego vector; n += changed bytes when STATS.
template <bool STATS>
__device__ __forceinline__ uint4 embed_vec16_at(const EmbedView &a, uint64_t k0, const uint4 &c,
                                                uint32_t p, uint32_t &n)
{
    if (k0 >= a.t_bytes)
        return c;
    uint4 o;
    const uint32_t r0 = __byte_perm(p, 0u, 0x0000u);
    const uint32_t r1 = __byte_perm(p, 0u, 0x1111u);
    o.x = (c.x & 0xFEFEFEFEu) | spread_hi(r0);
    o.y = (c.y & 0xFEFEFEFEu) | spread_lo(r0);
    o.z = (c.z & 0xFEFEFEFEu) | spread_hi(r1);
    o.w = (c.w & 0xFEFEFEFEu) | spread_lo(r1);
    if (k0 + 16 > a.t_bytes)
        o = keep_past_end(o, c, (uint32_t)(a.t_bytes - k0));
    if (STATS)
        n += vec_changes(o, c);
    return o;
}

// Cover and stego with the same misalignment: h = (-cover) mod 16 head
// bytes, then aligned vectors j at cover + h + 16j (j < j_end), each with
// the stream bits of bytes h + 16j onwards.  Head and tail bytes are left to
// the caller.
template <int V, bool STATS>
__device__ __forceinline__ void embed_shift_range(const EmbedView &a, uint32_t h,
                                                  uint64_t j_first, uint64_t j_end,
                                                  uint64_t step, unsigned long long &changed,
                                                  unsigned long long &sse)
{
    const uint4 *__restrict__ src = reinterpret_cast<const uint4 *>(a.cover + h);
    uint4 *dst = reinterpret_cast<uint4 *>(a.stego + h);
    uint32_t n = 0;
    // cover byte h + 16j carries stream bit h + 16j: stream byte h/8 + 2j
    // (message byte m0 + 2j), cut at bit h % 8
    const uintptr_t m0 = (uintptr_t)a.msg + (h >> 3) - (a.header ? 4u : 0u);
    const uint32_t bsh = h & 7u;
    for (uint64_t j0 = j_first; j0 < j_end; j0 += step) {
        uint4 c[V];
        uint32_t p[V];
        const uint64_t jl = j0 + (uint64_t)(V - 1) * blockDim.x;
        if (jl < j_end && window_inner(a, h + (j0 << 4), h + (jl << 4))) {
            // the whole round inside the message: no per-vector checks
#pragma unroll
            for (int u = 0; u < V; ++u)
                c[u] = __ldcs(src + j0 + (uint64_t)u * blockDim.x);
            // the V windows start 2 * blockDim.x message bytes apart, a
            // multiple of 4: the same offset within an aligned word
            const uintptr_t pm = m0 + 2u * j0;
            const uint32_t *__restrict__ wp =
                reinterpret_cast<const uint32_t *>(pm & ~(uintptr_t)3u);
            const uint32_t wsh = 8u * (uint32_t)(pm & 3u);
#pragma unroll
            for (int u = 0; u < V; ++u) {
                const uint32_t *w = wp + (uint64_t)u * (blockDim.x >> 1);
                p[u] = bits16_from(__funnelshift_r(__ldg(w), __ldg(w + 1), wsh), bsh);
            }
#pragma unroll
            for (int u = 0; u < V; ++u) {
                const uint4 o = spread16(c[u], p[u]);
                if (STATS)
                    n += vec_changes(o, c[u]);
                __stcs(dst + j0 + (uint64_t)u * blockDim.x, o);
            }
            continue;
        }
        if (jl < j_end && h + (j0 << 4) >= a.t_bytes) {
            // the whole round past the carrying bytes: a copy, all loads
            // first
#pragma unroll
            for (int u = 0; u < V; ++u)
                c[u] = __ldcs(src + j0 + (uint64_t)u * blockDim.x);
#pragma unroll
            for (int u = 0; u < V; ++u)
                __stcs(dst + j0 + (uint64_t)u * blockDim.x, c[u]);
            continue;
        }
        // a round at an edge: one vector at a time, with the checks
#pragma unroll 1
        for (int u = 0; u < V; ++u) {
            const uint64_t j = j0 + (uint64_t)u * blockDim.x;
            if (j >= j_end)
                break;
            const uint64_t k0 = h + (j << 4);
            const uint32_t pw = k0 < a.t_bytes ? stream_bits16(a, k0) : 0u;
            __stcs(dst + j, embed_vec16_at<STATS>(a, k0, __ldcs(src + j), pw, n));
        }
    }
    if (STATS) {
        changed += n;
        sse += n;
    }
}

// 16 bytes starting at byte 4Q + b of the 32 bytes lo:hi (lo first);
// sel = b | (b+1) << 4 | (b+2) << 8 | (b+3) << 12 selects them per word.
template <int Q>
__device__ __forceinline__ uint4 funnel16(const uint4 &lo, const uint4 &hi, uint32_t sel)
{
    const uint32_t w[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
    return make_uint4(__byte_perm(w[Q], w[Q + 1], sel), __byte_perm(w[Q + 1], w[Q + 2], sel),
                      __byte_perm(w[Q + 2], w[Q + 3], sel), __byte_perm(w[Q + 3], w[Q + 4], sel));
}

// The aligned vector after lane l's lo[u] in a warp's block of 32*V
// consecutive vectors (lane l + 1's lo[u]; for lane 31 lane 0's lo[u + 1], or
// x, the vector after the block): one shuffle per word.  Lane 0's offer is
// read only by lane 31.
template <int V>
__device__ __forceinline__ uint4 next_vec(const uint4 (&lo)[V], const uint4 &x, int u,
                                          uint32_t lane)
{
    const uint4 give = lane == 0 ? (u + 1 < V ? lo[u + 1 < V ? u + 1 : u] : x) : lo[u];
    const uint32_t src = (lane + 1u) & 31u;
    return make_uint4(__shfl_sync(0xFFFFFFFFu, give.x, src), __shfl_sync(0xFFFFFFFFu, give.y, src),
                      __shfl_sync(0xFFFFFFFFu, give.z, src), __shfl_sync(0xFFFFFFFFu, give.w, src));
}

// Stego vector j of embed_funnel_warp with every check: its cover bytes
// from the two aligned cover vectors around them when both lie inside the
// cover, else one by one; returns its changed bytes (0 without STATS).
template <int Q, bool STATS>
static __device__ __noinline__ uint32_t funnel_edge_vec(const EmbedView &a, uint32_t h,
                                                        uint32_t sel, uint64_t j)
{
    const uint4 *A = reinterpret_cast<const uint4 *>((uintptr_t)(a.cover + h) & ~(uintptr_t)15u);
    const uintptr_t lo_ok = (uintptr_t)a.cover, hi_ok = (uintptr_t)a.cover + a.n_bytes;
    const uintptr_t b = (uintptr_t)(A + j);
    const uint64_t k0 = h + (j << 4);
    uint4 c;
    if (b >= lo_ok && b + 32u <= hi_ok) {
        const uint4 lo = __ldcs(A + j), hi = __ldcs(A + j + 1);
        c = funnel16<Q>(lo, hi, sel);
    } else {
        uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int t = 0; t < 16; ++t)
            w[t >> 2] |= (uint32_t)a.cover[k0 + t] << (8 * (t & 3));
        c = make_uint4(w[0], w[1], w[2], w[3]);
    }
    const uint32_t p = k0 < a.t_bytes ? stream_bits16(a, k0) : 0u;
    uint32_t n = 0;
    __stcs(reinterpret_cast<uint4 *>(a.stego + h) + j, embed_vec16_at<STATS>(a, k0, c, p, n));
    return n;
}

// Cover and stego at different addresses mod 16 (out of place, n_bytes =
// C): h = (-stego) mod 16 head bytes, then aligned stego vectors j at stego
// + h + 16j (j_lo <= j < j_hi).  The cover bytes of vector j, h + 16j .. h +
// 16j + 15, start at byte d = (cover + h) mod 16 = 4Q + (sel's b) of the
// aligned cover vector A[j] at or below them: they are A[j]'s last 16 - d
// bytes and A[j + 1]'s first d, joined by funnel16.
//
// Warp `warp` of `nwarps` takes rounds of 32*V consecutive stego vectors,
// lane l vectors r + 32u + l.  Each lane loads only its own A[j]; A[j + 1] is
// the next lane's, passed by one shuffle per word, and lane 31's is the
// next block's first vector (lane 0 passes A[r + 32(u+1)], and one extra
// vector A[r + 32V] per round): one cover load per stego vector, and 4V + 4
// registers of cover data in flight where the two-load form needs 8V.
// Rounds wholly inside the cover and the message (or wholly past the
// carrying bytes: a copy) run without per-vector tests; a round at an edge
// goes vector by vector, reading its 16 cover bytes one by one where A[j] or
// A[j + 1] is not inside the cover.  Head and tail bytes are left to the
// caller.
template <int Q, bool STATS, int V>
__device__ __forceinline__ void embed_funnel_warp(const EmbedView &a, uint32_t h, uint32_t sel,
                                                  uint64_t j_lo, uint64_t j_hi, uint64_t warp,
                                                  uint64_t nwarps, unsigned long long &changed,
                                                  unsigned long long &sse)
{
    const uintptr_t c0 = (uintptr_t)(a.cover + h);
    const uint4 *__restrict__ A = reinterpret_cast<const uint4 *>(c0 & ~(uintptr_t)15u);
    const uintptr_t lo_ok = (uintptr_t)a.cover, hi_ok = (uintptr_t)a.cover + a.n_bytes;
    uint4 *dst = reinterpret_cast<uint4 *>(a.stego + h);
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t n = 0;
    // stego vectors [safe_lo, safe_hi) have both cover vectors inside the cover
    const uint64_t safe_lo = (uintptr_t)A >= lo_ok ? 0u : 1u;
    const uint64_t nv = (hi_ok - (uintptr_t)A) >> 4;
    const uint64_t safe_hi = nv >= 1 ? nv - 1 : 0u;
    // cover byte h + 16j carries stream bit h + 16j: stream byte h/8 + 2j
    // (message byte m0 + 2j), cut at bit h % 8
    const uintptr_t m0 = (uintptr_t)a.msg + (h >> 3) - (a.header ? 4u : 0u);
    const uint32_t bsh = h & 7u;
    for (uint64_t r = j_lo + warp * 32u * V; r < j_hi; r += nwarps * 32u * V) {
        const uint64_t re = r + 32u * V; // one past the round's last vector
        const bool inside = re <= j_hi && r >= safe_lo && re <= safe_hi;
        if (inside && window_inner(a, h + (r << 4), h + ((re - 1) << 4))) {
            // the whole round inside the cover and the message
            const uint4 *__restrict__ Ar = A + r + lane;
            uint4 lo[V];
#pragma unroll
            for (int u = 0; u < V; ++u)
                lo[u] = __ldcs(Ar + 32u * u);
            uint4 x = make_uint4(0u, 0u, 0u, 0u);
            if (lane == 0)
                x = __ldcs(Ar + 32u * V);
            // stream bytes of vector j start at message byte m0 + 2j: the
            // same offset within an aligned word for all V vectors of a lane
            const uintptr_t pm = m0 + 2u * (r + lane);
            const uint32_t *__restrict__ wp = reinterpret_cast<const uint32_t *>(pm & ~(uintptr_t)3u);
            const uint32_t wsh = 8u * (uint32_t)(pm & 3u);
            uint32_t p[V];
#pragma unroll
            for (int u = 0; u < V; ++u)
                p[u] = bits16_from(__funnelshift_r(__ldg(wp + 16u * u), __ldg(wp + 16u * u + 1), wsh),
                                   bsh);
            uint4 *Dr = dst + r + lane;
#pragma unroll
            for (int u = 0; u < V; ++u) {
                const uint4 c = funnel16<Q>(lo[u], next_vec<V>(lo, x, u, lane), sel);
                const uint4 o = spread16(c, p[u]);
                if (STATS)
                    n += vec_changes(o, c);
                __stcs(Dr + 32u * u, o);
            }
            continue;
        }
        if (inside && h + (r << 4) >= a.t_bytes) {
            // the whole round past the carrying bytes: a copy
            const uint4 *__restrict__ Ar = A + r + lane;
            uint4 lo[V];
#pragma unroll
            for (int u = 0; u < V; ++u)
                lo[u] = __ldcs(Ar + 32u * u);
            uint4 x = make_uint4(0u, 0u, 0u, 0u);
            if (lane == 0)
                x = __ldcs(Ar + 32u * V);
            uint4 *Dr = dst + r + lane;
#pragma unroll
            for (int u = 0; u < V; ++u)
                __stcs(Dr + 32u * u, funnel16<Q>(lo[u], next_vec<V>(lo, x, u, lane), sel));
            continue;
        }
        // a round at an edge: one vector at a time, with the checks, out of
        // line (inlined, its registers doubled those of the batched kernel)
#pragma unroll 1
        for (int u = 0; u < V; ++u) {
            const uint64_t j = r + 32u * u + lane;
            if (j >= j_hi)
                break;
            n += funnel_edge_vec<Q, STATS>(a, h, sel, j);
        }
    }
    if (STATS) {
        changed += n;
        sse += n;
    }
}

// One byte k of a job (tails and unaligned buffers).
template <bool STATS>
__device__ __forceinline__ void embed_one(const EmbedView &a, uint64_t k, uint32_t s,
                                          unsigned long long &changed, unsigned long long &sse)
{
    const uint32_t cb = a.cover[k];
    uint32_t ob = cb;
    if (k < a.t_bytes)
        ob = (cb & 0xFEu) | ((s >> (7u - (uint32_t)(k & 7u))) & 1u);
    a.stego[k] = (uint8_t)ob;
    if (STATS) {
        const uint32_t d = ob > cb ? ob - cb : cb - ob;
        changed += d != 0;
        sse += d * d;
    }
}

// Bytes after the last whole vector (n_bytes % 16 of them), one per thread
// of the calling CTA.
template <bool STATS>
__device__ __forceinline__ void embed_tail(const EmbedView &a, unsigned long long &changed,
                                           unsigned long long &sse)
{
    if (threadIdx.x < (uint32_t)(a.n_bytes & 15u)) {
        const uint64_t k = ((a.n_bytes >> 4) << 4) + threadIdx.x;
        const uint32_t s = k < a.t_bytes ? stream_byte(a, k >> 3) : 0u;
        embed_one<STATS>(a, k, s, changed, sse);
    }
}

// Unaligned buffers: stream-byte units q = q_first + i*step (eight cover
// bytes each), q < q_end.
template <bool STATS>
__device__ __forceinline__ void embed_bytes_range(const EmbedView &a, uint64_t q_first,
                                                  uint64_t q_end, uint64_t step,
                                                  unsigned long long &changed,
                                                  unsigned long long &sse)
{
    for (uint64_t q = q_first; q < q_end; q += step) {
        const uint32_t s = q < a.slen ? stream_byte(a, q) : 0u;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const uint64_t k = (q << 3) + b;
            if (k >= a.n_bytes)
                break;
            embed_one<STATS>(a, k, s, changed, sse);
        }
    }
}

// Bit 0 of each byte of w, first byte as the most significant of a nibble.
// (w & 0x01010101) has bits at 0, 8, 16, 24; the multiplier's terms
// 2^27, 2^18, 2^9, 2^0 move them to bits 27, 26, 25, 24 and no other partial
// product lands in bits 24..31.
__device__ __forceinline__ uint32_t gather4(uint32_t w)
{
    return ((w & 0x01010101u) * 0x08040201u) >> 24;
}

// 16 stego bytes -> two message bytes, as m[2v] | m[2v+1] << 8.
__device__ __forceinline__ uint32_t gather16(const uint4 &c)
{
    const uint32_t s0 = (gather4(c.x) << 4) | gather4(c.y);
    const uint32_t s1 = (gather4(c.z) << 4) | gather4(c.w);
    return s0 | (s1 << 8);
}

// Vectors v (16 stego bytes from base + 16v) -> message bytes 2v, 2v+1, for
// v = v_first + i*step (+ u*blockDim.x), v < v_end; st + base 16-byte aligned.
template <int V>
__device__ __forceinline__ void extract_vec_range(const ExtractView &x, uint64_t v_first,
                                                  uint64_t v_end, uint64_t step)
{
    const uint4 *__restrict__ src = reinterpret_cast<const uint4 *>(x.st + x.base);
    unsigned short *mw = reinterpret_cast<unsigned short *>(x.msg);
    for (uint64_t v0 = v_first; v0 < v_end; v0 += step) {
        uint4 c[V];
        if (x.msg_even && v0 + (uint64_t)(V - 1) * blockDim.x < v_end) {
            // a whole round: no per-vector checks, 16-bit message stores
#pragma unroll
            for (int u = 0; u < V; ++u)
                c[u] = __ldcs(src + v0 + (uint64_t)u * blockDim.x);
#pragma unroll
            for (int u = 0; u < V; ++u)
                mw[v0 + (uint64_t)u * blockDim.x] = (unsigned short)gather16(c[u]);
            continue;
        }
#pragma unroll
        for (int u = 0; u < V; ++u) {
            const uint64_t v = v0 + (uint64_t)u * blockDim.x;
            if (v < v_end)
                c[u] = __ldcs(src + v);
        }
#pragma unroll
        for (int u = 0; u < V; ++u) {
            const uint64_t v = v0 + (uint64_t)u * blockDim.x;
            if (v >= v_end)
                continue;
            const uint32_t pair = gather16(c[u]);
            if (x.msg_even) {
                *reinterpret_cast<unsigned short *>(x.msg + 2 * v) = (unsigned short)pair;
            } else {
                x.msg[2 * v] = (uint8_t)pair;
                x.msg[2 * v + 1] = (uint8_t)(pair >> 8);
            }
        }
    }
}

// Message byte q from its eight stego bytes (tails and unaligned stegos).
__device__ __forceinline__ void extract_one(const ExtractView &x, uint64_t q)
{
    const uint8_t *p = x.st + x.base + (q << 3);
    uint32_t s = 0;
#pragma unroll
    for (int b = 0; b < 8; ++b)
        s |= (uint32_t)(p[b] & 1u) << (7 - b);
    x.msg[q] = (uint8_t)s;
}

__device__ __forceinline__ void extract_bytes_range(const ExtractView &x, uint64_t q_first,
                                                    uint64_t q_end, uint64_t step)
{
    for (uint64_t q = q_first; q < q_end; q += step)
        extract_one(x, q);
}

// The 16 LSBs of an aligned stego vector, its first byte's on top.
__device__ __forceinline__ uint32_t lsb16(const uint4 &c)
{
    return (gather4(c.x) << 12) | (gather4(c.y) << 8) | (gather4(c.z) << 4) | gather4(c.w);
}

// A misaligned stego (a = its carrying bytes' address mod 16), warp by warp:
// lane l of a round loads aligned vector r + 32u + l once and reduces it to
// its 16 LSBs; the pair starting a bytes into vector v takes the low 16 - a
// of them and the top a LSBs of vector v + 1, which come from the next lane
// by one shuffle (from lane 0 of the next unit, or a load of the last lane,
// at the end of a unit).  Pairs v in [v_lo, v_hi); warp `warp` of `nwarps`
// takes rounds of 32*V pairs.  Pairs whose two vectors are not both inside
// the stego go byte by byte.
template <int V>
__device__ __forceinline__ void extract_shift_lsb(const ExtractView &x, uint64_t C, uint64_t v_lo,
                                                  uint64_t v_hi, uint64_t warp, uint64_t nwarps)
{
    const uintptr_t p0 = (uintptr_t)(x.st + x.base);
    const uint32_t a = (uint32_t)(p0 & 15u);
    const uint4 *__restrict__ A = reinterpret_cast<const uint4 *>(p0 - a);
    const uintptr_t lo_ok = (uintptr_t)x.st, hi_ok = (uintptr_t)x.st + C;
    const uint32_t lane = threadIdx.x & 31u;
    // pairs [safe_lo, safe_hi) have both vectors inside the stego
    const uint64_t safe_lo = (uintptr_t)A >= lo_ok ? 0u : 1u;
    const uint64_t nv = (hi_ok - (uintptr_t)A) >> 4; // vectors of A inside the stego
    const uint64_t safe_hi = nv >= 1 ? (nv - 1 < v_hi ? nv - 1 : v_hi) : 0u;
    for (uint64_t r = v_lo + warp * 32u * V; r < v_hi; r += nwarps * 32u * V) {
        if (r >= safe_lo && r + 32u * V <= safe_hi) {
            // the whole round inside: no per-pair checks
            uint4 c[V];
#pragma unroll
            for (int u = 0; u < V; ++u)
                c[u] = __ldcs(A + r + (uint64_t)u * 32u + lane);
            uint4 e = make_uint4(0u, 0u, 0u, 0u);
            if (lane == 31u)
                e = __ldcs(A + r + (uint64_t)V * 32u);
            uint32_t L[V];
#pragma unroll
            for (int u = 0; u < V; ++u)
                L[u] = lsb16(c[u]);
            const uint32_t Le = lsb16(e);
#pragma unroll
            for (int u = 0; u < V; ++u) {
                uint32_t nx = __shfl_down_sync(0xFFFFFFFFu, L[u], 1);
                const uint32_t first =
                    u + 1 < V ? __shfl_sync(0xFFFFFFFFu, L[u + 1 < V ? u + 1 : u], 0) : Le;
                if (lane == 31u)
                    nx = first;
                const uint32_t bits = ((L[u] << a) | (nx >> (16u - a))) & 0xFFFFu;
                const uint32_t pair = (bits >> 8) | ((bits & 0xFFu) << 8);
                const uint64_t v = r + (uint64_t)u * 32u + lane;
                if (x.msg_even) {
                    *reinterpret_cast<unsigned short *>(x.msg + 2 * v) = (unsigned short)pair;
                } else {
                    x.msg[2 * v] = (uint8_t)pair;
                    x.msg[2 * v + 1] = (uint8_t)(pair >> 8);
                }
            }
            continue;
        }
        // a round at an edge: one unit at a time, with the checks
#pragma unroll 1
        for (int u = 0; u < V; ++u) {
            const uint64_t v = r + (uint64_t)u * 32u + lane;
            const uintptr_t b = (uintptr_t)(A + v);
            uint4 c = make_uint4(0u, 0u, 0u, 0u);
            if (v <= v_hi && b >= lo_ok && b + 16u <= hi_ok)
                c = __ldcs(A + v);
            const uint64_t ve = r + (uint64_t)u * 32u + 32u;
            const uintptr_t be = (uintptr_t)(A + ve);
            uint4 e = make_uint4(0u, 0u, 0u, 0u);
            if (lane == 31u && ve <= v_hi && be >= lo_ok && be + 16u <= hi_ok)
                e = __ldcs(A + ve);
            const uint32_t L = lsb16(c);
            uint32_t nx = __shfl_down_sync(0xFFFFFFFFu, L, 1);
            if (lane == 31u)
                nx = lsb16(e);
            if (v >= v_hi)
                continue;
            if (!(b >= lo_ok && b + 32u <= hi_ok)) {
                extract_one(x, 2 * v);
                extract_one(x, 2 * v + 1);
                continue;
            }
            const uint32_t bits = ((L << a) | (nx >> (16u - a))) & 0xFFFFu;
            const uint32_t pair = (bits >> 8) | ((bits & 0xFFu) << 8);
            if (x.msg_even) {
                *reinterpret_cast<unsigned short *>(x.msg + 2 * v) = (unsigned short)pair;
            } else {
                x.msg[2 * v] = (uint8_t)pair;
                x.msg[2 * v + 1] = (uint8_t)(pair >> 8);
            }
        }
    }
}

// Validity of a header value: the count must be whole bytes, fit the stego
// after the 32 header bytes, and fit the caller's buffer.
__device__ __forceinline__ int header_status(uint64_t C, uint64_t cap, uint32_t nbits)
{
    if (C < 32)
        return STEGO_E_BAD_HEADER;
    if (nbits & 7u)
        return STEGO_E_BAD_HEADER;
    if (32ull + nbits > C)
        return STEGO_E_BAD_HEADER;
    if ((uint64_t)(nbits >> 3) > cap)
        return STEGO_E_MSG_TOO_SMALL;
    return STEGO_OK;
}

// The 32-bit header, read by one whole warp: lane l loads stego byte l and a
// ballot of the LSBs gives the header bits with bit l = header bit 31-l, so
// the count is the bit-reversed ballot.  Every lane gets the value.
__device__ __forceinline__ uint32_t warp_read_header(const uint8_t *st, uint64_t C)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t byte = (lane < C) ? (uint32_t)st[lane] : 0u;
    return __brev(__ballot_sync(0xFFFFFFFFu, byte & 1u));
}

struct ExtractArgs {
    const uint8_t *st;
    uint64_t C;
    uint8_t *msg;
    uint64_t cap;
    uint64_t raw_len;
    uint32_t header;
    uint32_t msg_even;
    stego_result *res;
    uint64_t max_vec; // most 16-byte vectors the call can need (length bound)
};

// Length and status of the call: from the header (read by warp 0 of every
// CTA with one ballot) or the caller's length.  Block 0 publishes them.
__device__ __forceinline__ int extract_prologue(const ExtractArgs &a, ExtractView &x)
{
    __shared__ int s_status;
    __shared__ unsigned long long s_len;
    x.st = a.st;
    x.msg = a.msg;
    x.msg_even = a.msg_even;
    x.pad = 0;
    if (a.header) {
        if (threadIdx.x < 32) {
            const uint32_t nbits = s1::warp_read_header(a.st, a.C);
            if (threadIdx.x == 0) {
                const int st = s1::header_status(a.C, a.cap, nbits);
                s_status = st;
                s_len = st == STEGO_OK ? (nbits >> 3) : 0u;
            }
        }
        __syncthreads();
        x.len = s_len;
        x.base = 32;
    } else {
        if (threadIdx.x == 0) {
            s_status = STEGO_OK;
            s_len = a.raw_len;
        }
        __syncthreads();
        x.len = a.raw_len;
        x.base = 0;
    }
    const int status = s_status;
    if (a.res && blockIdx.x == 0 && threadIdx.x == 0) {
        a.res->changed = 0;
        a.res->sse = 0;
        a.res->msg_bytes = x.len;
        a.res->status = status;
        a.res->reserved = 0;
    }
    return status;
}

} // namespace s1
} // namespace stego
